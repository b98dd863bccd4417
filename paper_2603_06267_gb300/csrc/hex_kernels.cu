// CUDA kernels of the DG-SEM step on general hexahedra (trilinear elements).
//
// Setup (untimed, FP64): geometric factors and element masses at the GLL
// nodes, the assembled lumped mass, the face data of Algorithm 3 and the
// matching itself (normal filter, stored-vertex radius filter, Newton-Raphson
// reference position, containment), then the per-node interface data.
// Step (one launch each): element stiffness into element-local residual slots,
// SIPG interface terms into per-group slot blocks, residual assembly by a
// fixed-order gather over each node's slots fused with the leapfrog update of
// Algorithm 1, and the tail (PMUT forcing slots, receivers, step counter).
#include <cuda_runtime.h>

#include <type_traits>

#include "hex_geom.h"
#include "hex_step.cuh"

namespace hex {

// ---------------------------------------------------------------------------
// Setup kernels
// ---------------------------------------------------------------------------
__global__ void geom_kernel(const __grid_constant__ GeomArgs a) {
  const int n = a.n, nl = n * n * n;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)a.ne * nl) return;
  const int e = (int)(t / nl), i = (int)(t - (long long)e * nl);
  const int ia = i % n, ib = (i / n) % n, ic = i / (n * n);
  double V[24];
  for (int c = 0; c < 8; ++c) {
    const long long v = a.elem[8LL * e + c];
    V[3 * c] = a.vert[3 * v];
    V[3 * c + 1] = a.vert[3 * v + 1];
    V[3 * c + 2] = a.vert[3 * v + 2];
  }
  const double r[3] = {a.xi[ia], a.xi[ib], a.xi[ic]};
  double X[3], J[3][3], Ji[3][3];
  tri_map(V, r, X, J);
  const double det = inv3(J, Ji);
  if (!(det > 0.0)) atomicAdd(a.bad, 1);
  const double wq = a.w[ia] * a.w[ib] * a.w[ic];
  const double s = a.c2 * wq * det;
  const int comp[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int k = 0; k < 6; ++k) {
    const int d = comp[k][0], f = comp[k][1];
    const double g = s * (Ji[d][0] * Ji[f][0] + Ji[d][1] * Ji[f][1] + Ji[d][2] * Ji[f][2]);
    const long long o = (6LL * e + k) * gstride(n) + i;
    a.G64[o] = g;
    a.G32[o] = (float)g;
  }
  a.Mloc[(long long)e * nl + i] = wq * det;
}

// Lumped mass M_jj = sum of the element masses at node j (its volume slots,
// which come first in its ascending slot list).
__global__ void mass_kernel(const double* Mloc, const int* ptr, const int* slot, long long nvol, long long ndof,
                            double* Minv64, float* Minv32, double* M) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= ndof) return;
  double m = 0.0;
  for (int k = ptr[j]; k < ptr[j + 1]; ++k) {
    const int s = slot[k];
    if (s >= nvol) break;
    m += Mloc[s];
  }
  M[j] = m;
  Minv64[j] = 1.0 / m;
  Minv32[j] = (float)(1.0 / m);
}

__global__ void face_kernel(const __grid_constant__ FaceArgs a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= a.nf) return;
  const int e = a.faces[2 * f], lf = a.faces[2 * f + 1];
  double V[24];
  for (int c = 0; c < 8; ++c) {
    const long long v = a.elem[8LL * e + c];
    for (int k = 0; k < 3; ++k) V[3 * c + k] = a.vert[3 * v + k];
  }
  const int ax = lf >> 1, side = lf & 1;
  int cs[4], nc = 0;
  for (int c = 0; c < 8; ++c)
    if (((c >> ax) & 1) == side) cs[nc++] = c;
  double diam = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double d = V[3 * cs[i] + k] - V[3 * cs[j] + k];
        d2 += d * d;
      }
      diam = fmax(diam, sqrt(d2));
    }
  double r[3], X[3], J[3][3], nrm[3];
  face_ref(lf, 0.0, 0.0, r);
  tri_map(V, r, X, J);
  face_normal(lf, J, nrm);
  double area = 0.0;
  for (int tb = 0; tb < a.n; ++tb)
    for (int sa = 0; sa < a.n; ++sa) {
      face_ref(lf, a.xi[sa], a.xi[tb], r);
      tri_map(V, r, X, J);
      double nn[3];
      area += a.w[sa] * a.w[tb] * face_normal(lf, J, nn);
    }
  const int nl = a.n * a.n * a.n;
  double vol = 0.0;
  for (int i = 0; i < nl; ++i) vol += a.Mloc[(long long)e * nl + i];
  double* o = a.out + 8LL * f;
  o[0] = nrm[0]; o[1] = nrm[1]; o[2] = nrm[2];
  o[3] = V[3 * cs[0]]; o[4] = V[3 * cs[0] + 1]; o[5] = V[3 * cs[0] + 2];
  o[6] = diam;
  o[7] = vol / area;
}

// Algorithm 3, one thread per Gauss node of a fine face: the first coarse face
// (list order) whose centre normal is opposite within tol, whose stored vertex
// is within max(diam) + eps of the node, and whose element contains the node.
__global__ void match_kernel(const __grid_constant__ MatchArgs a) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int qq = a.q * a.q;
  if (t >= (long long)a.nff * qq) return;
  const int f = (int)(t / qq), j = (int)(t - (long long)f * qq);
  const int e = a.ff[2 * f], lf = a.ff[2 * f + 1];
  double V[24];
  for (int c = 0; c < 8; ++c) {
    const long long v = a.elem_p[8LL * e + c];
    for (int k = 0; k < 3; ++k) V[3 * c + k] = a.vert_p[3 * v + k];
  }
  double r[3], x[3], J[3][3];
  face_ref(lf, a.g[j % a.q], a.g[j / a.q], r);
  tri_map(V, r, x, J);
  const double* fd = a.fdat + 8LL * f;
  int found = -1;
  double rm[3] = {0.0, 0.0, 0.0};
  for (int g = 0; g < a.ncf && found < 0; ++g) {
    const double* cd = a.cdat + 8LL * g;
    const double s0 = fd[0] + cd[0], s1 = fd[1] + cd[1], s2 = fd[2] + cd[2];
    if (!(sqrt(s0 * s0 + s1 * s1 + s2 * s2) < a.tol)) continue;
    const double d0 = cd[3] - x[0], d1 = cd[4] - x[1], d2 = cd[5] - x[2];
    if (sqrt(d0 * d0 + d1 * d1 + d2 * d2) > fmax(fd[6], cd[6]) + a.eps) continue;
    const int ec = a.cf[2 * g];
    double W[24];
    for (int c = 0; c < 8; ++c) {
      const long long v = a.elem_m[8LL * ec + c];
      for (int k = 0; k < 3; ++k) W[3 * c + k] = a.vert_m[3 * v + k];
    }
    double rr[3];
    if (newton_ref(W, x, rr) && inside_ref(rr)) {
      found = g;
      rm[0] = rr[0]; rm[1] = rr[1]; rm[2] = rr[2];
    }
  }
  a.match[t] = found;
  a.refm[3 * t] = rm[0];
  a.refm[3 * t + 1] = rm[1];
  a.refm[3 * t + 2] = rm[2];
}

// Interface data of every matched fine Gauss node: outward normal n+ of the
// fine face, a+- = J+-^-1 n+ (so that d psi / d n+ = grad^ psi . a), the
// weight w_s w_t |J+| |J+^-T e|, and gamma_F with h = min(|K|/|F|) of the two
// faces.
__global__ void ipoint_kernel(const __grid_constant__ MatchArgs a) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int qq = a.q * a.q;
  if (t >= (long long)a.nff * qq) return;
  const int g = a.match[t];
  if (g < 0) return;
  const int f = (int)(t / qq), j = (int)(t - (long long)f * qq);
  const int e = a.ff[2 * f], lf = a.ff[2 * f + 1];
  double V[24], W[24];
  for (int c = 0; c < 8; ++c) {
    const long long v = a.elem_p[8LL * e + c];
    for (int k = 0; k < 3; ++k) V[3 * c + k] = a.vert_p[3 * v + k];
  }
  const int ec = a.cf[2 * g];
  for (int c = 0; c < 8; ++c) {
    const long long v = a.elem_m[8LL * ec + c];
    for (int k = 0; k < 3; ++k) W[3 * c + k] = a.vert_m[3 * v + k];
  }
  const int is = j % a.q, it = j / a.q;
  double rp[3], x[3], Jp[3][3], Jpi[3][3], nrm[3];
  face_ref(lf, a.g[is], a.g[it], rp);
  tri_map(V, rp, x, Jp);
  const double dS = face_normal(lf, Jp, nrm);
  inv3(Jp, Jpi);
  const double* rm = a.refm + 3 * t;
  double Jm[3][3], Jmi[3][3], xm[3];
  tri_map(W, rm, xm, Jm);
  inv3(Jm, Jmi);
  double* o = a.pdat + (long long)PDAT * t;
  for (int k = 0; k < 3; ++k) {
    o[k] = rp[k];
    o[3 + k] = rm[k];
    o[6 + k] = Jpi[k][0] * nrm[0] + Jpi[k][1] * nrm[1] + Jpi[k][2] * nrm[2];
    o[9 + k] = Jmi[k][0] * nrm[0] + Jmi[k][1] * nrm[1] + Jmi[k][2] * nrm[2];
  }
  o[12] = a.gw[is] * a.gw[it] * dS;
  o[13] = a.alpha_cbar2_n2 / fmin(a.fdat[8LL * f + 7], a.cdat[8LL * g + 7]);
}

// ---------------------------------------------------------------------------
// Step kernels
// ---------------------------------------------------------------------------

// SIPG interface terms of eq. (Wf_2) for one group of fine Gauss nodes that
// share a fine element K+ and a coarse element K-.  With jump J = p+ - p-
// and A = 1/2 (c+^2 dp+/dn+ + c-^2 dp-/dn+):
//   r_i(K+) += W (gamma J - A) psi_i - 1/2 W J c+^2 d psi_i / d n+
//   r_i(K-) -= W (gamma J - A) psi_i + 1/2 W J c-^2 d psi_i / d n+
template <typename T, int BB>
__global__ void __launch_bounds__(128) hex_iface_kernel(const __grid_constant__ HexIfaceArgs<T> A) {
  using P = Pack<T, BB>;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const int g = blockIdx.x;
  const int np = A.np, nm = A.nm;
  const int nlp = np * np * np, nlm = nm * nm * nm;
  const int p0 = A.g_pt[g], npts = A.g_pt[g + 1] - p0;
  const int Q = A.max_pts;
  P* up = reinterpret_cast<P*>(smem_raw);
  P* um = up + nlp;
  P* sv = um + nlm;                 // [Q]
  P* sd = sv + Q;                   // [Q]
  T* tp = reinterpret_cast<T*>(sd + Q);   // [Q][3][2][np]: l, l' per axis, fine side
  T* tm = tp + (long long)Q * 6 * np;     // [Q][3][2][nm]
  T* av = tm + (long long)Q * 6 * nm;     // [Q][8]: a+(3) a-(3) W gamma
  const int tid = threadIdx.x;
  {
    // the group's rows of the per-point tables (built once at setup), into
    // the per-order strides of the shared arrays
    const T* trow = A.gtab + (long long)p0 * kGenTab;
    for (int i = tid; i < npts * kGenTab; i += blockDim.x) {
      const int j = i / kGenTab, c = i - j * kGenTab;
      const T v = trow[i];
      if (c < 12 * MAXN1) {
        const int side = c / (6 * MAXN1), r = (c / MAXN1) % 6, k = c % MAXN1;   // r = 2 axis + (0: l, 1: l')
        if (side == 0 && k < np) tp[(j * 6 + r) * np + k] = v;
        else if (side == 1 && k < nm) tm[(j * 6 + r) * nm + k] = v;
      } else {
        av[8 * j + c - 12 * MAXN1] = v;
      }
    }
  }
  const int fe = A.g_fe[g], ce = A.g_ce[g];
  const long long slot = A.g_slot[g];
  const T c2p = T(A.c2p), c2m = T(A.c2m);
  const int nch = A.Bp / BB;
  for (int ch = 0; ch < nch; ++ch) {
    for (int i = tid; i < nlp; i += blockDim.x)
      up[i] = reinterpret_cast<const P*>(A.p + (long long)A.conn_p[(long long)fe * nlp + i] * A.Bp)[ch];
    for (int i = tid; i < nlm; i += blockDim.x)
      um[i] = reinterpret_cast<const P*>(A.p + (long long)A.conn_m[(long long)ce * nlm + i] * A.Bp)[ch];
    __syncthreads();
    for (int j = tid; j < npts; j += blockDim.x) {
      T vp[BB], dp0[BB], dp1[BB], dp2[BB], vm[BB], dm0[BB], dm1[BB], dm2[BB];
#pragma unroll
      for (int b = 0; b < BB; ++b) vp[b] = dp0[b] = dp1[b] = dp2[b] = vm[b] = dm0[b] = dm1[b] = dm2[b] = T(0);
      {
        const T* lx = tp + (j * 3 + 0) * 2 * np;
        const T* ly = tp + (j * 3 + 1) * 2 * np;
        const T* lz = tp + (j * 3 + 2) * 2 * np;
        for (int c = 0; c < np; ++c)
          for (int bb = 0; bb < np; ++bb) {
            T s0[BB], s1[BB];
#pragma unroll
            for (int b = 0; b < BB; ++b) s0[b] = s1[b] = T(0);
            for (int a = 0; a < np; ++a) {
              const P uv = up[(c * np + bb) * np + a];
              const T la = lx[a], da = lx[np + a];
#pragma unroll
              for (int b = 0; b < BB; ++b) {
                s0[b] = fma_(la, uv.v[b], s0[b]);
                s1[b] = fma_(da, uv.v[b], s1[b]);
              }
            }
            const T yz = mul_(ly[bb], lz[c]), dyz = mul_(ly[np + bb], lz[c]), ydz = mul_(ly[bb], lz[np + c]);
#pragma unroll
            for (int b = 0; b < BB; ++b) {
              vp[b] = fma_(yz, s0[b], vp[b]);
              dp0[b] = fma_(yz, s1[b], dp0[b]);
              dp1[b] = fma_(dyz, s0[b], dp1[b]);
              dp2[b] = fma_(ydz, s0[b], dp2[b]);
            }
          }
      }
      {
        const T* lx = tm + (j * 3 + 0) * 2 * nm;
        const T* ly = tm + (j * 3 + 1) * 2 * nm;
        const T* lz = tm + (j * 3 + 2) * 2 * nm;
        for (int c = 0; c < nm; ++c)
          for (int bb = 0; bb < nm; ++bb) {
            T s0[BB], s1[BB];
#pragma unroll
            for (int b = 0; b < BB; ++b) s0[b] = s1[b] = T(0);
            for (int a = 0; a < nm; ++a) {
              const P uv = um[(c * nm + bb) * nm + a];
              const T la = lx[a], da = lx[nm + a];
#pragma unroll
              for (int b = 0; b < BB; ++b) {
                s0[b] = fma_(la, uv.v[b], s0[b]);
                s1[b] = fma_(da, uv.v[b], s1[b]);
              }
            }
            const T yz = mul_(ly[bb], lz[c]), dyz = mul_(ly[nm + bb], lz[c]), ydz = mul_(ly[bb], lz[nm + c]);
#pragma unroll
            for (int b = 0; b < BB; ++b) {
              vm[b] = fma_(yz, s0[b], vm[b]);
              dm0[b] = fma_(yz, s1[b], dm0[b]);
              dm1[b] = fma_(dyz, s0[b], dm1[b]);
              dm2[b] = fma_(ydz, s0[b], dm2[b]);
            }
          }
      }
      const T* a8 = av + 8 * j;
      P s, dd;
#pragma unroll
      for (int b = 0; b < BB; ++b) {
        const T jump = sub_(vp[b], vm[b]);
        const T dnp = fma_(dp2[b], a8[2], fma_(dp1[b], a8[1], mul_(dp0[b], a8[0])));
        const T dnm = fma_(dm2[b], a8[5], fma_(dm1[b], a8[4], mul_(dm0[b], a8[3])));
        const T avg = mul_(T(0.5), add_(mul_(c2p, dnp), mul_(c2m, dnm)));
        s.v[b] = mul_(a8[6], sub_(mul_(a8[7], jump), avg));
        dd.v[b] = mul_(mul_(T(-0.5), a8[6]), jump);
      }
      sv[j] = s;
      sd[j] = dd;
    }
    __syncthreads();
    for (int i = tid; i < nlp + nlm; i += blockDim.x) {
      const bool plus = i < nlp;
      const int n = plus ? np : nm;
      const int k = plus ? i : i - nlp;
      const int ia = k % n, ib = (k / n) % n, ic = k / (n * n);
      const T* tb = plus ? tp : tm;
      const T c2 = plus ? c2p : c2m;
      const T sgn = plus ? T(1) : T(-1);
      T r[BB];
#pragma unroll
      for (int b = 0; b < BB; ++b) r[b] = T(0);
      for (int j = 0; j < npts; ++j) {
        const T* lx = tb + (j * 3 + 0) * 2 * n;
        const T* ly = tb + (j * 3 + 1) * 2 * n;
        const T* lz = tb + (j * 3 + 2) * 2 * n;
        const T* a8 = av + 8 * j + (plus ? 0 : 3);
        const T psi = mul_(sgn, mul_(mul_(lx[ia], ly[ib]), lz[ic]));
        const T t0 = mul_(mul_(lx[n + ia], ly[ib]), lz[ic]);
        const T t1 = mul_(mul_(lx[ia], ly[n + ib]), lz[ic]);
        const T t2 = mul_(mul_(lx[ia], ly[ib]), lz[n + ic]);
        const T dn = mul_(c2, fma_(a8[2], t2, fma_(a8[1], t1, mul_(a8[0], t0))));
        const P s = sv[j], dd = sd[j];
#pragma unroll
        for (int b = 0; b < BB; ++b) r[b] = fma_(dd.v[b], dn, fma_(s.v[b], psi, r[b]));
      }
      P o;
#pragma unroll
      for (int b = 0; b < BB; ++b) o.v[b] = r[b];
      reinterpret_cast<P*>(A.S + (slot + i) * A.Bp)[ch] = o;
    }
    __syncthreads();
  }
}

// Interface terms when every Gauss node of a group lies on one face of K+
// and on one face of K- (a geometrically conforming interface): on a face,
// psi_abc = delta_{c,face} l_a l_b and d psi / d xi_normal = l_a l_b l_c'(+-1),
// so each side first collapses to two face arrays (the face layer u_f and the
// normal derivative u_n = sum_c l_c'(+-1) u_abc), the Gauss-node values and
// reference gradients cost O(n^2) each, and the projection back collapses the
// same way: R_f (value and tangential terms) on the face layer and R_n (the
// normal-derivative term) spread along each normal line by l_c'(+-1).
// Per-point tables of the general interface kernel (setup, once per
// precision): for each side, the 1-D Lagrange values and derivatives along
// its three reference axes at the node's reference coordinates, then the
// normal's reference components a+ and a-, W and gamma; row p0 + j of group g.
template <typename T>
__global__ void __launch_bounds__(128) iface_gtable_kernel(const __grid_constant__ HexIfaceArgs<T> A, T* tab) {
  const int g = blockIdx.x;
  const int p0 = A.g_pt[g], npts = A.g_pt[g + 1] - p0;
  for (int j = threadIdx.x; j < npts; j += blockDim.x) {
    T* row = tab + (long long)(p0 + j) * kGenTab;
    const double* d = A.pdat + (long long)PDAT * A.pt_idx[p0 + j];
    double l[MAXN1], dl[MAXN1];
    for (int side = 0; side < 2; ++side) {
      const int n = side ? A.nm : A.np;
      for (int ax = 0; ax < 3; ++ax) {
        lagrange(n, side ? A.xim : A.xip, d[3 * side + ax], l, dl);
        T* r = row + (side * 6 + ax * 2) * MAXN1;
        for (int k = 0; k < MAXN1; ++k) {
          r[k] = k < n ? T(l[k]) : T(0);
          r[MAXN1 + k] = k < n ? T(dl[k]) : T(0);
        }
      }
    }
    for (int k = 0; k < 8; ++k) row[12 * MAXN1 + k] = T(d[6 + k]);
  }
}

// Per-point tables of the face-collapsed interface kernel (setup, once per
// precision): for each side, the 1-D Lagrange values and derivatives along
// the two axes of its face at the node's reference coordinate, c^2 times the
// normal's reference components, then W and gamma; row p0 + j of group g.
template <typename T>
__global__ void __launch_bounds__(128) iface_table_kernel(const __grid_constant__ HexIfaceArgs<T> A, T* tab) {
  const int g = blockIdx.x;
  const int np = A.np, nm = A.nm;
  const int p0 = A.g_pt[g], npts = A.g_pt[g + 1] - p0;
  const int fp = A.g_face[2 * g], fm = A.g_face[2 * g + 1];
  for (int j = threadIdx.x; j < npts; j += blockDim.x) {
    T* tb = tab + (long long)(p0 + j) * kFaceTab;
    T* av = tb + 8 * MAXN1;
    const double* d = A.pdat + (long long)PDAT * A.pt_idx[p0 + j];
    double l[MAXN1], dl[MAXN1];
    for (int side = 0; side < 2; ++side) {
      const int f = side ? fm : fp, n = side ? nm : np, ax = f >> 1;
      const int t0 = ax == 0 ? 1 : 0, t1 = ax == 2 ? 1 : 2;
      const int ta[2] = {t0, t1};
      const double* ref = d + 3 * side;
      for (int k = 0; k < 2; ++k) {
        lagrange(n, side ? A.xim : A.xip, ref[ta[k]], l, dl);
        T* row = tb + (side * 2 + k) * 2 * MAXN1;
        for (int i = 0; i < MAXN1; ++i) {
          row[i] = i < n ? T(l[i]) : T(0);
          row[MAXN1 + i] = i < n ? T(dl[i]) : T(0);
        }
      }
      const double c2 = side ? A.c2m : A.c2p;
      const double* a = d + 6 + 3 * side;
      av[3 * side] = T(c2 * a[t0]);
      av[3 * side + 1] = T(c2 * a[t1]);
      av[3 * side + 2] = T(c2 * a[ax]);
    }
    av[6] = T(d[12]);
    av[7] = T(d[13]);
  }
}

template <typename T, int BB>
__global__ void __launch_bounds__(128) hex_iface_face_kernel(const __grid_constant__ HexIfaceArgs<T> A) {
  using P = Pack<T, BB>;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const int g = blockIdx.x;
  const int np = A.np, nm = A.nm;
  const int nlp = np * np * np, nlm = nm * nm * nm;
  const int p0 = A.g_pt[g], npts = A.g_pt[g + 1] - p0;
  const int Q = A.max_pts;
  P* up = reinterpret_cast<P*>(smem_raw);
  P* um = up + nlp;
  P* cf = um + nlm;                      // [np^2] u_f+, [np^2] u_n+, [nm^2] u_f-, [nm^2] u_n-
  P* pv = cf + 2 * (np * np + nm * nm);  // [Q][4]: value and d/dn+ of each side
  P* sv = pv + 4 * Q;                    // [Q]
  P* sd = sv + Q;                        // [Q]
  T* tb = reinterpret_cast<T*>(sd + Q);  // [Q][2 sides][2 axes][2][MAXN1]: l, l' along the face axes
  T* av = tb + (long long)Q * 8 * MAXN1; // [Q][8]: c+^2 a+ (t0, t1, n), c-^2 a- (t0, t1, n), W, gamma
  const int tid = threadIdx.x;
  const int fp = A.g_face[2 * g], fm = A.g_face[2 * g + 1];
  {
    // the group's rows of the per-point tables (built once at setup)
    const T* trow = A.ftab + (long long)p0 * kFaceTab;
    for (int i = tid; i < npts * kFaceTab; i += blockDim.x) {
      const int r = i / kFaceTab, c = i - r * kFaceTab;
      const T v = trow[i];
      if (c < 8 * MAXN1) tb[r * 8 * MAXN1 + c] = v;
      else av[r * 8 + c - 8 * MAXN1] = v;
    }
  }
  const int fe = A.g_fe[g], ce = A.g_ce[g];
  const long long slot = A.g_slot[g];
  const int nch = A.Bp / BB;
  for (int ch = 0; ch < nch; ++ch) {
    for (int i = tid; i < nlp; i += blockDim.x)
      up[i] = reinterpret_cast<const P*>(A.p + (long long)A.conn_p[(long long)fe * nlp + i] * A.Bp)[ch];
    for (int i = tid; i < nlm; i += blockDim.x)
      um[i] = reinterpret_cast<const P*>(A.p + (long long)A.conn_m[(long long)ce * nlm + i] * A.Bp)[ch];
    __syncthreads();
    // collapse each side to its face layer and normal derivative
    for (int t = tid; t < np * np + nm * nm; t += blockDim.x) {
      const bool plus = t < np * np;
      const int n = plus ? np : nm, k = plus ? t : t - np * np;
      const int f = plus ? fp : fm, ax = f >> 1;
      const int s[3] = {1, n, n * n};
      const int st0 = s[ax == 0 ? 1 : 0], st1 = s[ax == 2 ? 1 : 2], sn = s[ax];
      const int fi = (f & 1) ? n - 1 : 0;
      const int base = (k % n) * st0 + (k / n) * st1;
      const P* u = plus ? up : um;
      const T(*D)[MAXN1] = plus ? A.Dp : A.Dm;
      P un = vmul(D[fi][0], u[base]);
      for (int c = 1; c < n; ++c) vfma(un, D[fi][c], u[base + c * sn]);
      P* dst = cf + (plus ? 0 : 2 * np * np);
      dst[k] = u[base + fi * sn];
      dst[n * n + k] = un;
    }
    __syncthreads();
    // value and normal derivative (d/dn+) of each side at each Gauss node
    for (int t = tid; t < 2 * npts; t += blockDim.x) {
      const int side = t >= npts, j = side ? t - npts : t;
      const int n = side ? nm : np;
      const P* uf = cf + (side ? 2 * np * np : 0);
      const P* un = uf + n * n;
      const T* L0 = tb + ((j * 2 + side) * 2 + 0) * 2 * MAXN1;
      const T* L1 = tb + ((j * 2 + side) * 2 + 1) * 2 * MAXN1;
      P v = vzero<T, BB>(), d0 = vzero<T, BB>(), d1 = vzero<T, BB>(), dn = vzero<T, BB>();
      for (int i1 = 0; i1 < n; ++i1) {
        P s0 = vzero<T, BB>(), s1 = vzero<T, BB>(), sn = vzero<T, BB>();
        for (int i0 = 0; i0 < n; ++i0) {
          const P a = uf[i0 + n * i1], b = un[i0 + n * i1];
          vfma(s0, L0[i0], a);
          vfma(s1, L0[MAXN1 + i0], a);
          vfma(sn, L0[i0], b);
        }
        vfma(v, L1[i1], s0);
        vfma(d0, L1[i1], s1);
        vfma(d1, L1[MAXN1 + i1], s0);
        vfma(dn, L1[i1], sn);
      }
      // c^2 dp/dn+ = c^2 (a_t0 d0 + a_t1 d1 + a_n dn)
      const T* a = av + 8 * j + 3 * side;
      P w = vmul(a[0], d0);
      vfma(w, a[1], d1);
      vfma(w, a[2], dn);
      pv[4 * j + 2 * side] = v;
      pv[4 * j + 2 * side + 1] = w;
    }
    __syncthreads();
    for (int j = tid; j < npts; j += blockDim.x) {
      const T W = av[8 * j + 6], gam = av[8 * j + 7];
      const P jump = vsub(pv[4 * j], pv[4 * j + 2]);
      // A = 1/2 (c+^2 dp+/dn+ + c-^2 dp-/dn+)
      const P avg = vmul(T(0.5), vadd(pv[4 * j + 1], pv[4 * j + 3]));
      sv[j] = vmul(W, vsub(vmul(gam, jump), avg));
      sd[j] = vmul(mul_(T(-0.5), W), jump);
    }
    __syncthreads();
    // projection back onto each side's element: face arrays, then normal lines
    for (int t = tid; t < np * np + nm * nm; t += blockDim.x) {
      const bool plus = t < np * np;
      const int side = plus ? 0 : 1;
      const int n = plus ? np : nm, k = plus ? t : t - np * np;
      const int i0 = k % n, i1 = k / n;
      const T sgn = plus ? T(1) : T(-1);
      P Rf = vzero<T, BB>(), Rn = vzero<T, BB>();
      for (int j = 0; j < npts; ++j) {
        const T* L0 = tb + ((j * 2 + side) * 2 + 0) * 2 * MAXN1;
        const T* L1 = tb + ((j * 2 + side) * 2 + 1) * 2 * MAXN1;
        const T* a = av + 8 * j + 3 * side;
        const T psi = mul_(L0[i0], L1[i1]);
        const T gt = fma_(a[1], mul_(L0[i0], L1[MAXN1 + i1]), mul_(a[0], mul_(L0[MAXN1 + i0], L1[i1])));
        const T gn = mul_(a[2], psi);
        vfma(Rf, mul_(sgn, psi), sv[j]);
        vfma(Rf, gt, sd[j]);
        vfma(Rn, gn, sd[j]);
      }
      const int f = plus ? fp : fm, ax = f >> 1;
      const int s[3] = {1, n, n * n};
      const int st0 = s[ax == 0 ? 1 : 0], st1 = s[ax == 2 ? 1 : 2], sn = s[ax];
      const int fi = (f & 1) ? n - 1 : 0;
      const T(*D)[MAXN1] = plus ? A.Dp : A.Dm;
      const long long sb = slot + (plus ? 0 : nlp) + i0 * st0 + i1 * st1;
      for (int c = 0; c < n; ++c) {
        P r = vmul(D[fi][c], Rn);
        if (c == fi) r = vadd(r, Rf);
        reinterpret_cast<P*>(A.S + (sb + (long long)c * sn) * A.Bp)[ch] = r;
      }
    }
    __syncthreads();
  }
}

// Residual assembly and leapfrog update, one thread per (node, BB members):
// r = sum of the node's slots (ascending slot order, so the sum is the same
// in every run and for every batch width), v += cv (damp v + M^-1 r),
// p_out = p_in + cp v.
template <typename T, int BB>
__global__ void __launch_bounds__(256) hex_update_kernel(const __grid_constant__ HexUpdateArgs<T> A) {
  using P = Pack<T, BB>;
  const int nch = A.Bp / BB;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long j = t / nch;
  if (j >= A.ndof) return;
  const int ch = (int)(t - j * nch);
  const int k0 = A.node_ptr[j], k1 = A.node_ptr[j + 1];
  const T mi = A.Minv[j];
  P r = vzero<T, BB>();
  for (int k = k0; k < k1; ++k) r = vadd(r, reinterpret_cast<const P*>(A.S + (long long)A.node_slot[k] * A.Bp)[ch]);
  P* vp = reinterpret_cast<P*>(A.v + j * A.Bp) + ch;
  const P pin = reinterpret_cast<const P*>(A.p_in + j * A.Bp)[ch];
  P pv = pin, vv = *vp;
  // damping on the predicted velocity: C p'_pred of Algorithm 1, alpha p'_pred of a layer
  if (A.damp) vfma(vv, mul_(A.cv, A.damp[j]), P(vv));
  if (A.psi) {
    // layer terms beta p^{n+1} + gamma psi^{n+1}, psi^{n+1} = psi^{n+1/2} + dt/2 p^{n+1}
    P* sp = reinterpret_cast<P*>(A.psi + j * A.Bp) + ch;
    const P ps = *sp;
    P psi_int = ps;
    vfma(psi_int, A.hpsi, pin);
    vfma(vv, mul_(A.cv, A.beta[j]), pin);
    vfma(vv, mul_(A.cv, A.gamma[j]), psi_int);
    P pn = ps;
    vfma(pn, A.dpsi, pin);
    *sp = pn;
  }
  vfma(vv, mul_(A.cv, mi), r);
  vfma(pv, A.cp, vv);
  *vp = vv;
  reinterpret_cast<P*>(A.p_out + j * A.Bp)[ch] = pv;
}

__device__ __forceinline__ double hex_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) hex_tail_kernel(const __grid_constant__ HexTailArgs<T> A) {
  const int n = A.n + (A.step ? *A.step : 0);
  if ((int)blockIdx.x < A.fblocks) {
    // forcing slot of footprint entry e: kappa sum_m q''_km B_em (= -f, eq. f_i)
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < (long long)A.nnz * A.B) {
      const int e = (int)(t / A.B), b = (int)(t - (long long)e * A.B);
      const int k = A.ent_k[e];
      const double* q = A.qdd + ((long long)b * A.K + k) * A.M;
      const double* Bv = A.Bm + (long long)e * A.M;
      double s = 0.0;
      for (int m = 0; m < A.M; ++m) s += q[m] * Bv[m];
      A.S[(A.fslot + e) * A.Bp + b] = T(A.kappa * s);
    }
  } else {
    const int warp = (int)(((blockIdx.x - A.fblocks) * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp < A.B * A.R) {
      const int b = warp / A.R, r = warp - b * A.R;
      const double* w = A.rw + (long long)r * A.rstride;
      const long long* off = A.roff + (long long)r * A.rstride;
      double s = 0.0;
      for (int t = lane; t < A.rnn[r]; t += 32) s += w[t] * (double)A.p[off[t] * A.Bp + b];
      s = hex_warp_sum(s);
      if (lane == 0) A.traces[b * A.tbs + r * A.trs + n] = s;
    }
  }
  // the last block to finish advances the step counter (every block has read it)
  if (A.step) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned done = atomicAdd(A.done, 1u);
      if (done == gridDim.x - 1) {
        *A.done = 0u;
        *A.step = *A.step + 1;
        __threadfence();
      }
    }
  }
}

// Perfectly matched layer of eq. (full_problem) rows 1-3 on one element (the
// reading of the box path): at every GLL node the physical gradients of
// p^{n+1} and psi^{n+1} = psi^{n+1/2} + dt/2 p^{n+1} (J^-T grad^),
//   Phi_d <- [(1 - dt z_d/2) Phi_d + dt c^2 ((alpha - 2 z_d) dp/dx_d
//            + z_e z_f dpsi/dx_d)] / (1 + dt z_d/2),
// and the element residual sum_q w |J| (Phi^{n+1/2} + Phi^{n+3/2})/2 . grad psi_j.
template <typename T, int BB>
__global__ void __launch_bounds__(1024) hex_pml_kernel(const __grid_constant__ HexPmlArgs<T> A, int n) {
  using P = Pack<T, BB>;
  extern __shared__ __align__(32) unsigned char smem_raw[];
  const int nl = n * n * n;
  P* u = reinterpret_cast<P*>(smem_raw);   // p^{n+1}
  P* w = u + nl;                           // psi^{n+1}
  P* F = w + nl;                           // [3][nl]
  T* D = reinterpret_cast<T*>(F + 3 * nl); // [n][n]
  const int i = threadIdx.x;
  const int ep = blockIdx.x;
  const int e = A.elem[ep];
  if (i < n * n) D[i] = A.D[i / n][i % n];
  const bool act = i < nl;
  const int ia = i % n, ib = (i / n) % n, ic = i / (n * n);
  long long node = 0;
  T Ji[9], wJ = T(0), z[3] = {T(0), T(0), T(0)};
  if (act) {
    node = A.conn[(long long)e * nl + i];
    const T* g = A.geo + (long long)ep * 10 * nl + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) Ji[k] = g[(long long)k * nl];
    wJ = g[9LL * nl];
#pragma unroll
    for (int d = 0; d < 3; ++d) z[d] = A.zeta[d * A.ndof + node];
  }
  const T alpha = add_(add_(z[0], z[1]), z[2]);
  const T h = mul_(T(0.5), A.dt);
  const int nch = A.Bp / BB;
  for (int ch = 0; ch < nch; ++ch) {
    if (act) {
      const P pv = reinterpret_cast<const P*>(A.p + node * A.Bp)[ch];
      P sv = reinterpret_cast<const P*>(A.psi + node * A.Bp)[ch];
      vfma(sv, h, pv);
      u[i] = pv;
      w[i] = sv;
    }
    __syncthreads();
    if (act) {
      // reference gradients (difference form), then physical ones
      P gp[3], gs[3];
      for (int d = 0; d < 3; ++d) {
        gp[d] = vzero<T, BB>();
        gs[d] = vzero<T, BB>();
      }
      const P ui = u[i], wi = w[i];
      for (int m = 0; m < n; ++m) {
        const int k0 = ic * n * n + ib * n + m, k1 = ic * n * n + m * n + ia, k2 = m * n * n + ib * n + ia;
        const T d0 = D[ia * n + m], d1 = D[ib * n + m], d2 = D[ic * n + m];
        vfma(gp[0], d0, vsub(u[k0], ui));
        vfma(gp[1], d1, vsub(u[k1], ui));
        vfma(gp[2], d2, vsub(u[k2], ui));
        vfma(gs[0], d0, vsub(w[k0], wi));
        vfma(gs[1], d1, vsub(w[k1], wi));
        vfma(gs[2], d2, vsub(w[k2], wi));
      }
      P favg[3];
      for (int x = 0; x < 3; ++x) {
        // d/dx_x = sum_d (J^-1)_{d x} d/dxi_d
        P px = vmul(Ji[x], gp[0]), sx = vmul(Ji[x], gs[0]);
        vfma(px, Ji[3 + x], gp[1]);
        vfma(px, Ji[6 + x], gp[2]);
        vfma(sx, Ji[3 + x], gs[1]);
        vfma(sx, Ji[6 + x], gs[2]);
        const T zx = z[x], z3 = mul_(z[(x + 1) % 3], z[(x + 2) % 3]);
        const T a1 = sub_(T(1), mul_(h, zx)), den = add_(T(1), mul_(h, zx));
        const T ca = mul_(mul_(A.dt, A.c2), sub_(alpha, mul_(T(2), zx))), cz = mul_(mul_(A.dt, A.c2), z3);
        P* ph = reinterpret_cast<P*>(A.phi + (((long long)ep * 3 + x) * nl + i) * A.Bp) + ch;
        const P old = *ph;
        P nw = vmul(a1, old);
        vfma(nw, ca, px);
        vfma(nw, cz, sx);
#pragma unroll
        for (int b = 0; b < BB; ++b) nw.v[b] = div_(nw.v[b], den);
        *ph = nw;
        favg[x] = vmul(T(0.5), vadd(old, nw));
      }
      // F_d = w |J| sum_x (J^-1)_{d x} Phi_avg,x
      for (int d = 0; d < 3; ++d) {
        P f = vmul(Ji[3 * d], favg[0]);
        vfma(f, Ji[3 * d + 1], favg[1]);
        vfma(f, Ji[3 * d + 2], favg[2]);
        F[d * nl + i] = vmul(wJ, f);
      }
    }
    __syncthreads();
    if (act) {
      P r = vzero<T, BB>();
      for (int m = 0; m < n; ++m) {
        vfma(r, D[m * n + ia], F[ic * n * n + ib * n + m]);
        vfma(r, D[m * n + ib], F[nl + ic * n * n + m * n + ia]);
        vfma(r, D[m * n + ic], F[2 * nl + m * n * n + ib * n + ia]);
      }
      reinterpret_cast<P*>(A.S + (A.slot_base + (long long)ep * nl + i) * A.Bp)[ch] = r;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Power iteration helpers (FP64, one batch member): sum of squares, scaling
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) norm2_kernel(const double* x, long long n, double* out) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s = fma(x[i], x[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += w[k];
    atomicAdd(out, t);
  }
}

__global__ void __launch_bounds__(256) scale_kernel(double* dst, const double* src, const double* norm2, long long n) {
  const double s = 1.0 / sqrt(*norm2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] * s;
}

// e[b] += 1/2 sum_j M_j (v_jb^2 + p_jb w_jb) over a field [ndof][Bp] (energy diagnostic)
__global__ void __launch_bounds__(256) energy_kernel(const double* M, const double* v, const double* p, const double* w,
                                                   long long ndof, int B, int Bp, double* e) {
  const int b = blockIdx.y;
  double s = 0.0;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < ndof; j += (long long)gridDim.x * blockDim.x) {
    const long long o = j * Bp + b;
    s += M[j] * (v[o] * v[o] + p[o] * w[o]);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
    atomicAdd(e + b, 0.5 * t);
  }
}

cudaError_t launch_energy(const double* M, const double* v, const double* p, const double* w, long long ndof, int B,
                          int Bp, double* e, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(e, 0, sizeof(double) * B, s);
  if (err != cudaSuccess || B == 0) return err;
  energy_kernel<<<dim3(304, B), 256, 0, s>>>(M, v, p, w, ndof, B, Bp, e);
  return cudaGetLastError();
}

cudaError_t launch_norm2(const double* x, long long n, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  norm2_kernel<<<1216, 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* dst, const double* src, const double* norm2, long long n, cudaStream_t s) {
  scale_kernel<<<1216, 256, 0, s>>>(dst, src, norm2, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_geom(const GeomArgs& a, cudaStream_t s) {
  const long long n = (long long)a.ne * a.n * a.n * a.n;
  if (n == 0) return cudaSuccess;
  geom_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mass(const double* Mloc, const int* node_ptr, const int* node_slot, long long nvol, long long ndof,
                        double* Minv64, float* Minv32, double* M, cudaStream_t s) {
  if (ndof == 0) return cudaSuccess;
  mass_kernel<<<(unsigned)((ndof + 255) / 256), 256, 0, s>>>(Mloc, node_ptr, node_slot, nvol, ndof, Minv64, Minv32, M);
  return cudaGetLastError();
}

cudaError_t launch_faces(const FaceArgs& a, cudaStream_t s) {
  if (a.nf == 0) return cudaSuccess;
  face_kernel<<<(a.nf + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_match(const MatchArgs& a, cudaStream_t s) {
  const long long n = (long long)a.nff * a.q * a.q;
  if (n == 0) return cudaSuccess;
  match_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ipoints(const MatchArgs& a, cudaStream_t s) {
  const long long n = (long long)a.nff * a.q * a.q;
  if (n == 0) return cudaSuccess;
  ipoint_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int BB>
size_t iface_smem(const HexIfaceArgs<T>& a) {
  const long long Q = a.max_pts;
  const long long nlp = (long long)a.np * a.np * a.np, nlm = (long long)a.nm * a.nm * a.nm;
  return sizeof(T) * BB * (size_t)(nlp + nlm + 2 * Q) + sizeof(T) * (size_t)(Q * 6 * a.np + Q * 6 * a.nm + 8 * Q);
}

template <typename T, int BB>
size_t iface_face_smem(const HexIfaceArgs<T>& a) {
  const long long Q = a.max_pts;
  const long long nlp = (long long)a.np * a.np * a.np, nlm = (long long)a.nm * a.nm * a.nm;
  const long long nf = 2LL * (a.np * a.np + a.nm * a.nm);
  return sizeof(T) * BB * (size_t)(nlp + nlm + nf + 6 * Q) + sizeof(T) * (size_t)(Q * 8 * MAXN1 + 8 * Q);
}

template <typename T, int BB>
cudaError_t iface_face_bb(const HexIfaceArgs<T>& a, cudaStream_t s) {
  const size_t sm = iface_face_smem<T, BB>(a);
  if (sm > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(hex_iface_face_kernel<T, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  hex_iface_face_kernel<T, BB><<<a.ng, 128, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int BB>
cudaError_t iface_bb(const HexIfaceArgs<T>& a, cudaStream_t s) {
  if (a.onface) return iface_face_bb<T, BB>(a, s);
  const size_t sm = iface_smem<T, BB>(a);
  if (sm > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(hex_iface_kernel<T, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  hex_iface_kernel<T, BB><<<a.ng, 128, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_iface_table(const HexIfaceArgs<T>& a, T* tab, cudaStream_t s) {
  if (a.ng == 0) return cudaSuccess;
  iface_table_kernel<T><<<a.ng, 128, 0, s>>>(a, tab);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_iface_gtable(const HexIfaceArgs<T>& a, T* tab, cudaStream_t s) {
  if (a.ng == 0) return cudaSuccess;
  iface_gtable_kernel<T><<<a.ng, 128, 0, s>>>(a, tab);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_iface(const HexIfaceArgs<T>& a, cudaStream_t s) {
  if (a.ng == 0 || a.Bp == 0) return cudaSuccess;
  constexpr int V = vec_width<T>();
  return (a.Bp % V == 0) ? iface_bb<T, V>(a, s) : iface_bb<T, 1>(a, s);
}

template <typename T, int BB>
cudaError_t update_bb(const HexUpdateArgs<T>& a, cudaStream_t s) {
  const long long n = a.ndof * (a.Bp / BB);
  hex_update_kernel<T, BB><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_update(const HexUpdateArgs<T>& a, cudaStream_t s) {
  if (a.ndof == 0 || a.Bp == 0) return cudaSuccess;
  constexpr int V = vec_width<T>();
  return (a.Bp % V == 0) ? update_bb<T, V>(a, s) : update_bb<T, 1>(a, s);
}

template <typename T>
cudaError_t launch_hex_tail(const HexTailArgs<T>& a, cudaStream_t s) {
  const long long rth = (long long)a.B * a.R * 32;
  const long long blocks = a.fblocks + (rth + 255) / 256;
  hex_tail_kernel<T><<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int BB>
cudaError_t pml_bb(const HexPmlArgs<T>& a, int n, cudaStream_t s) {
  const int nl = n * n * n;
  const size_t sm = sizeof(Pack<T, BB>) * 5 * (size_t)nl + sizeof(T) * n * n;
  if (sm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(hex_pml_kernel<T, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  hex_pml_kernel<T, BB><<<a.npml, (nl + 31) / 32 * 32, sm, s>>>(a, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_pml(const HexPmlArgs<T>& a, int n, cudaStream_t s) {
  if (a.npml == 0 || a.Bp == 0) return cudaSuccess;
  constexpr int V = vec_width<T>();
  return (a.Bp % V == 0) ? pml_bb<T, V>(a, n, s) : pml_bb<T, 1>(a, n, s);
}

template cudaError_t launch_hex_pml<float>(const HexPmlArgs<float>&, int, cudaStream_t);
template cudaError_t launch_hex_pml<double>(const HexPmlArgs<double>&, int, cudaStream_t);
template cudaError_t launch_hex_iface<float>(const HexIfaceArgs<float>&, cudaStream_t);
template cudaError_t launch_hex_iface<double>(const HexIfaceArgs<double>&, cudaStream_t);
template cudaError_t launch_hex_iface_table<float>(const HexIfaceArgs<float>&, float*, cudaStream_t);
template cudaError_t launch_hex_iface_table<double>(const HexIfaceArgs<double>&, double*, cudaStream_t);
template cudaError_t launch_hex_iface_gtable<float>(const HexIfaceArgs<float>&, float*, cudaStream_t);
template cudaError_t launch_hex_iface_gtable<double>(const HexIfaceArgs<double>&, double*, cudaStream_t);
template cudaError_t launch_hex_update<float>(const HexUpdateArgs<float>&, cudaStream_t);
template cudaError_t launch_hex_update<double>(const HexUpdateArgs<double>&, cudaStream_t);
template cudaError_t launch_hex_tail<float>(const HexTailArgs<float>&, cudaStream_t);
template cudaError_t launch_hex_tail<double>(const HexTailArgs<double>&, cudaStream_t);

}  // namespace hex
