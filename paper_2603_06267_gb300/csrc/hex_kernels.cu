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

#include "hex_geom.h"

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
    const long long o = (6LL * e + k) * nl + i;
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
// Element stiffness of eq. (Wf_2) on one element per CTA, for every batch
// member: grad^ u by the GLL derivative matrix (difference form
// sum_m D_am (u_m - u_a), exact for constants in any precision), the
// geometric factors, then the transposed derivative; the element-local
// residual goes to the element's slots.
template <typename T, int N>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    hex_vol_kernel(const __grid_constant__ HexVolArgs<T> A) {
  constexpr int n = N + 1, nl = n * n * n;
  __shared__ T u[nl];
  __shared__ T F[3][nl];
  __shared__ T D[n][n];
  const int e = blockIdx.x;
  const int i = threadIdx.x;
  if (i < n * n) D[i / n][i % n] = A.D[i / n][i % n];
  const bool act = i < nl;
  const int ia = i % n, ib = (i / n) % n, ic = i / (n * n);
  int node = 0;
  T g[6];
  if (act) {
    node = A.conn[(long long)e * nl + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) g[k] = A.G[(6LL * e + k) * nl + i];
  }
  const long long slot = A.slot_base + (long long)e * nl + i;
  for (int b = 0; b < A.batch; ++b) {
    if (act) u[i] = A.p[b * A.p_bs + node];
    __syncthreads();
    if (act) {
      const T ui = u[i];
      T g0 = T(0), g1 = T(0), g2 = T(0);
#pragma unroll
      for (int m = 0; m < n; ++m) {
        g0 += D[ia][m] * (u[ic * n * n + ib * n + m] - ui);
        g1 += D[ib][m] * (u[ic * n * n + m * n + ia] - ui);
        g2 += D[ic][m] * (u[m * n * n + ib * n + ia] - ui);
      }
      F[0][i] = g[0] * g0 + g[3] * g1 + g[4] * g2;
      F[1][i] = g[3] * g0 + g[1] * g1 + g[5] * g2;
      F[2][i] = g[4] * g0 + g[5] * g1 + g[2] * g2;
    }
    __syncthreads();
    if (act) {
      T r = T(0);
#pragma unroll
      for (int m = 0; m < n; ++m) {
        r += D[m][ia] * F[0][ic * n * n + ib * n + m];
        r += D[m][ib] * F[1][ic * n * n + m * n + ia];
        r += D[m][ic] * F[2][m * n * n + ib * n + ia];
      }
      A.S[b * A.s_bs + slot] = r;
    }
    __syncthreads();
  }
}

// SIPG interface terms of eq. (Wf_2) for one group of fine Gauss nodes that
// share a fine element K+ and a coarse element K-.  With jump J = p+ - p-
// and A = 1/2 (c+^2 dp+/dn+ + c-^2 dp-/dn+):
//   r_i(K+) += W (gamma J - A) psi_i - 1/2 W J c+^2 d psi_i / d n+
//   r_i(K-) -= W (gamma J - A) psi_i + 1/2 W J c-^2 d psi_i / d n+
template <typename T>
__global__ void __launch_bounds__(128) hex_iface_kernel(const __grid_constant__ HexIfaceArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = blockIdx.x;
  const int np = A.np, nm = A.nm;
  const int nlp = np * np * np, nlm = nm * nm * nm;
  const int p0 = A.g_pt[g], npts = A.g_pt[g + 1] - p0;
  const int P = A.max_pts;
  T* up = reinterpret_cast<T*>(smem_raw);
  T* um = up + nlp;
  T* tp = um + nlm;                 // [P][3][2][np]: l, l' per axis, fine side
  T* tm = tp + (long long)P * 6 * np;   // [P][3][2][nm]
  T* av = tm + (long long)P * 6 * nm;   // [P][8]: a+(3) a-(3) W gamma
  T* sv = av + 8 * P;               // [P]
  T* sd = sv + P;                   // [P]
  const int tid = threadIdx.x;
  for (int j = tid; j < npts; j += blockDim.x) {
    const double* d = A.pdat + (long long)PDAT * A.pt_idx[p0 + j];
    double l[MAXN1], dl[MAXN1];
    for (int ax = 0; ax < 3; ++ax) {
      lagrange(np, A.xip, d[ax], l, dl);
      for (int k = 0; k < np; ++k) {
        tp[((j * 3 + ax) * 2) * np + k] = T(l[k]);
        tp[((j * 3 + ax) * 2 + 1) * np + k] = T(dl[k]);
      }
      lagrange(nm, A.xim, d[3 + ax], l, dl);
      for (int k = 0; k < nm; ++k) {
        tm[((j * 3 + ax) * 2) * nm + k] = T(l[k]);
        tm[((j * 3 + ax) * 2 + 1) * nm + k] = T(dl[k]);
      }
    }
    for (int k = 0; k < 8; ++k) av[8 * j + k] = T(d[6 + k]);
  }
  const int fe = A.g_fe[g], ce = A.g_ce[g];
  const long long slot = A.g_slot[g];
  const T c2p = T(A.c2p), c2m = T(A.c2m);
  for (int b = 0; b < A.batch; ++b) {
    for (int i = tid; i < nlp; i += blockDim.x) up[i] = A.p[b * A.p_bs + A.conn_p[(long long)fe * nlp + i]];
    for (int i = tid; i < nlm; i += blockDim.x) um[i] = A.p[b * A.p_bs + A.conn_m[(long long)ce * nlm + i]];
    __syncthreads();
    for (int j = tid; j < npts; j += blockDim.x) {
      T vp = 0, dp0 = 0, dp1 = 0, dp2 = 0;
      {
        const T* lx = tp + (j * 3 + 0) * 2 * np;
        const T* ly = tp + (j * 3 + 1) * 2 * np;
        const T* lz = tp + (j * 3 + 2) * 2 * np;
        for (int c = 0; c < np; ++c)
          for (int bb = 0; bb < np; ++bb) {
            T s0 = 0, s1 = 0;
            for (int a = 0; a < np; ++a) {
              const T uv = up[(c * np + bb) * np + a];
              s0 += lx[a] * uv;
              s1 += lx[np + a] * uv;
            }
            const T yz = ly[bb] * lz[c];
            vp += yz * s0;
            dp0 += yz * s1;
            dp1 += ly[np + bb] * lz[c] * s0;
            dp2 += ly[bb] * lz[np + c] * s0;
          }
      }
      T vm = 0, dm0 = 0, dm1 = 0, dm2 = 0;
      {
        const T* lx = tm + (j * 3 + 0) * 2 * nm;
        const T* ly = tm + (j * 3 + 1) * 2 * nm;
        const T* lz = tm + (j * 3 + 2) * 2 * nm;
        for (int c = 0; c < nm; ++c)
          for (int bb = 0; bb < nm; ++bb) {
            T s0 = 0, s1 = 0;
            for (int a = 0; a < nm; ++a) {
              const T uv = um[(c * nm + bb) * nm + a];
              s0 += lx[a] * uv;
              s1 += lx[nm + a] * uv;
            }
            const T yz = ly[bb] * lz[c];
            vm += yz * s0;
            dm0 += yz * s1;
            dm1 += ly[nm + bb] * lz[c] * s0;
            dm2 += ly[bb] * lz[nm + c] * s0;
          }
      }
      const T* a8 = av + 8 * j;
      const T jump = vp - vm;
      const T avg = T(0.5) * (c2p * (dp0 * a8[0] + dp1 * a8[1] + dp2 * a8[2]) +
                              c2m * (dm0 * a8[3] + dm1 * a8[4] + dm2 * a8[5]));
      sv[j] = a8[6] * (a8[7] * jump - avg);
      sd[j] = T(-0.5) * a8[6] * jump;
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
      T r = 0;
      for (int j = 0; j < npts; ++j) {
        const T* lx = tb + (j * 3 + 0) * 2 * n;
        const T* ly = tb + (j * 3 + 1) * 2 * n;
        const T* lz = tb + (j * 3 + 2) * 2 * n;
        const T* a8 = av + 8 * j + (plus ? 0 : 3);
        const T psi = lx[ia] * ly[ib] * lz[ic];
        const T dn = a8[0] * lx[n + ia] * ly[ib] * lz[ic] + a8[1] * lx[ia] * ly[n + ib] * lz[ic] +
                     a8[2] * lx[ia] * ly[ib] * lz[n + ic];
        r += sgn * sv[j] * psi + sd[j] * c2 * dn;
      }
      A.S[b * A.s_bs + slot + i] = r;
    }
    __syncthreads();
  }
}

// Residual assembly and leapfrog update, one thread per node and up to
// UB batch members: r = sum of the node's slots (ascending slot order, so
// the sum is the same in every run), v += cv M^-1 r, p += cp v.
constexpr int UB = 8;

template <typename T>
__global__ void __launch_bounds__(256) hex_update_kernel(const __grid_constant__ HexUpdateArgs<T> A) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= A.ndof) return;
  const int k0 = A.node_ptr[j], k1 = A.node_ptr[j + 1];
  const T mi = A.Minv[j];
  const int b0 = blockIdx.y * UB, b1 = min(A.batch, b0 + UB);
  for (int b = b0; b < b1; ++b) {
    const T* S = A.S + b * A.s_bs;
    T r = 0;
    for (int k = k0; k < k1; ++k) r += S[A.node_slot[k]];
    const long long o = b * A.p_bs + j;
    const T v = A.v[o] + A.cv * mi * r;
    A.v[o] = v;
    A.p[o] = A.p[o] + A.cp * v;
  }
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
    if (t < (long long)A.nnz * A.batch) {
      const int b = (int)(t / A.nnz), e = (int)(t - (long long)b * A.nnz);
      const int k = A.ent_k[e];
      const double* q = A.qdd + ((long long)b * A.K + k) * A.M;
      const double* Bv = A.Bm + (long long)e * A.M;
      double s = 0.0;
      for (int m = 0; m < A.M; ++m) s += q[m] * Bv[m];
      A.S[b * A.s_bs + A.fslot + e] = T(A.kappa * s);
    }
  } else {
    const int warp = (int)(((blockIdx.x - A.fblocks) * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp < A.batch * A.R) {
      const int b = warp / A.R, r = warp - b * A.R;
      const T* p = A.p + b * A.p_bs;
      const double* w = A.rw + (long long)r * A.rstride;
      const long long* off = A.roff + (long long)r * A.rstride;
      double s = 0.0;
      for (int t = lane; t < A.rnn[r]; t += 32) s += w[t] * (double)p[off[t]];
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

template <typename T, int N>
cudaError_t vol_n(const HexVolArgs<T>& a, cudaStream_t s) {
  constexpr int threads = ((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32;
  hex_vol_kernel<T, N><<<a.ne, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_vol(const HexVolArgs<T>& a, int n, cudaStream_t s) {
  if (a.ne == 0 || a.batch == 0) return cudaSuccess;
  switch (n - 1) {
    case 1: return vol_n<T, 1>(a, s);
    case 2: return vol_n<T, 2>(a, s);
    case 3: return vol_n<T, 3>(a, s);
    case 4: return vol_n<T, 4>(a, s);
    case 5: return vol_n<T, 5>(a, s);
    case 6: return vol_n<T, 6>(a, s);
    case 7: return vol_n<T, 7>(a, s);
    case 8: return vol_n<T, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
size_t iface_smem(const HexIfaceArgs<T>& a) {
  const long long P = a.max_pts;
  const long long nlp = (long long)a.np * a.np * a.np, nlm = (long long)a.nm * a.nm * a.nm;
  return sizeof(T) * (size_t)(nlp + nlm + P * 6 * a.np + P * 6 * a.nm + 8 * P + 2 * P);
}

template <typename T>
cudaError_t launch_hex_iface(const HexIfaceArgs<T>& a, cudaStream_t s) {
  if (a.ng == 0 || a.batch == 0) return cudaSuccess;
  const size_t sm = iface_smem(a);
  if (sm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(hex_iface_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  hex_iface_kernel<T><<<a.ng, 128, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_update(const HexUpdateArgs<T>& a, cudaStream_t s) {
  if (a.ndof == 0 || a.batch == 0) return cudaSuccess;
  const dim3 grid((unsigned)((a.ndof + 255) / 256), (a.batch + UB - 1) / UB);
  hex_update_kernel<T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_hex_tail(const HexTailArgs<T>& a, cudaStream_t s) {
  const long long rth = (long long)a.batch * a.R * 32;
  const long long blocks = a.fblocks + (rth + 255) / 256;
  hex_tail_kernel<T><<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_hex_vol<float>(const HexVolArgs<float>&, int, cudaStream_t);
template cudaError_t launch_hex_vol<double>(const HexVolArgs<double>&, int, cudaStream_t);
template cudaError_t launch_hex_iface<float>(const HexIfaceArgs<float>&, cudaStream_t);
template cudaError_t launch_hex_iface<double>(const HexIfaceArgs<double>&, cudaStream_t);
template cudaError_t launch_hex_update<float>(const HexUpdateArgs<float>&, cudaStream_t);
template cudaError_t launch_hex_update<double>(const HexUpdateArgs<double>&, cudaStream_t);
template cudaError_t launch_hex_tail<float>(const HexTailArgs<float>&, cudaStream_t);
template cudaError_t launch_hex_tail<double>(const HexTailArgs<double>&, cudaStream_t);

}  // namespace hex
