// Interface fluxes on Gamma_I (Sec. 5, eq. Wf_2 interface terms) and the
// PMUT modal step with receiver sampling (Algorithm 1 PMUT rows, eqs. g_m).
#include <type_traits>

#include "internal.h"

namespace {

constexpr int NP1 = DG_MAXN + 1;

// ---------------------------------------------------------------------------
// One CTA per listed coarse face F- (secondary bottom element) and chunk of
// batch members.  The fine faces F+ of F- (primary top elements, the finer
// side carrying the Gauss rule of Sec. 5) are processed in groups of up to
// FG at once, one thread per (fine face, Gauss node):
//   traces   p+, dp+/dn+ on F+ and p-, dp-/dn+ on F- at the Gauss nodes x_q
//            (x_q = X_{K+}(x^_q+), x^_q- = X_{K-}^-1(x_q): a fixed affine
//            sub-face map, folded into the interpolation table Ls),
//   jump  J = p+ - p-,  average  A = (c+^2 dp+/dn+ + c-^2 dp-/dn+) / 2,
//   weights  alpha = W (-A + gamma J),  beta+- = -W c+-^2 J / 2,
// then projects them back on the face GLL bases:
//   R_a = sum_q l_a(x_q) l_b(y_q) alpha_q,  R_b = sum_q l_a l_b beta_q.
// The residual of node (a,b,c) of K+ is R_a delta_{c,N} + d_c R_b with
// d_c = (2/h_z) l_c'(+1); of K- it is -R_a(alpha) delta_{c,0} + d_c R_b(beta-).
// Coarse sums run over the fine faces in list order (deterministic).
// ---------------------------------------------------------------------------
constexpr int FG = 4;          // fine faces per group
constexpr int IF_THREADS = 256;
constexpr int IF_BPC = 4;      // batch members per CTA
constexpr int NQ = DG_MAXQ, NP = NP1;

// Interpolation to the Gauss nodes and projection back are sum-factorised
// (one 1D contraction per direction), and every phase is spread over all
// threads of the CTA (items = face x field x line x node).
// CNP, CNS, CQ: compile-time (N+1) of both sides and Gauss points, or 0 for
// the runtime sizes of A (index arithmetic is the kernel's main cost).
template <typename T, int CNP, int CNS, int CQ>
__global__ void __launch_bounds__(IF_THREADS) iface_kernel(const __grid_constant__ IfaceArgs<T> A, int batch) {
  __shared__ T Lp[NQ * NP];
  __shared__ T Lsx[FG][NQ * NP], Lsy[FG][NQ * NP];
  __shared__ T Tp[FG][2][NP * NP];          // fine face: value / normal derivative at the face nodes
  __shared__ T Ts[2][NP * NP];              // coarse face
  __shared__ T W1[FG * 2 * NP * NQ * 2];    // x-interpolated (phase 2-3), then x-projected (phase 4-5)
  __shared__ T Q[FG][3][NQ * NQ];           // alpha, beta+, beta- at the Gauss nodes
  __shared__ T acc[2][NP * NP];             // coarse residual (alpha part, beta part)
  const int cf = blockIdx.x;
  const int tid = threadIdx.x;
  const int Np = CNP ? CNP - 1 : A.Np, Ns = CNS ? CNS - 1 : A.Ns, q = CQ ? CQ : A.q, qq = q * q;
  const int np1 = Np + 1, ns1 = Ns + 1, nf2 = np1 * np1, ns2 = ns1 * ns1;
  const int ccol = A.cf_col[cf];
  const int mx = ccol % A.nsx, my = ccol / A.nsx;
  const int f0 = A.cf_ptr[cf], f1 = A.cf_ptr[cf + 1];
  // W1 layout: fine part [f][w][line][node] (np1 lines x q nodes), coarse part after it
  T* U1p = W1;                                      // [FG][2][np1][q]
  T* U1s = W1 + FG * 2 * np1 * q;                   // [FG][2][ns1][q]
  for (int t = tid; t < q * np1; t += IF_THREADS) Lp[t] = A.Lp[t];
  const int b0 = blockIdx.y * IF_BPC, b1 = min(b0 + IF_BPC, batch);
  for (int b = b0; b < b1; ++b) {
    const T* pp = A.pp + (long long)b * A.bsp;
    const T* ps = A.ps + (long long)b * A.bss;
    __syncthreads();
    // coarse traces: value on the face (c = 0) and normal derivative
    for (int t = tid; t < ns2; t += IF_THREADS) {
      const int a = t % ns1, bb = t / ns1;
      const long long base = (long long)(my * Ns + bb) * A.pys + (mx * Ns + a);
      T g = T(0);
      for (int c = 0; c <= Ns; ++c) g += A.ds[c] * ps[base + (long long)c * A.pzs];
      Ts[0][t] = ps[base];
      Ts[1][t] = g;
      acc[0][t] = T(0);
      acc[1][t] = T(0);
    }
    for (int g0 = f0; g0 < f1; g0 += FG) {
      const int nfg = min(FG, f1 - g0);
      __syncthreads();
      // phase 1: tables of the group's sub-faces and the fine traces
      for (int t = tid; t < nfg * q * ns1; t += IF_THREADS) {
        const int f = t / (q * ns1), r = t - f * (q * ns1);
        Lsx[f][r] = A.Ls[(long long)A.ff_sx[g0 + f] * q * ns1 + r];
        Lsy[f][r] = A.Ls[(long long)A.ff_sy[g0 + f] * q * ns1 + r];
      }
      for (int t = tid; t < nfg * nf2; t += IF_THREADS) {
        const int f = t / nf2, r = t - f * nf2;
        const int fcol = A.ff_col[g0 + f];
        const int ex = fcol % A.npx, ey = fcol / A.npx;
        const int a = r % np1, bb = r / np1;
        const long long base = (long long)A.kp0 * A.pzp + (long long)(ey * Np + bb) * A.pyp + (ex * Np + a);
        T g = T(0);
        for (int c = 0; c <= Np; ++c) g += A.dp[c] * pp[base + (long long)c * A.pzp];
        Tp[f][0][r] = pp[base + (long long)Np * A.pzp];
        Tp[f][1][r] = g;
      }
      __syncthreads();
      // phase 2: interpolate along x to the Gauss abscissae (fine, and coarse per sub-face)
      {
        const int nfine = nfg * 2 * np1 * q, ncoarse = nfg * 2 * ns1 * q;
        for (int t = tid; t < nfine + ncoarse; t += IF_THREADS) {
          if (t < nfine) {
            const int qx = t % q, r = t / q;
            const int bb = r % np1, r2 = r / np1;
            const int w = r2 % 2, f = r2 / 2;
            const T* src = &Tp[f][w][bb * np1];
            T sum = T(0);
            for (int a = 0; a < np1; ++a) sum += Lp[qx * np1 + a] * src[a];
            U1p[((f * 2 + w) * np1 + bb) * q + qx] = sum;
          } else {
            const int u = t - nfine;
            const int qx = u % q, r = u / q;
            const int bb = r % ns1, r2 = r / ns1;
            const int w = r2 % 2, f = r2 / 2;
            const T* src = &Ts[w][bb * ns1];
            T sum = T(0);
            for (int a = 0; a < ns1; ++a) sum += Lsx[f][qx * ns1 + a] * src[a];
            U1s[((f * 2 + w) * ns1 + bb) * q + qx] = sum;
          }
        }
      }
      __syncthreads();
      // phase 3: along y, then jump / average / penalty weights at each Gauss node
      for (int t = tid; t < nfg * qq; t += IF_THREADS) {
        const int f = t / qq, r = t - f * qq;
        const int qx = r % q, qy = r / q;
        T up = T(0), dpv = T(0), um = T(0), dmv = T(0);
        for (int bb = 0; bb < np1; ++bb) {
          const T l = Lp[qy * np1 + bb];
          up += l * U1p[((f * 2 + 0) * np1 + bb) * q + qx];
          dpv += l * U1p[((f * 2 + 1) * np1 + bb) * q + qx];
        }
        for (int bb = 0; bb < ns1; ++bb) {
          const T l = Lsy[f][qy * ns1 + bb];
          um += l * U1s[((f * 2 + 0) * ns1 + bb) * q + qx];
          dmv += l * U1s[((f * 2 + 1) * ns1 + bb) * q + qx];
        }
        const T J = up - um;
        const T avg = T(0.5) * (A.cp2 * dpv + A.cm2 * dmv);
        const T W = A.Wq[r];
        Q[f][0][r] = W * (A.gamma * J - avg);
        Q[f][1][r] = -T(0.5) * W * A.cp2 * J;
        Q[f][2][r] = -T(0.5) * W * A.cm2 * J;
      }
      __syncthreads();
      // phase 4: project along x (fine: alpha, beta+; coarse: alpha, beta-)
      T* T2p = W1;                                  // [FG][2][q][np1]
      T* T2s = W1 + FG * 2 * q * np1;               // [FG][2][q][ns1]
      {
        const int nfine = nfg * 2 * q * np1, ncoarse = nfg * 2 * q * ns1;
        for (int t = tid; t < nfine + ncoarse; t += IF_THREADS) {
          if (t < nfine) {
            const int a = t % np1, r = t / np1;
            const int qy = r % q, r2 = r / q;
            const int w = r2 % 2, f = r2 / 2;
            const T* src = &Q[f][w][qy * q];
            T sum = T(0);
            for (int qx = 0; qx < q; ++qx) sum += Lp[qx * np1 + a] * src[qx];
            T2p[((f * 2 + w) * q + qy) * np1 + a] = sum;
          } else {
            const int u = t - nfine;
            const int a = u % ns1, r = u / ns1;
            const int qy = r % q, r2 = r / q;
            const int w = r2 % 2, f = r2 / 2;
            const T* src = &Q[f][w == 0 ? 0 : 2][qy * q];
            T sum = T(0);
            for (int qx = 0; qx < q; ++qx) sum += Lsx[f][qx * ns1 + a] * src[qx];
            T2s[((f * 2 + w) * q + qy) * ns1 + a] = sum;
          }
        }
      }
      __syncthreads();
      // phase 5: project along y; fine residuals out, coarse residual accumulated in face order
      {
        const int nfine = nfg * 2 * nf2;
        for (int t = tid; t < nfine + 2 * ns2; t += IF_THREADS) {
          if (t < nfine) {
            const int r = t % nf2, r2 = t / nf2;
            const int w = r2 % 2, f = r2 / 2;
            const int a = r % np1, bb = r / np1;
            T sum = T(0);
            for (int qy = 0; qy < q; ++qy) sum += Lp[qy * np1 + bb] * T2p[((f * 2 + w) * q + qy) * np1 + a];
            const long long o = (long long)b * A.rbp + (long long)A.ff_col[g0 + f] * nf2 + r;
            if (w == 0) A.Rap[o] = sum;
            else A.Rbp[o] = sum;
          } else {
            const int u = t - nfine;
            const int r = u % ns2, w = u / ns2;
            const int a = r % ns1, bb = r / ns1;
            T tot = acc[w][r];
            for (int f = 0; f < nfg; ++f) {
              T sum = T(0);
              for (int qy = 0; qy < q; ++qy) sum += Lsy[f][qy * ns1 + bb] * T2s[((f * 2 + w) * q + qy) * ns1 + a];
              tot += (w == 0) ? -sum : sum;
            }
            acc[w][r] = tot;
          }
        }
      }
    }
    __syncthreads();
    for (int t = tid; t < ns2; t += IF_THREADS) {
      const long long o = (long long)b * A.rbs + (long long)ccol * ns2 + t;
      A.Ras[o] = acc[0][t];
      A.Rbs[o] = acc[1][t];
    }
  }
}

// ---------------------------------------------------------------------------
// The same interface terms, organised for the production orders (compile-time
// NP1 = Np+1, NS1 = Ns+1, Q Gauss points, at most FS fine faces per coarse
// face).  One CTA takes one coarse face for BPC batch members at once.  A
// worker thread per (member, fine face, Gauss abscissa qx) contracts the
// face traces along x at its abscissa, then walks the Gauss rows qy: it
// interpolates along y, forms the jump / average / penalty weights at
// (qx, qy) and accumulates their projection along y onto the face GLL rows
// -- all in registers, with the 1D tables read from shared memory as
// broadcasts.  A last phase projects along x and writes the fine residuals
// and the coarse residual (summed over the fine faces in list order, so the
// result is deterministic).  Same arithmetic as iface_kernel, reordered.
// ---------------------------------------------------------------------------
constexpr int RB_THREADS = 256;

template <typename T, int NP1, int NS1, int Q, int FS, int BPC>
__global__ void __launch_bounds__(RB_THREADS, sizeof(T) == 4 ? 3 : 1) iface_rows_kernel(const __grid_constant__ IfaceArgs<T> A, int batch) {
  static_assert(BPC * FS * Q <= RB_THREADS, "one worker per (member, fine face, qx)");
  __shared__ T sLp[Q][NP1];
  __shared__ T sLsx[FS][Q][NS1], sLsy[FS][Q][NS1];
  __shared__ T sW[Q * Q];
  __shared__ T TF[BPC][FS][2][NP1 * NP1];      // fine traces: value, normal derivative
  __shared__ T TC[BPC][2][NS1 * NS1];          // coarse traces
  __shared__ T PF[BPC][FS][2][NP1][Q];         // y-projected fine weights (alpha, beta+) at (row, qx)
  __shared__ T PC[BPC][FS][2][NS1][Q];         // y-projected coarse weights (alpha, beta-)
  constexpr int NF2 = NP1 * NP1, NS2 = NS1 * NS1;
  const int cf = blockIdx.x;
  const int tid = threadIdx.x;
  const int b0 = blockIdx.y * BPC;
  const int nb = min(BPC, batch - b0);
  const int ccol = A.cf_col[cf];
  const int mx = ccol % A.nsx, my = ccol / A.nsx;
  const int f0 = A.cf_ptr[cf];
  const int nf = A.cf_ptr[cf + 1] - f0;
  const int Np = NP1 - 1, Ns = NS1 - 1;
  // tables
  for (int t = tid; t < Q * NP1; t += RB_THREADS) sLp[t / NP1][t % NP1] = A.Lp[t];
  for (int t = tid; t < nf * Q * NS1; t += RB_THREADS) {
    const int f = t / (Q * NS1), r = t - f * (Q * NS1);
    sLsx[f][r / NS1][r % NS1] = A.Ls[(long long)A.ff_sx[f0 + f] * Q * NS1 + r];
    sLsy[f][r / NS1][r % NS1] = A.Ls[(long long)A.ff_sy[f0 + f] * Q * NS1 + r];
  }
  for (int t = tid; t < Q * Q; t += RB_THREADS) sW[t] = A.Wq[t];
  // traces: coarse face (secondary bottom layer), then the fine faces (primary top layer)
  for (int t = tid; t < nb * NS2; t += RB_THREADS) {
    const int bl = t / NS2, r = t - bl * NS2;
    const int a = r % NS1, bb = r / NS1;
    const T* ps = A.ps + (long long)(b0 + bl) * A.bss;
    const long long base = (long long)(my * Ns + bb) * A.pys + (mx * Ns + a);
    T g = T(0);
#pragma unroll
    for (int c = 0; c < NS1; ++c) g += A.ds[c] * ps[base + (long long)c * A.pzs];
    TC[bl][0][r] = ps[base];
    TC[bl][1][r] = g;
  }
  for (int t = tid; t < nb * nf * NF2; t += RB_THREADS) {
    const int bl = t / (nf * NF2), r2 = t - bl * (nf * NF2);
    const int f = r2 / NF2, r = r2 - f * NF2;
    const int fcol = A.ff_col[f0 + f];
    const int ex = fcol % A.npx, ey = fcol / A.npx;
    const int a = r % NP1, bb = r / NP1;
    const T* pp = A.pp + (long long)(b0 + bl) * A.bsp;
    const long long base = (long long)A.kp0 * A.pzp + (long long)(ey * Np + bb) * A.pyp + (ex * Np + a);
    T g = T(0);
#pragma unroll
    for (int c = 0; c < NP1; ++c) g += A.dp[c] * pp[base + (long long)c * A.pzp];
    TF[bl][f][0][r] = pp[base + (long long)Np * A.pzp];
    TF[bl][f][1][r] = g;
  }
  __syncthreads();
  // workers: (member, fine face, qx)
  {
    const int bl = tid / (FS * Q);
    const int f = (tid / Q) % FS;
    const int qx = tid % Q;
    if (tid < BPC * FS * Q && bl < nb && f < nf) {
      T VF[2][NP1], VC[2][NS1];
      {
        T lx[NP1];
#pragma unroll
        for (int i = 0; i < NP1; ++i) lx[i] = sLp[qx][i];
#pragma unroll
        for (int w = 0; w < 2; ++w)
#pragma unroll
          for (int j = 0; j < NP1; ++j) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < NP1; ++i) s += lx[i] * TF[bl][f][w][j * NP1 + i];
            VF[w][j] = s;
          }
      }
      {
        T lx[NS1];
#pragma unroll
        for (int i = 0; i < NS1; ++i) lx[i] = sLsx[f][qx][i];
#pragma unroll
        for (int w = 0; w < 2; ++w)
#pragma unroll
          for (int j = 0; j < NS1; ++j) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < NS1; ++i) s += lx[i] * TC[bl][w][j * NS1 + i];
            VC[w][j] = s;
          }
      }
      T pa[NP1], pb[NP1], ca[NS1], cb[NS1];
#pragma unroll
      for (int j = 0; j < NP1; ++j) { pa[j] = T(0); pb[j] = T(0); }
#pragma unroll
      for (int j = 0; j < NS1; ++j) { ca[j] = T(0); cb[j] = T(0); }
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        T up = T(0), dup = T(0), um = T(0), dum = T(0);
#pragma unroll
        for (int j = 0; j < NP1; ++j) {
          const T l = sLp[qy][j];
          up += l * VF[0][j];
          dup += l * VF[1][j];
        }
#pragma unroll
        for (int j = 0; j < NS1; ++j) {
          const T l = sLsy[f][qy][j];
          um += l * VC[0][j];
          dum += l * VC[1][j];
        }
        const T J = up - um;
        const T avg = T(0.5) * (A.cp2 * dup + A.cm2 * dum);
        const T W = sW[qy * Q + qx];
        const T alpha = W * (A.gamma * J - avg);
        const T bp = -T(0.5) * W * A.cp2 * J;
        const T bm = -T(0.5) * W * A.cm2 * J;
#pragma unroll
        for (int j = 0; j < NP1; ++j) {
          const T l = sLp[qy][j];
          pa[j] += l * alpha;
          pb[j] += l * bp;
        }
#pragma unroll
        for (int j = 0; j < NS1; ++j) {
          const T l = sLsy[f][qy][j];
          ca[j] += l * alpha;
          cb[j] += l * bm;
        }
      }
#pragma unroll
      for (int j = 0; j < NP1; ++j) { PF[bl][f][0][j][qx] = pa[j]; PF[bl][f][1][j][qx] = pb[j]; }
#pragma unroll
      for (int j = 0; j < NS1; ++j) { PC[bl][f][0][j][qx] = ca[j]; PC[bl][f][1][j][qx] = cb[j]; }
    }
  }
  __syncthreads();
  // projection along x: fine residuals (alpha -> Rap, beta+ -> Rbp) ...
  for (int t = tid; t < nb * nf * 2 * NF2; t += RB_THREADS) {
    const int r = t % NF2, r2 = t / NF2;
    const int w = r2 % 2, r3 = r2 / 2;
    const int f = r3 % nf, bl = r3 / nf;
    const int i = r % NP1, j = r / NP1;
    T s = T(0);
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) s += sLp[qx][i] * PF[bl][f][w][j][qx];
    const long long o = (long long)(b0 + bl) * A.rbp + (long long)A.ff_col[f0 + f] * NF2 + r;
    if (w == 0) A.Rap[o] = s;
    else A.Rbp[o] = s;
  }
  // ... and the coarse residual (-alpha -> Ras, beta- -> Rbs), fine faces in list order
  for (int t = tid; t < nb * 2 * NS2; t += RB_THREADS) {
    const int r = t % NS2, r2 = t / NS2;
    const int w = r2 % 2, bl = r2 / 2;
    const int i = r % NS1, j = r / NS1;
    T tot = T(0);
    for (int f = 0; f < nf; ++f) {
      T s = T(0);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) s += sLsx[f][qx][i] * PC[bl][f][w][j][qx];
      tot += s;
    }
    const long long o = (long long)(b0 + bl) * A.rbs + (long long)ccol * NS2 + r;
    if (w == 0) A.Ras[o] = -tot;
    else A.Rbs[o] = tot;
  }
}

// ---------------------------------------------------------------------------
// Warps [0, B*K): PMUT (b, k).  g_{k,m} = sum_j B_{j,km} p^n_j (warp-shuffle
// reduction in FP64), then the Newmark predictor / solve / corrector of the
// modal ODE mu (q'' + 2 zeta w q' + w^2 q) = g + eta phi^n on lanes m < M.
// Warps [B*K, B*K + B*R): receiver (b, r): tensor Lagrange interpolation of
// p^{n+1} in its element, FP64 accumulation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) pmut_recv_kernel(const __grid_constant__ PmutArgs<T> A) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int npw = A.B * A.K;
  if (warp < npw) {
    const int b = warp / A.K, k = warp - b * A.K;
    const int M = A.M;
    // loads that do not depend on the projection go first, so their latency
    // overlaps the footprint gather below
    const int n = A.n + (A.step ? *A.step : 0);
    const long long kb = ((long long)b * A.K + k) * M;
    const bool rx = A.rx_gain && (A.step_base ? *A.step_base : 0) + n >= A.rx_switch;
    const double drv = (!rx && A.drive) ? A.drive[b * A.dbs + k * A.dks + n] : 0.0;
    double q = 0.0, qd = 0.0, qdd = 0.0;
    if (lane < M) {
      q = A.q[kb + lane];
      qd = A.qd[kb + lane];
      qdd = A.qdd[kb + lane];
    }
    const T* p = A.p_prev + (long long)b * A.bsp;
    const int e1 = A.fp_ptr[k + 1];
    double gm = 0.0;
    if (std::is_same<T, float>::value && A.Bm32) {
      // FP32 state: products and sums in FP32 (a footprint sums ~10^2 terms,
      // rounding ~1e-7 relative, the size of the FP32 field's own error);
      // GB300's FP64 pipe made the FP64 sums most of this kernel's time.  The
      // modal state below stays FP64.
      float g[DG_MAXM];
#pragma unroll
      for (int m = 0; m < DG_MAXM; ++m) g[m] = 0.f;
      for (int e = A.fp_ptr[k] + lane; e < e1; e += 32) {
        const float pv = (float)p[A.fp_off[e]];
        const float* Bv = A.Bm32 + (long long)e * M;
#pragma unroll
        for (int m = 0; m < DG_MAXM; ++m)
          if (m < M) g[m] = fmaf(Bv[m], pv, g[m]);
      }
#pragma unroll
      for (int m = 0; m < DG_MAXM; ++m) {
        if (m < M) {
          const float s = warp_sum(g[m]);
          if (lane == m) gm = (double)s;
        }
      }
    } else {
      double g[DG_MAXM];
#pragma unroll
      for (int m = 0; m < DG_MAXM; ++m) g[m] = 0.0;
      for (int e = A.fp_ptr[k] + lane; e < e1; e += 32) {
        const double pv = (double)p[A.fp_off[e]];
        const double* Bv = A.Bm + (long long)e * M;
#pragma unroll
        for (int m = 0; m < DG_MAXM; ++m)
          if (m < M) g[m] += Bv[m] * pv;
      }
#pragma unroll
      for (int m = 0; m < DG_MAXM; ++m) {
        if (m < M) {
          const double s = warp_sum(g[m]);
          if (lane == m) gm = s;
        }
      }
    }
    // voltage of membrane k at t^n: the drive (TX) or, from step rx_switch on,
    // the open-circuit value s / C_k sum_m eta_km q_km^n (RX, eq. ode row 2)
    double phi = drv;
    if (rx) phi = warp_sum((lane < M) ? A.eta[k * M + lane] * q : 0.0) * A.rx_gain[k];
    if (lane < M) {
      const int km = k * M + lane;
      const long long idx = kb + lane;
      const double dt = A.dt;
      const double qn = q + dt * qd + 0.5 * dt * dt * qdd;          // predictor
      const double qdp = qd + 0.5 * dt * qdd;
      const double qddn = -A.omega2[km] * qn - A.twozw[km] * qdp + (gm + A.eta[km] * phi) * A.inv_mu[km];
      A.q[idx] = qn;
      A.qd[idx] = qdp + 0.5 * dt * qddn;                                // corrector
      A.qdd[idx] = qddn;
      if (A.qdd32) A.qdd32[idx] = (float)qddn;
    }
    if (A.volt && lane == 0) A.volt[b * A.vbs + k * A.vks + n] = phi;
    return;
  }
  const int rw = warp - npw;
  if (rw >= A.B * A.R) return;
  const int b = rw / A.R, r = rw - b * A.R;
  const T* p = (A.rdom[r] == 0) ? A.pc0 + (long long)b * A.bs0 : A.pc1 + (long long)b * A.bs1;
  double s = 0.0;
  const int nn = A.rnn[r];
  const double* w = A.rw + (long long)r * A.rstride;
  const long long* off = A.roff + (long long)r * A.rstride;
  for (int t = lane; t < nn; t += 32) s += w[t] * (double)p[off[t]];
  s = warp_sum(s);
  if (lane == 0) A.traces[b * A.tbs + r * A.trs + A.n + (A.step ? *A.step : 0)] = s;
}

// ---------------------------------------------------------------------------
// Face assembly (once per step): the interface residual of every face node,
// summed over the faces that touch it in a fixed order, and the PMUT forcing
// f_j = -kappa sum_{entries of j} sum_m q''_m B_{j,m} (eq. f_i) of every node
// of the primary's z-min face, accumulated in FP64.  The volume kernels read
// both as contiguous rows.
// ---------------------------------------------------------------------------
// A thread takes one face node for AB batch members, so the index work and
// the CSR walk are shared by them.
constexpr int AB = 8;

template <typename T, int N>
__global__ void __launch_bounds__(256) face_asm_kernel(const __grid_constant__ FaceAsmArgs<T> A, int batch) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)A.L0 * A.L1) return;
  const int i = (int)(t % A.L0), j = (int)(t / A.L0);
  const int b0 = blockIdx.y * AB, b1 = min(batch, b0 + AB);
  // face entries touching node (i, j), in the order of face_gather
  int fx = i / N, ax = i - fx * N, fy = j / N, ay = j - fy * N;
  if (fx == A.ne0) { fx = A.ne0 - 1; ax = N; }
  if (fy == A.ne1) { fy = A.ne1 - 1; ay = N; }
  constexpr int F = (N + 1) * (N + 1);
  long long off[4];
  int n = 0;
  off[n++] = (long long)(fy * A.ne0 + fx) * F + ay * (N + 1) + ax;
  if (ax == 0 && fx > 0) off[n++] = (long long)(fy * A.ne0 + fx - 1) * F + ay * (N + 1) + N;
  if (ay == 0 && fy > 0) off[n++] = (long long)((fy - 1) * A.ne0 + fx) * F + N * (N + 1) + ax;
  if (ax == 0 && fx > 0 && ay == 0 && fy > 0) off[n++] = (long long)((fy - 1) * A.ne0 + fx - 1) * F + N * (N + 1) + N;
  for (int b = b0; b < b1; ++b) {
    const T* Ra = A.Ra + (long long)b * A.rbs;
    const T* Rb = A.Rb + (long long)b * A.rbs;
    T sa = Ra[off[0]], sb = Rb[off[0]];
    for (int q = 1; q < n; ++q) {
      sa += Ra[off[q]];
      sb += Rb[off[q]];
    }
    const long long o = (long long)b * A.gbs + (long long)j * A.py + i;
    A.ga[o] = sa;
    A.gb[o] = sb;
  }
}

// FP64 state: q'' and B in FP64.  FP32 state: their FP32 copies, summed in
// FP32 (a node sums one or two footprint entries of a few modes; the result
// joins an FP32 state update, and GB300's FP64 pipe is narrow).
template <typename T>
__global__ void __launch_bounds__(256) pmut_force_kernel(const __grid_constant__ PmutForceArgs A, int batch) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)A.L0 * A.L1) return;
  const int i = (int)(t % A.L0), j = (int)(t / A.L0);
  const int b0 = blockIdx.y * AB, nb = min(batch - b0, AB);
  const T* qdd;
  const T* Bm;
  if constexpr (sizeof(T) == 4) { qdd = reinterpret_cast<const T*>(A.qdd32); Bm = reinterpret_cast<const T*>(A.Bm32); }
  else { qdd = reinterpret_cast<const T*>(A.qdd); Bm = reinterpret_cast<const T*>(A.Bm); }
  T f[AB];
#pragma unroll
  for (int q = 0; q < AB; ++q) f[q] = T(0);
  const int e1 = A.node_ptr[t + 1];
  for (int e = A.node_ptr[t]; e < e1; ++e) {
    const int ent = A.node_ent[e];
    const int k = A.ent_pmut[ent];
    const T* Bv = Bm + (long long)ent * A.M;
    for (int m = 0; m < A.M; ++m) {
      const T bm = Bv[m];
#pragma unroll
      for (int q = 0; q < AB; ++q)
        if (q < nb) f[q] += qdd[((long long)(b0 + q) * A.K + k) * A.M + m] * bm;
    }
  }
  const T kap = T(-A.kappa);
#pragma unroll
  for (int q = 0; q < AB; ++q)
    if (q < nb) static_cast<T*>(A.f)[(long long)(b0 + q) * A.fbs + (long long)j * A.py + i] = kap * f[q];
}

// ---------------------------------------------------------------------------
// Power-iteration helpers (setup only): M-weighted dot product over a box
// lattice with the lumped mass M = scale * w_x(i) w_y(j) w_z(k), and scaling.
// ---------------------------------------------------------------------------
template <typename TX>
__global__ void __launch_bounds__(256) mdot_kernel(const TX* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ wx, const double* __restrict__ wy,
                                                   const double* __restrict__ wz, int L0, int L1, int L2, int py,
                                                   long long pz, double scale, double* out) {
  __shared__ double red[8];
  const long long n = (long long)L0 * L1 * L2;
  double s = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % L0);
    const long long r = t / L0;
    const int j = (int)(r % L1), k = (int)(r / L1);
    const long long g = (long long)k * pz + (long long)j * py + i;
    s += wx[i] * wy[j] * wz[k] * (double)x[g] * y[g];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) atomicAdd(out, v * scale);
  }
}

// y = x, FP32 -> FP64 (exact)
__global__ void widen_kernel(const float* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    y[t] = (double)x[t];
}

__global__ void scale_kernel(double* __restrict__ x, const double* __restrict__ y, double a, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    x[t] = a * y[t];
}

}  // namespace

cudaError_t launch_mdot(const double* x, const double* y, const double* wx, const double* wy, const double* wz, int L0,
                        int L1, int L2, int py, long long pz, double scale, double* out, cudaStream_t s) {
  mdot_kernel<double><<<4 * 152, 256, 0, s>>>(x, y, wx, wy, wz, L0, L1, L2, py, pz, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_mdot(const float* x, const double* y, const double* wx, const double* wy, const double* wz, int L0,
                        int L1, int L2, int py, long long pz, double scale, double* out, cudaStream_t s) {
  mdot_kernel<float><<<4 * 152, 256, 0, s>>>(x, y, wx, wy, wz, L0, L1, L2, py, pz, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* x, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  widen_kernel<<<4 * 152, 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* x, const double* y, double a, long long n, cudaStream_t s) {
  scale_kernel<<<4 * 152, 256, 0, s>>>(x, y, a, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_iface(const IfaceArgs<T>& a, int batch, cudaStream_t s) {
  if (a.ncf <= 0) return cudaSuccess;
  constexpr int BPC = sizeof(T) == 4 ? 8 : 4;   // static shared memory stays under 48 KB
  if (a.max_ff <= 4 && a.Np == 4 && a.Ns == 6 && a.q == 7) {
    iface_rows_kernel<T, 5, 7, 7, 4, BPC><<<dim3(a.ncf, (batch + BPC - 1) / BPC), RB_THREADS, 0, s>>>(a, batch);
  } else if (a.max_ff <= 4 && a.Np == 4 && a.Ns == 4 && a.q == 5) {
    iface_rows_kernel<T, 5, 5, 5, 4, BPC><<<dim3(a.ncf, (batch + BPC - 1) / BPC), RB_THREADS, 0, s>>>(a, batch);
  } else {
    dim3 grid(a.ncf, (batch + IF_BPC - 1) / IF_BPC);
    iface_kernel<T, 0, 0, 0><<<grid, IF_THREADS, 0, s>>>(a, batch);
  }
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) nonfinite_kernel(const double* x, size_t n, int* flag) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad = bad || !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

cudaError_t launch_nonfinite(const double* x, size_t n, int* flag, cudaStream_t s) {
  if (n == 0 || !x) return cudaSuccess;
  const size_t blocks = std::min<size_t>((n + 255) / 256, 1216);
  nonfinite_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, flag);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pmut_recv(const PmutArgs<T>& a, cudaStream_t s) {
  const long long warps = (long long)a.B * a.K + (long long)a.B * a.R;
  if (warps <= 0) return cudaSuccess;
  const long long blocks = (warps * 32 + 255) / 256;
  pmut_recv_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_face_asm(const FaceAsmArgs<T>& a, int batch, cudaStream_t s) {
  const long long n = (long long)a.L0 * a.L1;
  if (n == 0 || batch <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((n + 255) / 256), (batch + AB - 1) / AB);
  switch (a.N) {
    case 1: face_asm_kernel<T, 1><<<grid, 256, 0, s>>>(a, batch); break;
    case 2: face_asm_kernel<T, 2><<<grid, 256, 0, s>>>(a, batch); break;
    case 3: face_asm_kernel<T, 3><<<grid, 256, 0, s>>>(a, batch); break;
    case 4: face_asm_kernel<T, 4><<<grid, 256, 0, s>>>(a, batch); break;
    case 5: face_asm_kernel<T, 5><<<grid, 256, 0, s>>>(a, batch); break;
    case 6: face_asm_kernel<T, 6><<<grid, 256, 0, s>>>(a, batch); break;
    case 7: face_asm_kernel<T, 7><<<grid, 256, 0, s>>>(a, batch); break;
    case 8: face_asm_kernel<T, 8><<<grid, 256, 0, s>>>(a, batch); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pmut_force(const PmutForceArgs& a, int batch, cudaStream_t s) {
  const long long n = (long long)a.L0 * a.L1;
  if (n == 0 || batch <= 0) return cudaSuccess;
  pmut_force_kernel<T><<<dim3((unsigned)((n + 255) / 256), (batch + AB - 1) / AB), 256, 0, s>>>(a, batch);
  return cudaGetLastError();
}

template cudaError_t launch_face_asm<float>(const FaceAsmArgs<float>&, int, cudaStream_t);
template cudaError_t launch_face_asm<double>(const FaceAsmArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pmut_force<float>(const PmutForceArgs&, int, cudaStream_t);
template cudaError_t launch_pmut_force<double>(const PmutForceArgs&, int, cudaStream_t);
template cudaError_t launch_iface<float>(const IfaceArgs<float>&, int, cudaStream_t);
template cudaError_t launch_iface<double>(const IfaceArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pmut_recv<float>(const PmutArgs<float>&, cudaStream_t);
template cudaError_t launch_pmut_recv<double>(const PmutArgs<double>&, cudaStream_t);
