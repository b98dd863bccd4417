// Interface fluxes on Gamma_I (Sec. 5, eq. Wf_2 interface terms) and the
// PMUT modal step with receiver sampling (Algorithm 1 PMUT rows, eqs. g_m).
#include "internal.h"

namespace {

constexpr int NP1 = DG_MAXN + 1;

// ---------------------------------------------------------------------------
// One CTA per listed coarse face F- (secondary bottom element).  For each of
// its fine faces F+ (primary top elements, the finer side carrying the Gauss
// rule of Sec. 5):
//   traces   p+, dp+/dn+ on F+ and p-, dp-/dn+ on F- at the Gauss nodes x_q
//            (x_q = X_{K+}(x^_q+), x^_q- = X_{K-}^-1(x_q): a fixed affine
//            sub-face map, folded into the interpolation table Ls),
//   jump  J = p+ - p-,  average  A = (c+^2 dp+/dn+ + c-^2 dp-/dn+) / 2,
//   weights  alpha = W (-A + gamma J),  beta+- = -W c+-^2 J / 2,
// and projects them back on the face GLL basis:
//   R_a = sum_q l_a(x_q) l_b(y_q) alpha_q,  R_b = sum_q l_a l_b beta_q.
// The residual of a node (a,b,c) of K+ is R_a delta_{c,N} + d_c R_b with
// d_c = (2/h_z) l_c'(+1); of K- it is -R_a(alpha) delta_{c,0} + d_c R_b(beta-).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) iface_kernel(const __grid_constant__ IfaceArgs<T> A) {
  __shared__ T Ts[NP1 * NP1], Gs[NP1 * NP1];
  __shared__ T Tp[NP1 * NP1], Gp[NP1 * NP1];
  __shared__ T al[DG_MAXQ * DG_MAXQ], bp[DG_MAXQ * DG_MAXQ], bm[DG_MAXQ * DG_MAXQ];
  __shared__ T Lp[DG_MAXQ * NP1], Lsx[DG_MAXQ * NP1], Lsy[DG_MAXQ * NP1];
  const int cf = blockIdx.x;
  const int b = blockIdx.y;
  const int tid = threadIdx.x;
  const int Np = A.Np, Ns = A.Ns, q = A.q;
  const int np1 = Np + 1, ns1 = Ns + 1;
  const T* pp = A.pp + (long long)b * A.bsp;
  const T* ps = A.ps + (long long)b * A.bss;
  const int ccol = A.cf_col[cf];
  const int mx = ccol % A.nsx, my = ccol / A.nsx;

  for (int t = tid; t < q * np1; t += blockDim.x) Lp[t] = A.Lp[t];
  // coarse traces: value on the face (c = 0) and normal derivative
  for (int t = tid; t < ns1 * ns1; t += blockDim.x) {
    const int a = t % ns1, bb = t / ns1;
    const long long base = (long long)(my * Ns + bb) * A.pys + (mx * Ns + a);
    T g = T(0);
    for (int c = 0; c <= Ns; ++c) g += A.ds[c] * ps[base + (long long)c * A.pzs];
    Ts[t] = ps[base];
    Gs[t] = g;
  }
  // per-thread accumulators of the coarse residual (t = a + ns1*b)
  T accA[2] = {T(0), T(0)}, accB[2] = {T(0), T(0)};
  for (int f = A.cf_ptr[cf]; f < A.cf_ptr[cf + 1]; ++f) {
    const int fcol = A.ff_col[f];
    const int ex = fcol % A.npx, ey = fcol / A.npx;
    __syncthreads();
    for (int t = tid; t < q * ns1; t += blockDim.x) {
      Lsx[t] = A.Ls[(long long)A.ff_sx[f] * q * ns1 + t];
      Lsy[t] = A.Ls[(long long)A.ff_sy[f] * q * ns1 + t];
    }
    for (int t = tid; t < np1 * np1; t += blockDim.x) {
      const int a = t % np1, bb = t / np1;
      const long long base = (long long)A.kp0 * A.pzp + (long long)(ey * Np + bb) * A.pyp + (ex * Np + a);
      T g = T(0);
      for (int c = 0; c <= Np; ++c) g += A.dp[c] * pp[base + (long long)c * A.pzp];
      Tp[t] = pp[base + (long long)Np * A.pzp];
      Gp[t] = g;
    }
    __syncthreads();
    for (int t = tid; t < q * q; t += blockDim.x) {
      const int qx = t % q, qy = t / q;
      T up = T(0), dpv = T(0);
      for (int bb = 0; bb < np1; ++bb) {
        T su = T(0), sd = T(0);
        for (int a = 0; a < np1; ++a) {
          su += Lp[qx * np1 + a] * Tp[bb * np1 + a];
          sd += Lp[qx * np1 + a] * Gp[bb * np1 + a];
        }
        up += Lp[qy * np1 + bb] * su;
        dpv += Lp[qy * np1 + bb] * sd;
      }
      T um = T(0), dmv = T(0);
      for (int bb = 0; bb < ns1; ++bb) {
        T su = T(0), sd = T(0);
        for (int a = 0; a < ns1; ++a) {
          su += Lsx[qx * ns1 + a] * Ts[bb * ns1 + a];
          sd += Lsx[qx * ns1 + a] * Gs[bb * ns1 + a];
        }
        um += Lsy[qy * ns1 + bb] * su;
        dmv += Lsy[qy * ns1 + bb] * sd;
      }
      const T J = up - um;
      const T avg = T(0.5) * (A.cp2 * dpv + A.cm2 * dmv);
      const T W = A.Wq[t];
      al[t] = W * (A.gamma * J - avg);
      bp[t] = -T(0.5) * W * A.cp2 * J;
      bm[t] = -T(0.5) * W * A.cm2 * J;
    }
    __syncthreads();
    // fine face residual
    T* Rap = A.Rap + (long long)b * A.rbp + (long long)fcol * np1 * np1;
    T* Rbp = A.Rbp + (long long)b * A.rbp + (long long)fcol * np1 * np1;
    for (int t = tid; t < np1 * np1; t += blockDim.x) {
      const int a = t % np1, bb = t / np1;
      T sa = T(0), sb = T(0);
      for (int qy = 0; qy < q; ++qy) {
        T ta = T(0), tb = T(0);
        for (int qx = 0; qx < q; ++qx) {
          ta += Lp[qx * np1 + a] * al[qy * q + qx];
          tb += Lp[qx * np1 + a] * bp[qy * q + qx];
        }
        sa += Lp[qy * np1 + bb] * ta;
        sb += Lp[qy * np1 + bb] * tb;
      }
      Rap[t] = sa;
      Rbp[t] = sb;
    }
    // coarse face residual (accumulated over the fine faces in list order)
    for (int s = 0; s < 2; ++s) {
      const int t = tid + s * blockDim.x;
      if (t >= ns1 * ns1) continue;
      const int a = t % ns1, bb = t / ns1;
      T sa = T(0), sb = T(0);
      for (int qy = 0; qy < q; ++qy) {
        T ta = T(0), tb = T(0);
        for (int qx = 0; qx < q; ++qx) {
          ta += Lsx[qx * ns1 + a] * al[qy * q + qx];
          tb += Lsx[qx * ns1 + a] * bm[qy * q + qx];
        }
        sa += Lsy[qy * ns1 + bb] * ta;
        sb += Lsy[qy * ns1 + bb] * tb;
      }
      accA[s] -= sa;
      accB[s] += sb;
    }
  }
  T* Ras = A.Ras + (long long)b * A.rbs + (long long)ccol * ns1 * ns1;
  T* Rbs = A.Rbs + (long long)b * A.rbs + (long long)ccol * ns1 * ns1;
  for (int s = 0; s < 2; ++s) {
    const int t = tid + s * blockDim.x;
    if (t >= ns1 * ns1) continue;
    Ras[t] = accA[s];
    Rbs[t] = accB[s];
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

template <typename T>
__global__ void __launch_bounds__(256) pmut_recv_kernel(const __grid_constant__ PmutArgs<T> A) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int npw = A.B * A.K;
  if (warp < npw) {
    const int b = warp / A.K, k = warp - b * A.K;
    const int M = A.M;
    double g[DG_MAXM];
#pragma unroll
    for (int m = 0; m < DG_MAXM; ++m) g[m] = 0.0;
    const T* p = A.p_prev + (long long)b * A.bsp;
    const int e1 = A.fp_ptr[k + 1];
    for (int e = A.fp_ptr[k] + lane; e < e1; e += 32) {
      const double pv = (double)p[A.fp_off[e]];
      const double* Bv = A.Bm + (long long)e * M;
#pragma unroll
      for (int m = 0; m < DG_MAXM; ++m)
        if (m < M) g[m] += Bv[m] * pv;
    }
    double gm = 0.0;
#pragma unroll
    for (int m = 0; m < DG_MAXM; ++m) {
      if (m < M) {
        const double s = warp_sum(g[m]);
        if (lane == m) gm = s;
      }
    }
    if (lane < M) {
      const int km = k * M + lane;
      const long long idx = ((long long)b * A.K + k) * M + lane;
      const double dt = A.dt;
      const double q = A.q[idx], qd = A.qd[idx], qdd = A.qdd[idx];
      const double phi = A.drive ? A.drive[b * A.dbs + k * A.dks + A.n] : 0.0;
      const double qn = q + dt * qd + 0.5 * dt * dt * qdd;          // predictor
      const double qdp = qd + 0.5 * dt * qdd;
      const double qddn = -A.omega2[km] * qn - A.twozw[km] * qdp + (gm + A.eta[km] * phi) * A.inv_mu[km];
      A.q[idx] = qn;
      A.qd[idx] = qdp + 0.5 * dt * qddn;                                // corrector
      A.qdd[idx] = qddn;
    }
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
  if (lane == 0) A.traces[b * A.tbs + r * A.trs + A.n] = s;
}

}  // namespace

template <typename T>
cudaError_t launch_iface(const IfaceArgs<T>& a, int batch, cudaStream_t s) {
  if (a.ncf <= 0) return cudaSuccess;
  dim3 grid(a.ncf, batch);
  iface_kernel<T><<<grid, 128, 0, s>>>(a);
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

template cudaError_t launch_iface<float>(const IfaceArgs<float>&, int, cudaStream_t);
template cudaError_t launch_iface<double>(const IfaceArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pmut_recv<float>(const PmutArgs<float>&, cudaStream_t);
template cudaError_t launch_pmut_recv<double>(const PmutArgs<double>&, cudaStream_t);
