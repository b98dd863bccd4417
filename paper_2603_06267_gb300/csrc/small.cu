// Interface fluxes on Gamma_I (Sec. 5, eq. Wf_2 interface terms) and the
// PMUT modal step with receiver sampling (Algorithm 1 PMUT rows, eqs. g_m).
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

template <typename T>
__global__ void __launch_bounds__(IF_THREADS) iface_kernel(const __grid_constant__ IfaceArgs<T> A, int batch) {
  __shared__ T Lp[DG_MAXQ * NP1];
  __shared__ T Ts[NP1 * NP1], Gs[NP1 * NP1];
  __shared__ T Tp[FG][NP1 * NP1], Gp[FG][NP1 * NP1];
  __shared__ T Lsx[FG][DG_MAXQ * NP1], Lsy[FG][DG_MAXQ * NP1];
  __shared__ T al[FG][DG_MAXQ * DG_MAXQ], bp[FG][DG_MAXQ * DG_MAXQ], bm[FG][DG_MAXQ * DG_MAXQ];
  __shared__ T accA[NP1 * NP1], accB[NP1 * NP1];
  const int cf = blockIdx.x;
  const int tid = threadIdx.x;
  const int Np = A.Np, Ns = A.Ns, q = A.q, qq = q * q;
  const int np1 = Np + 1, ns1 = Ns + 1, nf2 = np1 * np1, ns2 = ns1 * ns1;
  const int ccol = A.cf_col[cf];
  const int mx = ccol % A.nsx, my = ccol / A.nsx;
  const int f0 = A.cf_ptr[cf], f1 = A.cf_ptr[cf + 1];
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
      Ts[t] = ps[base];
      Gs[t] = g;
      accA[t] = T(0);
      accB[t] = T(0);
    }
    for (int g0 = f0; g0 < f1; g0 += FG) {
      const int nfg = min(FG, f1 - g0);
      __syncthreads();
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
        Tp[f][r] = pp[base + (long long)Np * A.pzp];
        Gp[f][r] = g;
      }
      __syncthreads();
      for (int t = tid; t < nfg * qq; t += IF_THREADS) {
        const int f = t / qq, r = t - f * qq;
        const int qx = r % q, qy = r / q;
        T up = T(0), dpv = T(0);
        for (int bb = 0; bb < np1; ++bb) {
          T su = T(0), sd = T(0);
          for (int a = 0; a < np1; ++a) {
            su += Lp[qx * np1 + a] * Tp[f][bb * np1 + a];
            sd += Lp[qx * np1 + a] * Gp[f][bb * np1 + a];
          }
          up += Lp[qy * np1 + bb] * su;
          dpv += Lp[qy * np1 + bb] * sd;
        }
        T um = T(0), dmv = T(0);
        for (int bb = 0; bb < ns1; ++bb) {
          T su = T(0), sd = T(0);
          for (int a = 0; a < ns1; ++a) {
            su += Lsx[f][qx * ns1 + a] * Ts[bb * ns1 + a];
            sd += Lsx[f][qx * ns1 + a] * Gs[bb * ns1 + a];
          }
          um += Lsy[f][qy * ns1 + bb] * su;
          dmv += Lsy[f][qy * ns1 + bb] * sd;
        }
        const T J = up - um;
        const T avg = T(0.5) * (A.cp2 * dpv + A.cm2 * dmv);
        const T W = A.Wq[r];
        al[f][r] = W * (A.gamma * J - avg);
        bp[f][r] = -T(0.5) * W * A.cp2 * J;
        bm[f][r] = -T(0.5) * W * A.cm2 * J;
      }
      __syncthreads();
      // fine face residuals, then the coarse residual of this group (fixed order)
      for (int t = tid; t < nfg * nf2 + ns2; t += IF_THREADS) {
        if (t < nfg * nf2) {
          const int f = t / nf2, r = t - f * nf2;
          const int a = r % np1, bb = r / np1;
          T sa = T(0), sb = T(0);
          for (int qy = 0; qy < q; ++qy) {
            T ta = T(0), tb = T(0);
            for (int qx = 0; qx < q; ++qx) {
              ta += Lp[qx * np1 + a] * al[f][qy * q + qx];
              tb += Lp[qx * np1 + a] * bp[f][qy * q + qx];
            }
            sa += Lp[qy * np1 + bb] * ta;
            sb += Lp[qy * np1 + bb] * tb;
          }
          const long long o = (long long)b * A.rbp + (long long)A.ff_col[g0 + f] * nf2 + r;
          A.Rap[o] = sa;
          A.Rbp[o] = sb;
        } else {
          const int r = t - nfg * nf2;
          const int a = r % ns1, bb = r / ns1;
          T sa_tot = accA[r], sb_tot = accB[r];
          for (int f = 0; f < nfg; ++f) {
            T sa = T(0), sb = T(0);
            for (int qy = 0; qy < q; ++qy) {
              T ta = T(0), tb = T(0);
              for (int qx = 0; qx < q; ++qx) {
                ta += Lsx[f][qx * ns1 + a] * al[f][qy * q + qx];
                tb += Lsx[f][qx * ns1 + a] * bm[f][qy * q + qx];
              }
              sa += Lsy[f][qy * ns1 + bb] * ta;
              sb += Lsy[f][qy * ns1 + bb] * tb;
            }
            sa_tot -= sa;
            sb_tot += sb;
          }
          accA[r] = sa_tot;
          accB[r] = sb_tot;
        }
      }
    }
    __syncthreads();
    for (int t = tid; t < ns2; t += IF_THREADS) {
      const long long o = (long long)b * A.rbs + (long long)ccol * ns2 + t;
      A.Ras[o] = accA[t];
      A.Rbs[o] = accB[t];
    }
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
      const int n = A.n + (A.step ? *A.step : 0);
      const double phi = A.drive ? A.drive[b * A.dbs + k * A.dks + n] : 0.0;
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
  if (lane == 0) A.traces[b * A.tbs + r * A.trs + A.n + (A.step ? *A.step : 0)] = s;
}

// ---------------------------------------------------------------------------
// Power-iteration helpers (setup only): M-weighted dot product over a box
// lattice with the lumped mass M = scale * w_x(i) w_y(j) w_z(k), and scaling.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) mdot_kernel(const double* __restrict__ x, const double* __restrict__ y,
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
    s += wx[i] * wy[j] * wz[k] * x[g] * y[g];
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

__global__ void scale_kernel(double* __restrict__ x, const double* __restrict__ y, double a, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    x[t] = a * y[t];
}

}  // namespace

cudaError_t launch_mdot(const double* x, const double* y, const double* wx, const double* wy, const double* wz, int L0,
                        int L1, int L2, int py, long long pz, double scale, double* out, cudaStream_t s) {
  mdot_kernel<<<4 * 152, 256, 0, s>>>(x, y, wx, wy, wz, L0, L1, L2, py, pz, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_scale(double* x, const double* y, double a, long long n, cudaStream_t s) {
  scale_kernel<<<4 * 152, 256, 0, s>>>(x, y, a, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_iface(const IfaceArgs<T>& a, int batch, cudaStream_t s) {
  if (a.ncf <= 0) return cudaSuccess;
  dim3 grid(a.ncf, (batch + IF_BPC - 1) / IF_BPC);
  iface_kernel<T><<<grid, IF_THREADS, 0, s>>>(a, batch);
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
