// Perfectly matched layer (Sec. 2, eq. full_problem rows 1-3): the auxiliary
// vector field Phi, stored element by element at the GLL nodes of the layer's
// elements, and its contribution to the pressure equation.
//
// One CTA per (layer element, batch member), one thread per element node:
//   psi^{n+1}   = psi^{n+1/2} + dt/2 p^{n+1}                    (nodal, read only)
//   grad p, grad psi at the node (1D GLL derivative along each axis)
//   Phi_d^{n+3/2} = [(1 - dt z_d/2) Phi_d^{n+1/2}
//                    + dt c^2 ((alpha - 2 z_d) d_d p + Z3_d d_d psi)] / (1 + dt z_d/2)
//   r_j = sum_q w_q |J| Phi^{n+1}(x_q) . grad psi_j(x_q),  Phi^{n+1} the mean of
//         the two half-step values (the int (div Phi) v term after integration
//         by parts; with collocated quadrature grad psi_j(x_q) is one 1D
//         derivative per axis)
// The residual is stored per element node, unassembled; the volume kernel
// gathers it node by node in a fixed order.
#include "internal.h"

namespace {

template <typename T, int N>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
    pml_kernel(const __grid_constant__ PmlArgs<T> A) {
  constexpr int NP = N + 1, NL = NP * NP * NP;
  __shared__ T sp[NL], sq[NL], sF[3][NL];
  const int e = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
  const int el = A.elem[e];
  const int ex = el % A.ne0, r1 = el / A.ne0;
  const int ey = r1 % A.ne1, ez = r1 / A.ne1;
  const int a = t % NP, bb = (t / NP) % NP, c = t / (NP * NP);
  const bool act = t < NL;
  if (act) {
    const long long g = (long long)b * A.bstride + (long long)(ez * N + c) * A.pz + (long long)(ey * N + bb) * A.py +
                        (ex * N + a);
    const T pv = A.p[g];
    sp[t] = pv;
    sq[t] = A.psi[g] + T(0.5) * A.dt * pv;
  }
  __syncthreads();
  if (act) {
    T gp[3] = {T(0), T(0), T(0)}, gs[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int ix = (c * NP + bb) * NP + q, iy = (c * NP + q) * NP + a, iz = (q * NP + bb) * NP + a;
      gp[0] += A.D[a][q] * sp[ix];
      gs[0] += A.D[a][q] * sq[ix];
      gp[1] += A.D[bb][q] * sp[iy];
      gs[1] += A.D[bb][q] * sq[iy];
      gp[2] += A.D[c][q] * sp[iz];
      gs[2] += A.D[c][q] * sq[iz];
    }
    const T z[3] = {A.zeta[0][ex * N + a], A.zeta[1][ey * N + bb], A.zeta[2][ez * N + c]};
    const T al = z[0] + z[1] + z[2];
    const T Z3[3] = {z[1] * z[2], z[2] * z[0], z[0] * z[1]};
    const T W = A.w[a] * A.w[bb] * A.w[c] * A.detJ;
    T* F = A.phi + (long long)b * A.phi_bs + (long long)e * 3 * NL;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const T Fo = F[d * NL + t];
      const T Fn = ((T(1) - T(0.5) * A.dt * z[d]) * Fo +
                    A.dt * A.c2 * ((al - T(2) * z[d]) * A.g[d] * gp[d] + Z3[d] * A.g[d] * gs[d])) /
                   (T(1) + T(0.5) * A.dt * z[d]);
      F[d * NL + t] = Fn;
      sF[d][t] = W * T(0.5) * (Fo + Fn);
    }
  }
  __syncthreads();
  if (act) {
    T r = T(0);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      r += A.g[0] * A.D[q][a] * sF[0][(c * NP + bb) * NP + q];
      r += A.g[1] * A.D[q][bb] * sF[1][(c * NP + q) * NP + a];
      r += A.g[2] * A.D[q][c] * sF[2][(q * NP + bb) * NP + a];
    }
    A.r[(long long)b * A.r_bs + (long long)e * NL + t] = r;
  }
}

template <typename T, int N>
cudaError_t launch_n(const PmlArgs<T>& a, int batch, cudaStream_t s) {
  constexpr int NL = (N + 1) * (N + 1) * (N + 1);
  pml_kernel<T, N><<<dim3(a.npml, batch), (NL + 31) / 32 * 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_pml(const PmlArgs<T>& a, int batch, cudaStream_t s) {
  if (a.npml <= 0 || batch <= 0) return cudaSuccess;
  switch (a.N) {
    case 1: return launch_n<T, 1>(a, batch, s);
    case 2: return launch_n<T, 2>(a, batch, s);
    case 3: return launch_n<T, 3>(a, batch, s);
    case 4: return launch_n<T, 4>(a, batch, s);
    case 5: return launch_n<T, 5>(a, batch, s);
    case 6: return launch_n<T, 6>(a, batch, s);
    case 7: return launch_n<T, 7>(a, batch, s);
    case 8: return launch_n<T, 8>(a, batch, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_pml<float>(const PmlArgs<float>&, int, cudaStream_t);
template cudaError_t launch_pml<double>(const PmlArgs<double>&, int, cudaStream_t);
