// Learned surrogate of the solver (project extension, no counterpart in the
// paper): MLP + transposed-convolution decoder, BF16 weights/activations with
// FP32 accumulation, MSE loss, Adam.  See include/surrogate.h.
//
// Dense layers run on the tensor cores (BF16 WMMA 16x16x16 fragments, FP32
// accumulators) with a fused epilogue (bias, GELU, BF16 copy); the three
// product shapes of a layer are  Z = A W^T (forward), dW = dZ^T A and
// dA = dZ W (backward).  The transposed convolutions are small and run on
// the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dgsem.h"
#include "../../include/surrogate.h"

using bf16 = __nv_bfloat16;

namespace {

thread_local std::string s_err;

int sfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  s_err = buf;
  return code;
}

#define S_TRY(expr)                                                                                \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return sfail(e_ == cudaErrorMemoryAllocation ? DGSEM_ENOMEM : DGSEM_ECUDA, "%s: %s", #expr, \
                   cudaGetErrorString(e_));                                                        \
  } while (0)

constexpr float kGeluS = 0.7978845608028654f;   // sqrt(2/pi)
constexpr float kGeluC = 0.044715f;

__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.f + tanhf(kGeluS * (z + kGeluC * z * z * z)));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float t = tanhf(kGeluS * (z + kGeluC * z * z * z));
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluS * (1.f + 3.f * kGeluC * z * z);
}

// ---------------------------------------------------------------------------
// C[M x N] = op(A) op(B) on the tensor cores.  TA = 0: A is [M][K] row-major;
// TA = 1: A is stored [K][M].  TB = 0: B is [K][N]; TB = 1: B is stored
// [N][K].  M, N multiples of 64, K a multiple of 16.  Epilogue: + bias[n],
// FP32 copy to C (ldc), BF16 copy of gelu(.) (act = 1) or of the value
// (act = 0) to Cb (ldcb).
// ---------------------------------------------------------------------------
struct Epi {
  const float* bias;
  float* C; int ldc;
  bf16* Cb; int ldcb; int act;
};

template <int TA, int TB>
__global__ void __launch_bounds__(128) gemm_bf16(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
                                                 int ldb, int M, int N, int K, Epi ep) {
  using namespace nvcuda;
  using LA = typename std::conditional<TA == 0, wmma::row_major, wmma::col_major>::type;
  using LB = typename std::conditional<TB == 0, wmma::row_major, wmma::col_major>::type;
  __shared__ float tile[64][64 + 4];
  const int warp = threadIdx.x >> 5;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int wm = m0 + (warp >> 1) * 32, wn = n0 + (warp & 1) * 32;
  wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) wmma::fill_fragment(acc[i][j], 0.f);
  for (int k0 = 0; k0 < K; k0 += 16) {
    wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, LA> fa[2];
    wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, LB> fb[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int m = wm + 16 * i;
      const bf16* pa = (TA == 0) ? A + (size_t)m * lda + k0 : A + (size_t)k0 * lda + m;
      wmma::load_matrix_sync(fa[i], pa, lda);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = wn + 16 * j;
      const bf16* pb = (TB == 0) ? B + (size_t)k0 * ldb + n : B + (size_t)n * ldb + k0;
      wmma::load_matrix_sync(fb[j], pb, ldb);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
      wmma::store_matrix_sync(&tile[(warp >> 1) * 32 + 16 * i][(warp & 1) * 32 + 16 * j], acc[i][j], 64 + 4,
                              wmma::mem_row_major);
  __syncthreads();
  for (int t = threadIdx.x; t < 64 * 64; t += 128) {
    const int r = t >> 6, c = t & 63;
    const int m = m0 + r, n = n0 + c;
    float v = tile[r][c];
    if (ep.bias) v += ep.bias[n];
    if (ep.C) ep.C[(size_t)m * ep.ldc + n] = v;
    if (ep.Cb) ep.Cb[(size_t)m * ep.ldcb + n] = __float2bfloat16(ep.act ? gelu_f(v) : v);
  }
}

template <int TA, int TB>
int gemm(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const Epi& ep, cudaStream_t s) {
  if (M % 64 || N % 64 || K % 16) return sfail(DGSEM_EINVAL, "gemm shape %d x %d x %d not tileable", M, N, K);
  dim3 grid(N / 64, M / 64);
  gemm_bf16<TA, TB><<<grid, 128, 0, s>>>(A, lda, B, ldb, M, N, K, ep);
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

// ---------------------------------------------------------------------------
// element-wise and small kernels
// ---------------------------------------------------------------------------
__global__ void to_bf16(const float* __restrict__ x, bf16* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// dz = da * gelu'(z) (FP32) and its BF16 copy
__global__ void gelu_bwd(const float* __restrict__ da, const float* __restrict__ z, float* __restrict__ dz,
                         bf16* __restrict__ dzb, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float g = da[i] * gelu_grad_f(z[i]);
    dz[i] = g;
    dzb[i] = __float2bfloat16(g);
  }
}

// db[n] = sum_m dz[m][n]
__global__ void col_sum(const float* __restrict__ dz, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dz[(size_t)m * N + n];
  db[n] = s;
}

// v[b][co][t] = bias[co] + sum_{ci, k: t = 2i - 1 + k} u[b][ci][i] W[ci][co][k]
// (ConvTranspose1d, kernel 4, stride 2, padding 1); u_next = bf16(gelu(v)) if act
__global__ void convt_fwd(const bf16* __restrict__ u, const bf16* __restrict__ W, const float* __restrict__ bias,
                          int B, int Ci, int Co, int Ti, float* __restrict__ v, bf16* __restrict__ u_next, int act) {
  const int To = 2 * Ti;
  const size_t n = (size_t)B * Co * To;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx % To);
    const int co = (int)((idx / To) % Co);
    const int b = (int)(idx / ((size_t)To * Co));
    float s = bias[co];
    for (int k = 0; k < 4; ++k) {
      const int r = t + 1 - k;
      if (r < 0 || (r & 1)) continue;
      const int i = r >> 1;
      if (i >= Ti) continue;
      const bf16* up = u + ((size_t)b * Ci) * Ti + i;
      const bf16* wp = W + (size_t)co * 4 + k;
      for (int ci = 0; ci < Ci; ++ci)
        s += __bfloat162float(up[(size_t)ci * Ti]) * __bfloat162float(wp[(size_t)ci * Co * 4]);
    }
    v[idx] = s;
    if (u_next) u_next[idx] = __float2bfloat16(act ? gelu_f(s) : s);
  }
}

// du[b][ci][i] = sum_{co, k} dv[b][co][2i - 1 + k] W[ci][co][k]
__global__ void convt_bwd_data(const float* __restrict__ dv, const bf16* __restrict__ W, int B, int Ci, int Co, int Ti,
                               float* __restrict__ du) {
  const int To = 2 * Ti;
  const size_t n = (size_t)B * Ci * Ti;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % Ti);
    const int ci = (int)((idx / Ti) % Ci);
    const int b = (int)(idx / ((size_t)Ti * Ci));
    float s = 0.f;
    for (int k = 0; k < 4; ++k) {
      const int t = 2 * i - 1 + k;
      if (t < 0 || t >= To) continue;
      const float* dp = dv + ((size_t)b * Co) * To + t;
      const bf16* wp = W + ((size_t)ci * Co) * 4 + k;
      for (int co = 0; co < Co; ++co) s += dp[(size_t)co * To] * __bfloat162float(wp[(size_t)co * 4]);
    }
    du[idx] = s;
  }
}

// dW[ci][co][k] = sum_{b, i} u[b][ci][i] dv[b][co][2i - 1 + k]
__global__ void convt_bwd_weight(const bf16* __restrict__ u, const float* __restrict__ dv, int B, int Ci, int Co,
                                 int Ti, float* __restrict__ dW) {
  const int To = 2 * Ti;
  const size_t n = (size_t)Ci * Co * 4;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % 4);
    const int co = (int)((idx / 4) % Co);
    const int ci = (int)(idx / ((size_t)4 * Co));
    float s = 0.f;
    for (int b = 0; b < B; ++b) {
      const bf16* up = u + ((size_t)b * Ci + ci) * Ti;
      const float* dp = dv + ((size_t)b * Co + co) * To;
      for (int i = 0; i < Ti; ++i) {
        const int t = 2 * i - 1 + k;
        if (t >= 0 && t < To) s += __bfloat162float(up[i]) * dp[t];
      }
    }
    dW[idx] = s;
  }
}

// db[co] = sum_{b, t} dv[b][co][t]
__global__ void convt_bwd_bias(const float* __restrict__ dv, int B, int Co, int To, float* __restrict__ db) {
  const int co = blockIdx.x * blockDim.x + threadIdx.x;
  if (co >= Co) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b)
    for (int t = 0; t < To; ++t) s += dv[((size_t)b * Co + co) * To + t];
  db[co] = s;
}

// dv = du * gelu'(v)
__global__ void act_bwd(const float* __restrict__ du, const float* __restrict__ v, float* __restrict__ dv, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dv[i] = du[i] * gelu_grad_f(v[i]);
}

// dy = 2 (y - target) / n, loss += sum (y - target)^2 / n
__global__ void mse(const float* __restrict__ y, const float* __restrict__ tgt, float* __restrict__ dy, size_t n,
                    double* __restrict__ loss) {
  double s = 0.0;
  const float inv = 1.0f / (float)n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = y[i] - tgt[i];
    dy[i] = 2.f * d * inv;
    s += (double)d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s / (double)n);
}

// Adam with bias correction on the FP32 masters; refresh the BF16 copies
__global__ void adam(float* __restrict__ p, bf16* __restrict__ pb, const float* __restrict__ g, float* __restrict__ m,
                     float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float q = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = q;
    pb[i] = __float2bfloat16(q);
  }
}

constexpr int EW_BLOCKS = 4 * 152, EW_THREADS = 256;

}  // namespace

// ---------------------------------------------------------------------------
// network object
// ---------------------------------------------------------------------------
struct srg_net {
  srg_config cfg;
  int max_batch = 0;
  int device = 0;
  size_t np = 0;
  std::vector<size_t> offW, offB;     // per layer (hidden..., decoder, convs...)
  float* P = nullptr; bf16* Pb = nullptr; float* G = nullptr; float* M1 = nullptr; float* M2 = nullptr;
  // activations
  std::vector<bf16*> a;               // [n_hidden + 1], a[0] = bf16(x)
  std::vector<float*> z;              // [n_hidden]
  float* zd = nullptr;                // decoder output
  std::vector<bf16*> u;               // [n_conv]: u[0] = bf16(zd), u[j] = bf16(gelu(v[j-1]))
  std::vector<float*> v;              // [n_conv]
  // gradients
  float *gv = nullptr, *gu = nullptr, *ga = nullptr, *gz = nullptr;
  bf16* gzb = nullptr;
  double* d_loss = nullptr;
  long long t = 0;                    // Adam step counter
  std::vector<void*> allocs;
};

namespace {

int salloc(srg_net* n, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return sfail(DGSEM_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  n->allocs.push_back(*p);
  return DGSEM_OK;
}

int conv_len(const srg_config& c, int j) { return c.t0 << j; }        // input length of conv j
int conv_cin(const srg_config& c, int j) { return j == 0 ? c.c0 : c.conv_ch[j - 1]; }

// forward pass keeping every activation; returns the output buffer
int forward_impl(srg_net* n, const float* x, int B, cudaStream_t s) {
  const srg_config& c = n->cfg;
  to_bf16<<<EW_BLOCKS, EW_THREADS, 0, s>>>(x, n->a[0], (size_t)B * c.d_in);
  S_TRY(cudaGetLastError());
  int fan = c.d_in;
  for (int l = 0; l < c.n_hidden; ++l) {
    Epi ep{n->P + n->offB[l], n->z[l], c.hidden, n->a[l + 1], c.hidden, 1};
    int rc = gemm<0, 1>(n->a[l], fan, n->Pb + n->offW[l], fan, B, c.hidden, fan, ep, s);
    if (rc) return rc;
    fan = c.hidden;
  }
  const int L = c.n_hidden;
  const int nd = c.c0 * c.t0;
  Epi ep{n->P + n->offB[L], n->zd, nd, n->u[0], nd, 0};
  int rc = gemm<0, 1>(n->a[L], fan, n->Pb + n->offW[L], fan, B, nd, fan, ep, s);
  if (rc) return rc;
  for (int j = 0; j < c.n_conv; ++j) {
    const int last = j == c.n_conv - 1;
    convt_fwd<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->u[j], n->Pb + n->offW[L + 1 + j], n->P + n->offB[L + 1 + j], B,
                                               conv_cin(c, j), c.conv_ch[j], conv_len(c, j), n->v[j],
                                               last ? nullptr : n->u[j + 1], 1);
    S_TRY(cudaGetLastError());
  }
  return DGSEM_OK;
}

int check_batch(const srg_net* n, int B) {
  if (B < 64 || B % 64 || B > n->max_batch)
    return sfail(DGSEM_EINVAL, "batch %d must be a positive multiple of 64 and <= max_batch %d", B, n->max_batch);
  return DGSEM_OK;
}

}  // namespace

extern "C" {

const char* srg_last_error(void) { return s_err.c_str(); }

int srg_create(const srg_config* cfg, int max_batch, unsigned long long seed, srg_net** out) {
  if (!cfg || !out) return sfail(DGSEM_EINVAL, "NULL argument");
  *out = nullptr;
  const srg_config& c = *cfg;
  if (c.d_in < 64 || c.d_in % 64 || c.hidden < 64 || c.hidden % 64 || c.n_hidden < 1 || c.n_hidden > 16)
    return sfail(DGSEM_EINVAL, "d_in and hidden must be positive multiples of 64, 1 <= n_hidden <= 16");
  if (c.c0 < 1 || c.t0 < 1 || (c.c0 * c.t0) % 64 || c.n_conv < 1 || c.n_conv > 8)
    return sfail(DGSEM_EINVAL, "c0*t0 must be a multiple of 64 and 1 <= n_conv <= 8");
  for (int j = 0; j < c.n_conv; ++j)
    if (c.conv_ch[j] < 1) return sfail(DGSEM_EINVAL, "conv_ch[%d] < 1", j);
  if (max_batch < 64 || max_batch % 64) return sfail(DGSEM_EINVAL, "max_batch must be a positive multiple of 64");
  srg_net* n = new srg_net();
  n->cfg = c;
  n->max_batch = max_batch;
  cudaGetDevice(&n->device);
  // parameter layout
  size_t o = 0;
  int fan = c.d_in;
  std::vector<int> fans, outs;
  for (int l = 0; l <= c.n_hidden; ++l) {
    const int out_f = l < c.n_hidden ? c.hidden : c.c0 * c.t0;
    n->offW.push_back(o); o += (size_t)out_f * fan;
    n->offB.push_back(o); o += out_f;
    fans.push_back(fan); outs.push_back(out_f);
    fan = out_f;
  }
  for (int j = 0; j < c.n_conv; ++j) {
    const int ci = conv_cin(c, j), co = c.conv_ch[j];
    n->offW.push_back(o); o += (size_t)ci * co * 4;
    n->offB.push_back(o); o += co;
    fans.push_back(ci * 4); outs.push_back(co);
  }
  n->np = o;
  // deterministic initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a 64-bit LCG
  std::vector<float> h(o);
  unsigned long long st = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) / 9007199254740992.0;
  };
  for (size_t layer = 0; layer < n->offW.size(); ++layer) {
    const size_t w0 = n->offW[layer], b0 = n->offB[layer];
    const size_t w1 = b0, b1 = (layer + 1 < n->offW.size()) ? n->offW[layer + 1] : o;
    const double lim = 1.0 / std::sqrt((double)fans[layer]);
    for (size_t i = w0; i < w1; ++i) h[i] = (float)((2.0 * uni() - 1.0) * lim);
    for (size_t i = b0; i < b1; ++i) h[i] = (float)((2.0 * uni() - 1.0) * lim);
  }
  int rc;
  auto A = [&](void** p, size_t bytes) { return salloc(n, p, bytes); };
  if ((rc = A((void**)&n->P, o * 4)) || (rc = A((void**)&n->Pb, o * 2)) || (rc = A((void**)&n->G, o * 4)) ||
      (rc = A((void**)&n->M1, o * 4)) || (rc = A((void**)&n->M2, o * 4)) || (rc = A((void**)&n->d_loss, 8))) {
    srg_destroy(n);
    return rc;
  }
  const size_t B = (size_t)max_batch;
  n->a.resize(c.n_hidden + 1);
  n->z.resize(c.n_hidden);
  if ((rc = A((void**)&n->a[0], B * c.d_in * 2))) { srg_destroy(n); return rc; }
  for (int l = 0; l < c.n_hidden; ++l)
    if ((rc = A((void**)&n->a[l + 1], B * c.hidden * 2)) || (rc = A((void**)&n->z[l], B * c.hidden * 4))) {
      srg_destroy(n);
      return rc;
    }
  const size_t nd = (size_t)c.c0 * c.t0;
  n->u.resize(c.n_conv);
  n->v.resize(c.n_conv);
  if ((rc = A((void**)&n->zd, B * nd * 4)) || (rc = A((void**)&n->u[0], B * nd * 2))) { srg_destroy(n); return rc; }
  size_t maxc = nd;
  for (int j = 0; j < c.n_conv; ++j) {
    const size_t outn = (size_t)c.conv_ch[j] * conv_len(c, j + 1);
    maxc = std::max(maxc, outn);
    if ((rc = A((void**)&n->v[j], B * outn * 4))) { srg_destroy(n); return rc; }
    if (j + 1 < c.n_conv && (rc = A((void**)&n->u[j + 1], B * outn * 2))) { srg_destroy(n); return rc; }
  }
  const size_t maxw = std::max((size_t)c.hidden, (size_t)c.d_in);
  if ((rc = A((void**)&n->gv, B * maxc * 4)) || (rc = A((void**)&n->gu, B * maxc * 4)) ||
      (rc = A((void**)&n->ga, B * std::max(maxw, nd) * 4)) || (rc = A((void**)&n->gz, B * std::max(maxw, nd) * 4)) ||
      (rc = A((void**)&n->gzb, B * std::max(maxw, nd) * 2))) {
    srg_destroy(n);
    return rc;
  }
  if ((rc = srg_set_params(n, h.data(), o))) { srg_destroy(n); return rc; }
  S_TRY(cudaMemset(n->M1, 0, o * 4));
  S_TRY(cudaMemset(n->M2, 0, o * 4));
  S_TRY(cudaMemset(n->G, 0, o * 4));
  *out = n;
  return DGSEM_OK;
}

size_t srg_num_params(const srg_net* n) { return n ? n->np : 0; }

int srg_get_params(const srg_net* n, float* host, size_t len) {
  if (!n || !host || len < n->np) return sfail(DGSEM_EINVAL, "bad arguments");
  S_TRY(cudaMemcpy(host, n->P, n->np * 4, cudaMemcpyDeviceToHost));
  return DGSEM_OK;
}

int srg_get_grads(const srg_net* n, float* host, size_t len) {
  if (!n || !host || len < n->np) return sfail(DGSEM_EINVAL, "bad arguments");
  S_TRY(cudaMemcpy(host, n->G, n->np * 4, cudaMemcpyDeviceToHost));
  return DGSEM_OK;
}

int srg_set_params(srg_net* n, const float* host, size_t len) {
  if (!n || !host || len < n->np) return sfail(DGSEM_EINVAL, "bad arguments");
  S_TRY(cudaMemcpy(n->P, host, n->np * 4, cudaMemcpyHostToDevice));
  to_bf16<<<EW_BLOCKS, EW_THREADS>>>(n->P, n->Pb, n->np);
  S_TRY(cudaGetLastError());
  S_TRY(cudaDeviceSynchronize());
  return DGSEM_OK;
}

int srg_forward(srg_net* n, const float* x, int B, float* y, void* stream) {
  if (!n || !x || !y) return sfail(DGSEM_EINVAL, "NULL argument");
  int rc = check_batch(n, B);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = forward_impl(n, x, B, s))) return rc;
  const srg_config& c = n->cfg;
  const size_t outn = (size_t)B * c.conv_ch[c.n_conv - 1] * conv_len(c, c.n_conv);
  S_TRY(cudaMemcpyAsync(y, n->v[c.n_conv - 1], outn * 4, cudaMemcpyDeviceToDevice, s));
  S_TRY(cudaStreamSynchronize(s));
  return DGSEM_OK;
}

int srg_backward(srg_net* n, const float* x, const float* target, int B, double* loss, void* stream) {
  if (!n || !x || !target) return sfail(DGSEM_EINVAL, "NULL argument");
  int rc = check_batch(n, B);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = forward_impl(n, x, B, s))) return rc;
  const srg_config& c = n->cfg;
  const int L = c.n_hidden, J = c.n_conv;
  // loss and dy (into gv)
  const size_t outn = (size_t)B * c.conv_ch[J - 1] * conv_len(c, J);
  S_TRY(cudaMemsetAsync(n->d_loss, 0, 8, s));
  mse<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->v[J - 1], target, n->gv, outn, n->d_loss);
  S_TRY(cudaGetLastError());
  // transposed convolutions, last to first: gv holds dv_j, gu receives du_j
  for (int j = J - 1; j >= 0; --j) {
    const int ci = conv_cin(c, j), co = c.conv_ch[j], ti = conv_len(c, j);
    convt_bwd_weight<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->u[j], n->gv, B, ci, co, ti, n->G + n->offW[L + 1 + j]);
    convt_bwd_bias<<<(co + 127) / 128, 128, 0, s>>>(n->gv, B, co, 2 * ti, n->G + n->offB[L + 1 + j]);
    convt_bwd_data<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->gv, n->Pb + n->offW[L + 1 + j], B, ci, co, ti, n->gu);
    S_TRY(cudaGetLastError());
    if (j > 0) {
      act_bwd<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->gu, n->v[j - 1], n->gv, (size_t)B * ci * ti);
      S_TRY(cudaGetLastError());
    }
  }
  // decoder: dzd = du_0 (FP32 in gu), BF16 copy in gzb
  const int nd = c.c0 * c.t0;
  to_bf16<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->gu, n->gzb, (size_t)B * nd);
  col_sum<<<(nd + 127) / 128, 128, 0, s>>>(n->gu, B, nd, n->G + n->offB[L]);
  S_TRY(cudaGetLastError());
  Epi ew{nullptr, n->G + n->offW[L], c.hidden, nullptr, 0, 0};
  if ((rc = gemm<1, 0>(n->gzb, nd, n->a[L], c.hidden, nd, c.hidden, B, ew, s))) return rc;
  Epi ea{nullptr, n->ga, c.hidden, nullptr, 0, 0};
  if ((rc = gemm<0, 0>(n->gzb, nd, n->Pb + n->offW[L], c.hidden, B, c.hidden, nd, ea, s))) return rc;
  // hidden layers, last to first
  for (int l = L - 1; l >= 0; --l) {
    const int fan = l == 0 ? c.d_in : c.hidden;
    gelu_bwd<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->ga, n->z[l], n->gz, n->gzb, (size_t)B * c.hidden);
    col_sum<<<(c.hidden + 127) / 128, 128, 0, s>>>(n->gz, B, c.hidden, n->G + n->offB[l]);
    S_TRY(cudaGetLastError());
    Epi eW{nullptr, n->G + n->offW[l], fan, nullptr, 0, 0};
    if ((rc = gemm<1, 0>(n->gzb, c.hidden, n->a[l], fan, c.hidden, fan, B, eW, s))) return rc;
    if (l > 0) {
      Epi eA{nullptr, n->ga, c.hidden, nullptr, 0, 0};
      if ((rc = gemm<0, 0>(n->gzb, c.hidden, n->Pb + n->offW[l], fan, B, fan, c.hidden, eA, s))) return rc;
    }
  }
  double l_host = 0.0;
  S_TRY(cudaMemcpyAsync(&l_host, n->d_loss, 8, cudaMemcpyDeviceToHost, s));
  S_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = l_host;
  return DGSEM_OK;
}

int srg_adam_step(srg_net* n, float lr, float b1, float b2, float eps, void* stream) {
  if (!n) return sfail(DGSEM_EINVAL, "NULL argument");
  n->t += 1;
  const float c1 = 1.f - std::pow(b1, (float)n->t), c2 = 1.f - std::pow(b2, (float)n->t);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  adam<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->P, n->Pb, n->G, n->M1, n->M2, n->np, lr, b1, b2, eps, c1, c2);
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

int srg_train_step(srg_net* n, const float* x, const float* target, int B, float lr, double* loss, void* stream) {
  int rc = srg_backward(n, x, target, B, loss, stream);
  if (rc) return rc;
  return srg_adam_step(n, lr, 0.9f, 0.999f, 1e-8f, stream);
}

void srg_destroy(srg_net* n) {
  if (!n) return;
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

}  // extern "C"
