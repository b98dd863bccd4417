// Learned surrogate of the solver (project extension, no counterpart in the
// paper): MLP + transposed-convolution decoder, BF16 weights/activations with
// FP32 accumulation, MSE loss, Adam.  See include/surrogate.h.
//
// Dense layers run on the tcgen05 tensor cores (tc_gemm.cuh: TMA-fed shared-
// memory operands, FP32 accumulators in tensor memory) with a fused epilogue
// (bias, GELU, BF16 copy).  Every product is taken in the form C = A B^T with
// both operands K-contiguous: the forward Z = A W^T directly; the backward
// dW = dZ^T A and dA = dZ W after BF16 transposes of dZ, A and W.  The
// transposed convolutions are small and run on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cuda.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dgsem.h"
#include "../../include/surrogate.h"
#include "tc_gemm.cuh"

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
// Dense products on the tcgen05 tensor cores: C[M x N] = A B^T, A [M][K] and
// B [N][K] BF16 row-major (K contiguous), K a multiple of 64, N a multiple of
// 64.  Rows of A beyond M are read as zeros (TMA fill) and not written.
// ---------------------------------------------------------------------------
using tcg::Epi;

struct DenseEpi {
  Epi e;
  __device__ __forceinline__ void operator()(int m, int n, const uint32_t* r) const {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + (e.bias ? e.bias[n + j] : 0.f);
    if (e.C) {
      float4* dst = reinterpret_cast<float4*>(e.C + (size_t)m * e.ldc + n);
#pragma unroll
      for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (e.Cb) {
      uint4* dst = reinterpret_cast<uint4*>(e.Cb + (size_t)m * e.ldcb + n);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float a = e.act ? gelu_f(v[8 * q + 2 * h]) : v[8 * q + 2 * h];
          const float b = e.act ? gelu_f(v[8 * q + 2 * h + 1]) : v[8 * q + 2 * h + 1];
          const __nv_bfloat162 p2 = __floats2bfloat162_rn(a, b);
          w[h] = *reinterpret_cast<const uint32_t*>(&p2);
        }
        dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2-D tensor map of a BF16 [rows][ld] matrix (cols = K used) for box_rows x 64
// tiles with 128-byte swizzle
int tmap_bf16(CUtensorMap* map, const bf16* base, int rows, int cols, int ld, int box_rows) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return sfail(DGSEM_ECUDA, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  if (reinterpret_cast<uintptr_t>(base) % 16 || (ld * 2) % 16) return sfail(DGSEM_EINVAL, "gemm operand misaligned");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)tcg::BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return sfail(DGSEM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGSEM_OK;
}

template <int BN, int STAGES>
int tc_launch(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const Epi& ep, int* err,
              cudaStream_t s) {
  CUtensorMap ta, tb;
  int rc;
  if ((rc = tmap_bf16(&ta, A, M, K, lda, tcg::BM)) || (rc = tmap_bf16(&tb, B, N, K, ldb, BN))) return rc;
  auto kern = tcg::gemm_kernel<BN, STAGES, DenseEpi>;
  constexpr int smem = tcg::Geo<BN, STAGES>::SMEM;
  S_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  dim3 grid(N / BN, (M + tcg::BM - 1) / tcg::BM);
  kern<<<grid, tcg::THREADS, smem, s>>>(ta, tb, M, K, DenseEpi{ep}, err, tcg::DenseA());
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

// C = A B^T with the tile width that gives the most CTAs up to one wave
int gemm_nt(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const Epi& ep, int* err,
            cudaStream_t s) {
  if (M < 1 || N % 64 || K % 64 || K < 64) return sfail(DGSEM_EINVAL, "gemm shape %d x %d x %d not tileable", M, N, K);
  const int mt = (M + tcg::BM - 1) / tcg::BM;
  // enough 128-wide tiles to fill the GPU: a three-stage ring (100 KB), so two CTAs
  // share an SM and a grid of up to 2 x 152 tiles runs in one wave
  if (N % 128 == 0 && mt * (N / 128) >= 148) return tc_launch<128, 3>(A, lda, B, ldb, M, N, K, ep, err, s);
  return tc_launch<64, 6>(A, lda, B, ldb, M, N, K, ep, err, s);
}

// out[c][r] = in[r][c] for a BF16 [R][C] matrix (blockIdx.z: one of a batch of them)
__global__ void transpose_bf16(const bf16* __restrict__ in, int R, int C, bf16* __restrict__ out) {
  __shared__ bf16 t[32][34];
  in += (size_t)blockIdx.z * R * C;
  out += (size_t)blockIdx.z * R * C;
  const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int r = r0 + i;
    if (r < R && c < C) t[i][threadIdx.x] = in[(size_t)r * C + c];
  }
  __syncthreads();
  const int r = r0 + threadIdx.x;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int cc = blockIdx.x * 32 + i;
    if (cc < C && r < R) out[(size_t)cc * R + r] = t[threadIdx.x][i];
  }
}

int transpose(const bf16* in, int R, int C, bf16* out, cudaStream_t s, int nbatch = 1) {
  dim3 grid((C + 31) / 32, (R + 31) / 32, nbatch);
  transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(in, R, C, out);
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

// ---------------------------------------------------------------------------
// Transposed convolution (kernel 4, stride 2, padding 1) on the tensor cores.
// Output sample t = 2m + par of channel co takes two taps of every input
// channel:  even (par 0): W[.][co][1] u[m] + W[.][co][3] u[m - 1];  odd
// (par 1): W[.][co][0] u[m + 1] + W[.][co][2] u[m].  With u in time-major
// layout [b][t][ci] each parity is one product C[(b, m)][co] = A B^T, K = 2 Ci:
// A's first Ci columns are u at time m + sh0, the next Ci at m + sh1 (zeros
// past either end), B = [W_k0 | W_k1]^T per output channel.
// ---------------------------------------------------------------------------
// Be / Bo [Co][2 Ci]: the even and odd tap pairs of W [Ci][Co][4]
__global__ void convt_taps(const bf16* __restrict__ W, int Ci, int Co, bf16* __restrict__ Be, bf16* __restrict__ Bo) {
  const size_t n = (size_t)Ci * Co;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int co = (int)(idx % Co), ci = (int)(idx / Co);
    const bf16* w = W + ((size_t)ci * Co + co) * 4;
    Be[(size_t)co * 2 * Ci + ci] = w[1];
    Be[(size_t)co * 2 * Ci + Ci + ci] = w[3];
    Bo[(size_t)co * 2 * Ci + ci] = w[0];
    Bo[(size_t)co * 2 * Ci + Ci + ci] = w[2];
  }
}

// Both parities in one product: K = 3 Ci over the input at times m - 1, m,
// m + 1, N = 2 Co with B3[co] = [W_3 | W_1 | 0] (even output) and
// B3[Co + co] = [0 | W_2 | W_0] (odd); the accumulator's column halves hold
// the even and odd samples of a channel, written as adjacent pairs.
__global__ void convt_taps3(const bf16* __restrict__ W, int Ci, int Co, bf16* __restrict__ B3) {
  const size_t n = (size_t)Ci * Co;
  const bf16 zero = __float2bfloat16(0.f);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int co = (int)(idx % Co), ci = (int)(idx / Co);
    const bf16* w = W + ((size_t)ci * Co + co) * 4;
    bf16* ev = B3 + (size_t)co * 3 * Ci;
    bf16* od = B3 + (size_t)(Co + co) * 3 * Ci;
    ev[ci] = w[3]; ev[Ci + ci] = w[1]; ev[2 * Ci + ci] = zero;
    od[ci] = zero; od[Ci + ci] = w[2]; od[2 * Ci + ci] = w[0];
  }
}

// rows (b, m), channels n .. n + 31: v[b][co][2m], v[b][co][2m + 1] (+ bias)
// as adjacent pairs (channel-major), and u_next = bf16(gelu(v)): channel-major
// [b][co][t] like v, or (tm) time-major [b][t][co], the layout the next
// transposed convolution reads, 32 consecutive channels per sample
struct PairConvEpi {
  static constexpr bool paired = true;
  float* v; bf16* un; const float* bias; int T, Co, tm;
  __device__ __forceinline__ void operator()(int r, int n, const uint32_t* ev, const uint32_t* od) const {
    const int b = r / T, m = r % T, To = 2 * T;
    const size_t o = ((size_t)b * Co + n) * To + 2 * m;
    if (un && tm) {
      bf16* ue = un + ((size_t)b * To + 2 * m) * Co + n;
      bf16* uo = ue + Co;
#pragma unroll
      for (int j = 0; j < 32; j += 8) {
        uint4 we, wo;
        uint32_t* pe = &we.x;
        uint32_t* po = &wo.x;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int q = j + 2 * h;
          const float e0 = __uint_as_float(ev[q]) + bias[n + q], e1 = __uint_as_float(ev[q + 1]) + bias[n + q + 1];
          const float d0 = __uint_as_float(od[q]) + bias[n + q], d1 = __uint_as_float(od[q + 1]) + bias[n + q + 1];
          *reinterpret_cast<float2*>(v + o + (size_t)q * To) = make_float2(e0, d0);
          *reinterpret_cast<float2*>(v + o + (size_t)(q + 1) * To) = make_float2(e1, d1);
          const __nv_bfloat162 ue2 = __floats2bfloat162_rn(gelu_f(e0), gelu_f(e1));
          const __nv_bfloat162 uo2 = __floats2bfloat162_rn(gelu_f(d0), gelu_f(d1));
          pe[h] = *reinterpret_cast<const uint32_t*>(&ue2);
          po[h] = *reinterpret_cast<const uint32_t*>(&uo2);
        }
        *reinterpret_cast<uint4*>(ue + j) = we;
        *reinterpret_cast<uint4*>(uo + j) = wo;
      }
      return;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float bj = bias[n + j];
      const float e = __uint_as_float(ev[j]) + bj, d = __uint_as_float(od[j]) + bj;
      *reinterpret_cast<float2*>(v + o + (size_t)j * To) = make_float2(e, d);
      if (un) *reinterpret_cast<__nv_bfloat162*>(un + o + (size_t)j * To) = __floats2bfloat162_rn(gelu_f(e), gelu_f(d));
    }
  }
};

// v[b][co][2m + par] = acc + bias[co]; u_next = bf16(gelu(v)), channel-major
// or (tm) time-major [b][t][co]
struct ConvEpi {
  float* v; bf16* un; const float* bias; int T, Co, par, tm;
  __device__ __forceinline__ void operator()(int r, int n, const uint32_t* acc) const {
    const int b = r / T, m = r % T, To = 2 * T;
    const size_t o = ((size_t)b * Co + n) * To + 2 * m + par;
    bf16* ut = un + ((size_t)b * To + 2 * m + par) * Co + n;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float val = __uint_as_float(acc[j]) + bias[n + j];
      v[o + (size_t)j * To] = val;
      if (un) {
        if (tm) ut[j] = __float2bfloat16(gelu_f(val));
        else un[o + (size_t)j * To] = __float2bfloat16(gelu_f(val));
      }
    }
  }
};

// 3-D tensor map of a BF16 [B][T][C] array for 128-row tiles of (b, t) pairs
int tmap_btc(CUtensorMap* map, const bf16* base, int B, int T, int C) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return sfail(DGSEM_ECUDA, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  if (!((T >= tcg::BM && T % tcg::BM == 0) || (T < tcg::BM && tcg::BM % T == 0)))
    return sfail(DGSEM_EINVAL, "time length %d neither divides nor is a multiple of 128", T);
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)T, (cuuint64_t)B};
  const cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)T * C * 2};
  const cuuint32_t box[3] = {(cuuint32_t)tcg::BK, (cuuint32_t)std::min(T, tcg::BM),
                             (cuuint32_t)std::max(1, tcg::BM / T)};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return sfail(DGSEM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGSEM_OK;
}

// one parity of a transposed convolution: u_tm [B][T][Ci] (time-major), taps
// Bw [Co][2 Ci]; rows (b, m) of C go to v / u_next at time 2m + par
template <int STAGES>
int convt_parity_launch(const CUtensorMap& ta, const CUtensorMap& tb, int B, int T, int Ci, int Co, int par,
                        const ConvEpi& ep, int* err, cudaStream_t s) {
  auto kern = tcg::gemm_kernel<64, STAGES, ConvEpi, tcg::ShiftA>;
  constexpr int smem = tcg::Geo<64, STAGES>::SMEM;
  S_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int M = B * T;
  dim3 grid(Co / 64, M / tcg::BM);
  const tcg::ShiftA al{Ci / tcg::BK, T, par == 0 ? 0 : 1, par == 0 ? -1 : 0};
  kern<<<grid, tcg::THREADS, smem, s>>>(ta, tb, M, 2 * Ci, ep, err, al);
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

int convt_parity(const bf16* u_tm, int B, int T, int Ci, const bf16* Bw, int Co, int par, const float* bias, float* v,
                 bf16* un, int tm, int* err, cudaStream_t s) {
  if (Ci % tcg::BK || Co % 64) return sfail(DGSEM_EINVAL, "convolution channels %d -> %d not tileable", Ci, Co);
  CUtensorMap ta, tb;
  int rc;
  if ((rc = tmap_btc(&ta, u_tm, B, T, Ci)) || (rc = tmap_bf16(&tb, Bw, Co, 2 * Ci, 2 * Ci, 64))) return rc;
  const ConvEpi ep{v, un, bias, T, Co, par, tm};
  // a short K (few k-tiles) takes a shallow ring, so that several CTAs share an
  // SM and one's epilogue overlaps another's products
  if (2 * Ci / tcg::BK <= 6) return convt_parity_launch<3>(ta, tb, B, T, Ci, Co, par, ep, err, s);
  return convt_parity_launch<6>(ta, tb, B, T, Ci, Co, par, ep, err, s);
}

// ---------------------------------------------------------------------------
// Gradients of a transposed convolution on the tensor cores (dv = dL/dv in
// FP32 [B][Co][To], To = 2 Ti; the products read it rounded to BF16):
//   du[b][ci][i] = sum_co sum_k W[ci][co][k] dv[b][co][2i - 1 + k]:
//     one product over rows (b, i), K = 4 Co in four segments (k = 0..3)
//     read from the parity-split, time-major dvp[par][b][m][co] at time
//     m = i - 1, i, i, i + 1 of parity 1, 0, 1, 0;  B = Bd[ci][k Co + co];
//   dW[ci][co][k] = sum_{b,i} u[b][ci][i] dv[b][co][2i - 1 + k]:
//     four products (one per k) over K = (b, i) with K-contiguous copies
//     uK[ci][b Ti + i] and dvK[k][co][b Ti + i], split over S parts of K
//     whose partial sums a fixed-order reduction adds;
//   db[co] = sum_{b,t} dv[b][co][t] in FP32 (no rounding).
// ---------------------------------------------------------------------------
// dvp[par][b][m][co] = bf16(dv[b][co][2m + par])
__global__ void convt_dv_split(const float* __restrict__ dv, int B, int Co, int Ti, bf16* __restrict__ dvp) {
  __shared__ float t[32][65];
  const int To = 2 * Ti;
  const int b = blockIdx.z, co0 = blockIdx.y * 32, t0 = blockIdx.x * 64;
  for (int r = threadIdx.y; r < 32; r += 8)
    for (int c = threadIdx.x; c < 64; c += 32) {
      const int co = co0 + r, tt = t0 + c;
      t[r][c] = (co < Co && tt < To) ? dv[((size_t)b * Co + co) * To + tt] : 0.f;
    }
  __syncthreads();
  const size_t plane = (size_t)B * Ti * Co;
  for (int c = threadIdx.y; c < 64; c += 8) {
    const int tt = t0 + c, co = co0 + threadIdx.x;
    if (tt < To && co < Co) dvp[(size_t)(tt & 1) * plane + ((size_t)b * Ti + (tt >> 1)) * Co + co] = __float2bfloat16(t[threadIdx.x][c]);
  }
}

// Bd[ci][k Co + co] = W[ci][co][k]
__global__ void convt_taps_data(const bf16* __restrict__ W, int Ci, int Co, bf16* __restrict__ Bd) {
  const size_t n = (size_t)Ci * Co * 4;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % 4), co = (int)((idx / 4) % Co), ci = (int)(idx / ((size_t)4 * Co));
    Bd[((size_t)ci * 4 + k) * Co + co] = W[idx];
  }
}

// uK[ci][b Ti + i] = u[b][ci][i]
__global__ void convt_u_kmajor(const bf16* __restrict__ u, int B, int Ci, int Ti, bf16* __restrict__ uK) {
  const size_t n = (size_t)B * Ci * Ti;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % Ti), ci = (int)((idx / Ti) % Ci), b = (int)(idx / ((size_t)Ti * Ci));
    uK[((size_t)ci * B + b) * Ti + i] = u[idx];
  }
}

// dvK[k][co][b Ti + i] = bf16(dv[b][co][2i - 1 + k]), zero where the time is outside [0, To)
__global__ void convt_dv_taps(const float* __restrict__ dv, int B, int Co, int Ti, bf16* __restrict__ dvK) {
  const int To = 2 * Ti;
  const size_t n = (size_t)B * Co * Ti;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % Ti), co = (int)((idx / Ti) % Co), b = (int)(idx / ((size_t)Ti * Co));
    const float* row = dv + ((size_t)b * Co + co) * To;
    const size_t o = ((size_t)co * B + b) * Ti + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int t = 2 * i - 1 + k;
      dvK[(size_t)k * Co * B * Ti + o] = __float2bfloat16((t >= 0 && t < To) ? row[t] : 0.f);
    }
  }
}

// dW[ci][co][k] = sum_z part[k][z][ci][co] (fixed order)
__global__ void convt_dw_reduce(const float* __restrict__ part, int S, int Ci, int Co, float* __restrict__ dW) {
  const size_t n = (size_t)Ci * Co * 4;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % 4), co = (int)((idx / 4) % Co), ci = (int)(idx / ((size_t)4 * Co));
    const float* p = part + (size_t)k * S * Ci * Co + (size_t)ci * Co + co;
    float acc = 0.f;
    for (int z = 0; z < S; ++z) acc += p[(size_t)z * Ci * Co];
    dW[idx] = acc;
  }
}

// db[co] = sum_{b,t} dv[b][co][t] in a fixed order: block (co, c) sums the
// rows of batch members c*BIAS_BPB .. (c+1)*BIAS_BPB - 1 into part[co][c]
// (tree over its threads), then convt_bias_sum adds the parts in order
constexpr int BIAS_BPB = 4;
__global__ void __launch_bounds__(256) convt_bias_part(const float* __restrict__ dv, int B, int Co, int To,
                                                       float* __restrict__ part) {
  __shared__ float red[256];
  const int co = blockIdx.x, c = blockIdx.y, nch = gridDim.y;
  float acc = 0.f;
  for (int b = c * BIAS_BPB; b < min(B, (c + 1) * BIAS_BPB); ++b) {
    const float* row = dv + ((size_t)b * Co + co) * To;
    for (int t = threadIdx.x; t < To; t += 256) acc += row[t];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)co * nch + c] = red[0];
}

__global__ void convt_bias_sum(const float* __restrict__ part, int Co, int nch, float* __restrict__ db) {
  const int co = blockIdx.x * blockDim.x + threadIdx.x;
  if (co >= Co) return;
  float acc = 0.f;
  for (int c = 0; c < nch; ++c) acc += part[(size_t)co * nch + c];
  db[co] = acc;
}

// round FP32 values to BF16 precision in place (the CUDA-core gradient path
// reads dv at the precision the tensor-core path reads it)
__global__ void round_bf16_inplace(float* __restrict__ x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] = __bfloat162float(__float2bfloat16(x[i]));
}

// du rows (b, i), 32 consecutive ci: gu[b][ci][i] (channel-major FP32)
struct DuEpi {
  float* du; int T, Ci;
  __device__ __forceinline__ void operator()(int r, int n, const uint32_t* acc) const {
    const int b = r / T, i = r % T;
    const size_t o = ((size_t)b * Ci + n) * T + i;
#pragma unroll
    for (int j = 0; j < 32; ++j) du[o + (size_t)j * T] = __uint_as_float(acc[j]);
  }
};

// partial dW_k rows ci, 32 consecutive co: part[z][ci][co] for K part z = blockIdx.z
struct PartEpi {
  float* part; int Ci, Co;
  __device__ __forceinline__ void operator()(int r, int n, const uint32_t* acc) const {
    float4* dst = reinterpret_cast<float4*>(part + ((size_t)blockIdx.z * Ci + r) * Co + n);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      dst[q] = make_float4(__uint_as_float(acc[4 * q]), __uint_as_float(acc[4 * q + 1]), __uint_as_float(acc[4 * q + 2]),
                           __uint_as_float(acc[4 * q + 3]));
  }
};

// 4-D tensor map of a BF16 [P][B][T][C] array for 128-row tiles of (b, t) pairs
int tmap_pbtc(CUtensorMap* map, const bf16* base, int P, int B, int T, int C) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return sfail(DGSEM_ECUDA, "cuTensorMapEncodeTiled is not available");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  if (!((T >= tcg::BM && T % tcg::BM == 0) || (T < tcg::BM && tcg::BM % T == 0)))
    return sfail(DGSEM_EINVAL, "time length %d neither divides nor is a multiple of 128", T);
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)T, (cuuint64_t)B, (cuuint64_t)P};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)T * C * 2, (cuuint64_t)B * T * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)tcg::BK, (cuuint32_t)std::min(T, tcg::BM),
                             (cuuint32_t)std::max(1, tcg::BM / T), 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return sfail(DGSEM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DGSEM_OK;
}

// K parts of the weight-gradient products: the largest divisor of the k-tile
// count that keeps the grid within about one wave
int dw_parts(int tiles, int ktiles) {
  int best = 1;
  for (int s = 1; s <= ktiles && s <= 64; ++s)
    if (ktiles % s == 0 && tiles * s <= 160) best = s;
  return best;
}

// a transposed convolution, both parities in one product (see convt_taps3):
// u_tm [B][T][Ci] time-major, B3 [2 Co][3 Ci]; v and u_next channel-major
template <int BN, int STAGES>
int convt_pair_launch(const bf16* u_tm, int B, int T, int Ci, const bf16* B3, int Co, const float* bias, float* v,
                      bf16* un, int tm, int* err, cudaStream_t s) {
  CUtensorMap ta, tb;
  int rc;
  if ((rc = tmap_pbtc(&ta, u_tm, 1, B, T, Ci)) || (rc = tmap_bf16(&tb, B3, 2 * Co, 3 * Ci, 3 * Ci, BN))) return rc;
  auto kern = tcg::gemm_kernel<BN, STAGES, PairConvEpi, tcg::SegA>;
  constexpr int smem = tcg::Geo<BN, STAGES>::SMEM;
  S_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int M = B * T;
  const tcg::SegA al{Ci / tcg::BK, T, {-1, 0, 1, 0}, {0, 0, 0, 0}};
  kern<<<dim3(1, M / tcg::BM, 1), tcg::THREADS, smem, s>>>(ta, tb, M, 3 * Ci, PairConvEpi{v, un, bias, T, Co, tm}, err,
                                                          al);
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

int convt_pair(const bf16* u_tm, int B, int T, int Ci, const bf16* B3, int Co, const float* bias, float* v, bf16* un,
               int tm, int* err, cudaStream_t s) {
  if (Ci % tcg::BK) return sfail(DGSEM_EINVAL, "convolution input channels %d not tileable", Ci);
  // a short K (few k-tiles) takes a shallow ring (96 KB of shared memory), so
  // that two CTAs share an SM and one's epilogue overlaps the other's products
  const bool shallow = 3 * Ci / tcg::BK <= 6;
  if (Co == 64)
    return shallow ? convt_pair_launch<128, 3>(u_tm, B, T, Ci, B3, Co, bias, v, un, tm, err, s)
                   : convt_pair_launch<128, 6>(u_tm, B, T, Ci, B3, Co, bias, v, un, tm, err, s);
  if (Co == 128)
    return shallow ? convt_pair_launch<256, 2>(u_tm, B, T, Ci, B3, Co, bias, v, un, tm, err, s)
                   : convt_pair_launch<256, 4>(u_tm, B, T, Ci, B3, Co, bias, v, un, tm, err, s);
  return sfail(DGSEM_EINVAL, "paired convolution product needs 64 or 128 output channels, not %d", Co);
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
  // BF16 transposes feeding the backward products (K-contiguous operands)
  bf16 *tA = nullptr, *tB = nullptr, *tW = nullptr;
  // tensor-core transposed convolutions: time-major input copy and tap pairs;
  // layers whose channel counts are not multiples of 64 run on the CUDA cores
  bf16 *utm = nullptr, *Bev = nullptr;
  std::vector<int> conv_tc;
  // tm_u[j]: u[j] is stored time-major [b][t][ci] (written so by the epilogue of
  // tensor-core layer j - 1 and read so by tensor-core layer j, no transpose)
  std::vector<int> tm_u;
  // forward tap matrices of each tensor-core layer, rebuilt only when the
  // BF16 weights have changed since (pb_ver counts their updates)
  std::vector<bf16*> b3;
  std::vector<unsigned long long> b3_ver;
  unsigned long long pb_ver = 1;
  // their gradients: parity-split dv, K-contiguous u and tap-shifted dv, and
  // the partial sums of the split weight-gradient products
  bf16 *dvp = nullptr, *uK = nullptr, *dvK = nullptr;
  float* part = nullptr;
  size_t part_n = 0;
  float* bias_part = nullptr;         // [Co][batch / 4] partial sums of the bias gradients
  int* d_err = nullptr;               // set by a tensor-core product whose bounded wait gave up
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

// forward pass keeping every activation; the last layer's output goes to
// yout when given (inference), else to v[n_conv - 1]
int forward_impl(srg_net* n, const float* x, int B, cudaStream_t s, float* yout = nullptr) {
  const srg_config& c = n->cfg;
  to_bf16<<<EW_BLOCKS, EW_THREADS, 0, s>>>(x, n->a[0], (size_t)B * c.d_in);
  S_TRY(cudaGetLastError());
  int fan = c.d_in;
  for (int l = 0; l < c.n_hidden; ++l) {
    Epi ep{n->P + n->offB[l], n->z[l], c.hidden, n->a[l + 1], c.hidden, 1};
    int rc = gemm_nt(n->a[l], fan, n->Pb + n->offW[l], fan, B, c.hidden, fan, ep, n->d_err, s);
    if (rc) return rc;
    fan = c.hidden;
  }
  const int L = c.n_hidden;
  const int nd = c.c0 * c.t0;
  Epi ep{n->P + n->offB[L], n->zd, nd, n->u[0], nd, 0};
  int rc = gemm_nt(n->a[L], fan, n->Pb + n->offW[L], fan, B, nd, fan, ep, n->d_err, s);
  if (rc) return rc;
  for (int j = 0; j < c.n_conv; ++j) {
    const int last = j == c.n_conv - 1;
    const int ci = conv_cin(c, j), co = c.conv_ch[j], ti = conv_len(c, j);
    float* vj = (last && yout) ? yout : n->v[j];
    bf16* un = last ? nullptr : n->u[j + 1];
    const int tm_next = last ? 0 : n->tm_u[j + 1];
    if (n->conv_tc[j]) {
      // the input in time-major layout (a transposed copy unless the previous
      // layer wrote it so), the tap matrix (cached per weight update), then
      // both parities in one product (64 or 128 output channels) or one
      // product per parity
      const bf16* uin = n->u[j];
      if (!n->tm_u[j]) {
        if ((rc = transpose(n->u[j], ci, ti, n->utm, s, B))) return rc;
        uin = n->utm;
      }
      const bool paired = co == 64 || co == 128;
      if (n->b3_ver[j] != n->pb_ver) {
        if (paired) {
          convt_taps3<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->Pb + n->offW[L + 1 + j], ci, co, n->b3[j]);
        } else {
          convt_taps<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->Pb + n->offW[L + 1 + j], ci, co, n->b3[j],
                                                      n->b3[j] + (size_t)co * 2 * ci);
        }
        S_TRY(cudaGetLastError());
        n->b3_ver[j] = n->pb_ver;
      }
      if (paired) {
        if ((rc = convt_pair(uin, B, ti, ci, n->b3[j], co, n->P + n->offB[L + 1 + j], vj, un, tm_next, n->d_err, s)))
          return rc;
      } else {
        for (int par = 0; par < 2; ++par)
          if ((rc = convt_parity(uin, B, ti, ci, n->b3[j] + (size_t)par * co * 2 * ci, co, par,
                                 n->P + n->offB[L + 1 + j], vj, un, tm_next, n->d_err, s)))
            return rc;
      }
    } else {
      convt_fwd<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->u[j], n->Pb + n->offW[L + 1 + j], n->P + n->offB[L + 1 + j], B,
                                                 ci, co, ti, vj, un, 1);
      S_TRY(cudaGetLastError());
    }
  }
  return DGSEM_OK;
}

// data and weight gradients of transposed convolution j on the tensor cores
// (dv in n->gv; du into n->gu, dW into the gradient vector)
int convt_backward_tc(srg_net* n, int j, int B, cudaStream_t s) {
  const srg_config& c = n->cfg;
  const int L = c.n_hidden;
  const int ci = conv_cin(c, j), co = c.conv_ch[j], ti = conv_len(c, j), to = 2 * ti;
  int rc;
  // du: rows (b, i), N = Ci, K = 4 Co from the parity-split time-major dv
  convt_dv_split<<<dim3((to + 63) / 64, (co + 31) / 32, B), dim3(32, 8), 0, s>>>(n->gv, B, co, ti, n->dvp);
  convt_taps_data<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->Pb + n->offW[L + 1 + j], ci, co, n->Bev);
  S_TRY(cudaGetLastError());
  {
    CUtensorMap ta, tb;
    if ((rc = tmap_pbtc(&ta, n->dvp, 2, B, ti, co)) || (rc = tmap_bf16(&tb, n->Bev, ci, 4 * co, 4 * co, 64))) return rc;
    const int M = B * ti;
    const tcg::SegA al{co / tcg::BK, ti, {-1, 0, 0, 1}, {1, 0, 1, 0}};
    const dim3 grid(ci / 64, M / tcg::BM, 1);
    const DuEpi ep{n->gu, ti, ci};
    // a short K takes a shallow ring (several CTAs per SM)
    if (4 * co / tcg::BK <= 6) {
      auto kern = tcg::gemm_kernel<64, 3, DuEpi, tcg::SegA>;
      constexpr int smem = tcg::Geo<64, 3>::SMEM;
      S_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      kern<<<grid, tcg::THREADS, smem, s>>>(ta, tb, M, 4 * co, ep, n->d_err, al);
    } else {
      auto kern = tcg::gemm_kernel<64, 6, DuEpi, tcg::SegA>;
      constexpr int smem = tcg::Geo<64, 6>::SMEM;
      S_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      kern<<<grid, tcg::THREADS, smem, s>>>(ta, tb, M, 4 * co, ep, n->d_err, al);
    }
    S_TRY(cudaGetLastError());
  }
  // dW_k: rows ci, N = Co, K = (b, i), split into S parts
  if (n->tm_u[j]) {
    // time-major u[j] is [(b, i)][ci]: its transpose is the K-contiguous copy
    if ((rc = transpose(n->u[j], B * ti, ci, n->uK, s))) return rc;
  } else {
    convt_u_kmajor<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->u[j], B, ci, ti, n->uK);
  }
  convt_dv_taps<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->gv, B, co, ti, n->dvK);
  S_TRY(cudaGetLastError());
  const int K = B * ti;
  const int mt = (ci + tcg::BM - 1) / tcg::BM;
  const int S = dw_parts(mt * (co / 64), K / tcg::BK);
  if ((size_t)4 * S * ci * co > n->part_n) return sfail(DGSEM_EINVAL, "weight-gradient partial buffer too small");
  for (int k = 0; k < 4; ++k) {
    CUtensorMap ta, tb;
    const bf16* dk = n->dvK + (size_t)k * co * K;
    if ((rc = tmap_bf16(&ta, n->uK, ci, K, K, tcg::BM)) || (rc = tmap_bf16(&tb, dk, co, K, K, 64))) return rc;
    auto kern = tcg::gemm_kernel<64, 6, PartEpi, tcg::DenseA>;
    constexpr int smem = tcg::Geo<64, 6>::SMEM;
    S_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    kern<<<dim3(co / 64, mt, S), tcg::THREADS, smem, s>>>(ta, tb, ci, K, PartEpi{n->part + (size_t)k * S * ci * co, ci, co},
                                                         n->d_err, tcg::DenseA());
    S_TRY(cudaGetLastError());
  }
  convt_dw_reduce<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->part, S, ci, co, n->G + n->offW[L + 1 + j]);
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

// a bounded wait of a tensor-core product gave up (the flag is cleared)
int check_err(srg_net* n) {
  int err = 0;
  S_TRY(cudaMemcpy(&err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    S_TRY(cudaMemset(n->d_err, 0, sizeof(int)));
    return sfail(DGSEM_ETIMEOUT, "a bounded wait of a tensor-core product gave up");
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
      (rc = A((void**)&n->gzb, B * std::max(maxw, nd) * 2)) ||
      (rc = A((void**)&n->tA, B * std::max((size_t)c.hidden, nd) * 2)) || (rc = A((void**)&n->tB, B * maxw * 2)) ||
      (rc = A((void**)&n->tW, std::max(nd * c.hidden, (size_t)c.hidden * maxw) * 2)) ||
      (rc = A((void**)&n->d_err, sizeof(int)))) {
    srg_destroy(n);
    return rc;
  }
  S_TRY(cudaMemset(n->d_err, 0, sizeof(int)));
  // which transposed convolutions take the tensor-core path (channel counts
  // multiples of 64; time lengths that tile 128 rows), and their scratch
  size_t utm_n = 0, bev_n = 0, dvp_n = 0, uk_n = 0, dvk_n = 0;
  n->conv_tc.assign(c.n_conv, 0);
  for (int j = 0; j < c.n_conv; ++j) {
    const int ci = conv_cin(c, j), co = c.conv_ch[j], ti = conv_len(c, j);
    const bool tiles_t = (ti >= 128 && ti % 128 == 0) || (ti < 128 && 128 % ti == 0);
    if (ci % 64 == 0 && co % 64 == 0 && tiles_t && ((size_t)max_batch * ti) % 128 == 0) {
      n->conv_tc[j] = 1;
      utm_n = std::max(utm_n, B * ci * ti);
      bev_n = std::max(bev_n, (size_t)4 * ci * co);   // the data-gradient taps
      dvp_n = std::max(dvp_n, B * 2 * ti * co);
      uk_n = std::max(uk_n, B * ci * ti);
      dvk_n = std::max(dvk_n, (size_t)4 * co * B * ti);
      // the weight-gradient parts for the smallest batch (64) the network takes, the most parts
      n->part_n = std::max(n->part_n, (size_t)4 * 64 * ci * co);
    }
  }
  n->tm_u.assign(c.n_conv, 0);
  n->b3.assign(c.n_conv, nullptr);
  n->b3_ver.assign(c.n_conv, 0);
  for (int j = 0; j < c.n_conv; ++j) {
    if (!n->conv_tc[j]) continue;
    n->tm_u[j] = j > 0 && n->conv_tc[j - 1];
    const int ci = conv_cin(c, j), co = c.conv_ch[j];
    const size_t nb3 = (size_t)((co == 64 || co == 128) ? 6 : 4) * ci * co;
    if ((rc = A((void**)&n->b3[j], nb3 * 2))) { srg_destroy(n); return rc; }
  }
  if (utm_n && ((rc = A((void**)&n->utm, utm_n * 2)) || (rc = A((void**)&n->Bev, bev_n * 2)) ||
                (rc = A((void**)&n->dvp, dvp_n * 2)) || (rc = A((void**)&n->uK, uk_n * 2)) ||
                (rc = A((void**)&n->dvK, dvk_n * 2)) || (rc = A((void**)&n->part, n->part_n * 4)))) {
    srg_destroy(n);
    return rc;
  }
  {
    int maxco = 0;
    for (int j = 0; j < c.n_conv; ++j) maxco = std::max(maxco, c.conv_ch[j]);
    if ((rc = A((void**)&n->bias_part, (size_t)maxco * ((max_batch + BIAS_BPB - 1) / BIAS_BPB) * 4))) {
      srg_destroy(n);
      return rc;
    }
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
  ++n->pb_ver;
  S_TRY(cudaGetLastError());
  S_TRY(cudaDeviceSynchronize());
  return DGSEM_OK;
}

int srg_forward(srg_net* n, const float* x, int B, float* y, void* stream) {
  if (!n || !x || !y) return sfail(DGSEM_EINVAL, "NULL argument");
  int rc = check_batch(n, B);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the last layer writes straight into y (its epilogue stores pairs of floats);
  // a y that is not 16-byte aligned gets the network's own buffer and a copy
  const bool direct = reinterpret_cast<uintptr_t>(y) % 16 == 0;
  if ((rc = forward_impl(n, x, B, s, direct ? y : nullptr))) return rc;
  if (!direct) {
    const srg_config& c = n->cfg;
    const size_t outn = (size_t)B * c.conv_ch[c.n_conv - 1] * conv_len(c, c.n_conv);
    S_TRY(cudaMemcpyAsync(y, n->v[c.n_conv - 1], outn * 4, cudaMemcpyDeviceToDevice, s));
  }
  S_TRY(cudaStreamSynchronize(s));
  return check_err(n);
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
    // the bias gradient from dv itself; the products read dv rounded to BF16
    {
      const int nch = (B + BIAS_BPB - 1) / BIAS_BPB;
      convt_bias_part<<<dim3(co, nch), 256, 0, s>>>(n->gv, B, co, 2 * ti, n->bias_part);
      convt_bias_sum<<<(co + 127) / 128, 128, 0, s>>>(n->bias_part, co, nch, n->G + n->offB[L + 1 + j]);
    }
    S_TRY(cudaGetLastError());
    if (n->conv_tc[j]) {
      if ((rc = convt_backward_tc(n, j, B, s))) return rc;
    } else {
      round_bf16_inplace<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->gv, (size_t)B * co * 2 * ti);
      convt_bwd_weight<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->u[j], n->gv, B, ci, co, ti, n->G + n->offW[L + 1 + j]);
      convt_bwd_data<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->gv, n->Pb + n->offW[L + 1 + j], B, ci, co, ti, n->gu);
    }
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
  // dW_dec [nd][hidden] = dZ^T a_L: operands dZ^T [nd][B] and a_L^T [hidden][B]
  Epi ew{nullptr, n->G + n->offW[L], c.hidden, nullptr, 0, 0};
  if ((rc = transpose(n->gzb, B, nd, n->tA, s)) || (rc = transpose(n->a[L], B, c.hidden, n->tB, s)) ||
      (rc = gemm_nt(n->tA, B, n->tB, B, nd, c.hidden, B, ew, n->d_err, s)))
    return rc;
  // da_L [B][hidden] = dZ W_dec: operands dZ [B][nd] and W_dec^T [hidden][nd]
  Epi ea{nullptr, n->ga, c.hidden, nullptr, 0, 0};
  if ((rc = transpose(n->Pb + n->offW[L], nd, c.hidden, n->tW, s)) ||
      (rc = gemm_nt(n->gzb, nd, n->tW, nd, B, c.hidden, nd, ea, n->d_err, s)))
    return rc;
  // hidden layers, last to first
  for (int l = L - 1; l >= 0; --l) {
    const int fan = l == 0 ? c.d_in : c.hidden;
    gelu_bwd<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->ga, n->z[l], n->gz, n->gzb, (size_t)B * c.hidden);
    col_sum<<<(c.hidden + 127) / 128, 128, 0, s>>>(n->gz, B, c.hidden, n->G + n->offB[l]);
    S_TRY(cudaGetLastError());
    // dW_l [hidden][fan] = dZ^T a_l: operands dZ^T [hidden][B] and a_l^T [fan][B]
    Epi eW{nullptr, n->G + n->offW[l], fan, nullptr, 0, 0};
    if ((rc = transpose(n->gzb, B, c.hidden, n->tA, s)) || (rc = transpose(n->a[l], B, fan, n->tB, s)) ||
        (rc = gemm_nt(n->tA, B, n->tB, B, c.hidden, fan, B, eW, n->d_err, s)))
      return rc;
    if (l > 0) {
      // da_l [B][fan] = dZ W_l: operands dZ [B][hidden] and W_l^T [fan][hidden]
      Epi eA{nullptr, n->ga, c.hidden, nullptr, 0, 0};
      if ((rc = transpose(n->Pb + n->offW[l], c.hidden, fan, n->tW, s)) ||
          (rc = gemm_nt(n->gzb, c.hidden, n->tW, c.hidden, B, fan, c.hidden, eA, n->d_err, s)))
        return rc;
    }
  }
  double l_host = 0.0;
  S_TRY(cudaMemcpyAsync(&l_host, n->d_loss, 8, cudaMemcpyDeviceToHost, s));
  S_TRY(cudaStreamSynchronize(s));
  if (loss) *loss = l_host;
  return check_err(n);
}

int srg_adam_step(srg_net* n, float lr, float b1, float b2, float eps, void* stream) {
  if (!n) return sfail(DGSEM_EINVAL, "NULL argument");
  n->t += 1;
  const float c1 = 1.f - std::pow(b1, (float)n->t), c2 = 1.f - std::pow(b2, (float)n->t);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  adam<<<EW_BLOCKS, EW_THREADS, 0, s>>>(n->P, n->Pb, n->G, n->M1, n->M2, n->np, lr, b1, b2, eps, c1, c2);
  ++n->pb_ver;
  S_TRY(cudaGetLastError());
  return DGSEM_OK;
}

int srg_train_step(srg_net* n, const float* x, const float* target, int B, float lr, double* loss, void* stream) {
  int rc = srg_backward(n, x, target, B, loss, stream);
  if (rc) return rc;
  return srg_adam_step(n, lr, 0.9f, 0.999f, 1e-8f, stream);
}

int srg_gemm_bench(int M, int N, int K, int reps, double* tflops, void* stream) {
  if (!tflops || reps < 1 || M < 1 || N < 64 || K < 64) return sfail(DGSEM_EINVAL, "bad arguments");
  *tflops = 0.0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bf16 *A = nullptr, *B = nullptr;
  float* C = nullptr;
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DGSEM_OK;
  auto cleanup = [&]() {
    cudaFree(A); cudaFree(B); cudaFree(C); cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&A, (size_t)M * K * 2) != cudaSuccess || cudaMalloc(&B, (size_t)N * K * 2) != cudaSuccess ||
      cudaMalloc(&C, (size_t)M * N * 4) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return sfail(DGSEM_ENOMEM, "gemm bench buffers");
  }
  do {
    if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess || cudaMemset(A, 0x3c, (size_t)M * K * 2) != cudaSuccess ||
        cudaMemset(B, 0x3c, (size_t)N * K * 2) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
      rc = sfail(DGSEM_ECUDA, "gemm bench set-up");
      break;
    }
    Epi ep{nullptr, C, N, nullptr, 0, 0};
    if ((rc = gemm_nt(A, K, B, K, M, N, K, ep, err, s))) break;     // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && !rc; ++r) rc = gemm_nt(A, K, B, K, M, N, K, ep, err, s);
    cudaEventRecord(e1, s);
    if (rc) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = sfail(DGSEM_ECUDA, "gemm bench launch"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int h_err = 0;
    cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (h_err) { rc = sfail(DGSEM_ETIMEOUT, "a bounded wait of the tensor-core product gave up"); break; }
    *tflops = 2.0 * M * N * (double)K * reps / (ms * 1e-3) / 1e12;
  } while (false);
  cleanup();
  return rc;
}

void srg_destroy(srg_net* n) {
  if (!n) return;
  for (void* p : n->allocs) cudaFree(p);
  delete n;
}

}  // extern "C"
