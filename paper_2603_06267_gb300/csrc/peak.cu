// Arithmetic-rate probe (no counterpart in the paper): every SM runs long
// chains of independent fused multiply-adds, timed with CUDA events on the
// caller's stream; the rate is the denominator of the arithmetic rooflines of
// the FP64 path (plain DFMA) and of the FP32 path (packed f32x2 FMA, the form
// the FP32 kernels issue).  Nothing here changes a clock or any other setting
// of the GPU: the rate is the one the GPU sustains at its clocks of the moment.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>

#include "../../include/dgsem.h"

int dg_fail_msg(int code, const char* msg);   // api.cu: sets the thread's last-error message

namespace {

constexpr int PK_CHAINS = 8;      // independent chains per thread (hide the FMA latency)
constexpr int PK_UNROLL = 16;     // FMAs per chain per loop iteration
constexpr int PK_THREADS = 256;
constexpr int PK_BLOCKS_PER_SM = 8;

__global__ void __launch_bounds__(PK_THREADS) fma_probe_f64(double* out, int iters, double b, double c) {
  double a[PK_CHAINS];
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = 1e-3 * (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PK_UNROLL; ++k)
#pragma unroll
      for (int i = 0; i < PK_CHAINS; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) s += a[i];
  // the chains converge to c / (1 - b) and stay finite; the store keeps them live
  if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) fma_probe_f32x2(float* out, int iters, float b, float c) {
  float2 a[PK_CHAINS];
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) a[i] = make_float2(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)i);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PK_UNROLL; ++k)
#pragma unroll
      for (int i = 0; i < PK_CHAINS; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < PK_CHAINS; ++i) s += a[i].x + a[i].y;
  if (s == -1.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int dgsem_measure_peak(int precision, double* tflops, void* stream) {
  if (!tflops) return dg_fail_msg(DGSEM_EINVAL, "tflops is NULL");
  if (precision != DGSEM_FP64 && precision != DGSEM_FP32_MIXED) return dg_fail_msg(DGSEM_EINVAL, "unknown precision");
  *tflops = 0.0;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return dg_fail_msg(DGSEM_ECUDA, "no current CUDA device");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = nsm * PK_BLOCKS_PER_SM;
  const bool f64 = precision == DGSEM_FP64;
  void* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * PK_THREADS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return dg_fail_msg(DGSEM_ENOMEM, "probe output buffer");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = DGSEM_OK;
  std::string msg;
  auto launch = [&](int iters) {
    if (f64) fma_probe_f64<<<blocks, PK_THREADS, 0, s>>>(static_cast<double*>(out), iters, 0.999999, 1e-6);
    else fma_probe_f32x2<<<blocks, PK_THREADS, 0, s>>>(static_cast<float*>(out), iters, 0.999f, 1e-3f);
    return cudaGetLastError();
  };
  auto timed = [&](int iters, float* ms) {
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch(iters);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e;
  };
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      rc = DGSEM_ECUDA; msg = "event creation"; break;
    }
    // size the launch to about 0.2 s, then keep the best of three launches
    int iters = 64;
    float ms = 0.f;
    cudaError_t e = launch(iters);          // warm-up (module load, clocks up)
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int k = 0; k < 12 && e == cudaSuccess; ++k) {
      e = timed(iters, &ms);
      if (e != cudaSuccess || ms > 20.f) break;
      iters *= 4;
    }
    if (e != cudaSuccess) { rc = DGSEM_ECUDA; msg = cudaGetErrorString(e); break; }
    iters = std::max(1, (int)std::min(2.0e9, iters * (200.0 / std::max(ms, 1e-3f))));
    double best = 0.0;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
      e = timed(iters, &ms);
      const double fma_per_thread = (double)iters * PK_UNROLL * PK_CHAINS * (f64 ? 1 : 2);
      const double flops = 2.0 * fma_per_thread * blocks * PK_THREADS;
      if (e == cudaSuccess && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    if (e != cudaSuccess) { rc = DGSEM_ECUDA; msg = cudaGetErrorString(e); break; }
    *tflops = best;
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc) return dg_fail_msg(rc, msg.c_str());
  return DGSEM_OK;
}
