/*
 * surrogate.h -- C ABI of the learned surrogate of the DG-SEM + PMUT solver.
 *
 * The paper has no counterpart: this network is a project extension that maps
 * an array drive pattern (per-PMUT delay and amplitude) to receiver pressure
 * traces for fast beam-pattern screening, trained on traces produced by
 * dgsem_run.  Architecture:
 *     x [d_in] -> (Linear + GELU(tanh)) x n_hidden (width `hidden`)
 *              -> Linear -> [c0][t0]
 *              -> (ConvTranspose1d k=4 s=2 p=1 + GELU) x (n_conv - 1)
 *              -> ConvTranspose1d -> y [conv_ch[n_conv-1]][t0 * 2^n_conv]
 * BF16 weights and activations, FP32 accumulation, FP32 master weights, MSE
 * loss, Adam.  Parameters are one flat FP32 vector: W_l [out][in], b_l for
 * each hidden layer, W_dec, b_dec, then Wc_j [c_in][c_out][4], bc_j.
 *
 * Conventions: every call returns 0 on success or a negative dgsem_status
 * (include/dgsem.h); srg_last_error() gives the message.  Device arrays are
 * FP32 and row-major: x [batch][d_in], y / target [batch][c_out][t_out].
 * batch must be a multiple of 64 and at most max_batch; d_in and hidden
 * multiples of 64; c0*t0 a multiple of 64.
 */
#ifndef SURROGATE_H
#define SURROGATE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srg_net srg_net;

typedef struct {
  int d_in;          /* input features (2 x number of PMUTs)       */
  int hidden;        /* width of the hidden layers                  */
  int n_hidden;      /* number of Linear+GELU layers (>= 1)         */
  int c0, t0;        /* decoder output: channels x samples          */
  int n_conv;        /* transposed convolutions (1..8)              */
  int conv_ch[8];    /* output channels of each convolution         */
} srg_config;

/* Create a network with parameters drawn uniformly in +-1/sqrt(fan_in)
 * (deterministic in `seed`) and buffers for up to max_batch patterns. */
int srg_create(const srg_config* cfg, int max_batch, unsigned long long seed, srg_net** out);

/* Number of parameters; copies of the FP32 master parameters and of the
 * gradients of the last srg_backward (host arrays of n floats). */
size_t srg_num_params(const srg_net* net);
int srg_get_params(const srg_net* net, float* host, size_t n);
int srg_set_params(srg_net* net, const float* host, size_t n);
int srg_get_grads(const srg_net* net, float* host, size_t n);

/* Forward pass for `batch` patterns; y receives the traces (device). */
int srg_forward(srg_net* net, const float* x, int batch, float* y, void* stream);

/* Forward + backward of the MSE loss against target; gradients are kept in
 * the network, the loss is written to *loss (host). */
int srg_backward(srg_net* net, const float* x, const float* target, int batch, double* loss, void* stream);

/* One Adam update of the master parameters with the kept gradients
 * (bias-corrected; the step counter is kept in the network). */
int srg_adam_step(srg_net* net, float lr, float beta1, float beta2, float eps, void* stream);

/* srg_backward followed by srg_adam_step (beta1 0.9, beta2 0.999, eps 1e-8). */
int srg_train_step(srg_net* net, const float* x, const float* target, int batch, float lr, double* loss,
                   void* stream);

/* Throughput of the dense-layer product on the tensor cores: C = A B^T with
 * A [M][K], B [N][K] BF16 (constant fill), FP32 C, reps launches after one
 * warm-up, timed with CUDA events on `stream`; *tflops = 2 M N K reps / time.
 * N and K multiples of 64.  Allocates its operands for the call. */
int srg_gemm_bench(int M, int N, int K, int reps, double* tflops, void* stream);

const char* srg_last_error(void);
void srg_destroy(srg_net* net);

#ifdef __cplusplus
}
#endif

#endif /* SURROGATE_H */
