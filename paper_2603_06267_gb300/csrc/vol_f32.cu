// FP32 instantiations of the fused volume kernel (see vol_impl.cuh), boxes
// without absorbing sides.
#include "vol_impl.cuh"

template cudaError_t launch_vol_flag<float, false>(const VolSpec&, int, cudaStream_t);
int vol_tma_box_f32(int N, int tile, unsigned box[3], unsigned vbox[3]) {
  return dgvol::tma_box<float>(N, tile, box, vbox);
}

namespace dgvol {
// Diagnostic for the failure path: one warp waits, with the pipeline's
// bounded wait, on an mbarrier that nothing arrives at, and records the
// give-up in the status word (3) like a stalled TMA stage would (1).
__global__ void wait_probe_kernel(int* err, long long budget) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0, budget) && threadIdx.x == 0) atomicExch(err, 3);
}
}  // namespace dgvol

cudaError_t launch_wait_probe(int* err, long long budget, cudaStream_t s) {
  dgvol::wait_probe_kernel<<<1, 32, 0, s>>>(err, budget);
  return cudaGetLastError();
}
