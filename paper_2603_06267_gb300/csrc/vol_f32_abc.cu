// FP32 instantiations of the fused volume kernel (see vol_impl.cuh), boxes
// with absorbing sides.
#include "vol_impl.cuh"

template cudaError_t launch_vol_flag<float, true>(const VolSpec&, int, cudaStream_t);
