// FP64 instantiations of the fused volume kernel (see vol_impl.cuh), boxes
// without absorbing sides.
#include "vol_impl.cuh"

template cudaError_t launch_vol_flag<double, false>(const VolSpec&, int, cudaStream_t);
int vol_tma_box_f64(int N, int tile, unsigned box[3], unsigned vbox[3]) {
  return dgvol::tma_box<double>(N, tile, box, vbox);
}
