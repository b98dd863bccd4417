// Element-stiffness kernels of the general-hexahedron step, FP64
// instantiations (kernel and variants in hex_vol.cuh).
#include "hex_vol.cuh"

namespace hex {

template <>
cudaError_t launch_hex_vol<double>(const HexVolArgs<double>& a, int n, int variant, cudaStream_t s) {
  return launch_hex_vol_impl<double>(a, n, variant, s);
}

}  // namespace hex
