// Instantiation unit: fused sum-factorised kernels for hex elements in double.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_hex_f64(int P, bool affine, const SFArgs<double>& a, cudaStream_t s) {
    return sf_dispatch<HP_HEX, double>(P, affine, a, s);
}
}  // namespace hp
