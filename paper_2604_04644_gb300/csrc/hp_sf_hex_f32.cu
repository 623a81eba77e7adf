// Instantiation unit: fused sum-factorised kernels for hex elements in float.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_hex_f32(int P, bool affine, int tile, const SFArgs<float>& a, cudaStream_t s) {
    return sf_dispatch<HP_HEX, float>(P, affine, tile, a, s);
}
}  // namespace hp
