// Instantiation unit: fused sum-factorised kernels for prism elements in float.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_prism_f32(int P, bool affine, int tile, const SFArgs<float>& a, cudaStream_t s) {
    return sf_dispatch<HP_PRISM, float>(P, affine, tile, a, s);
}
}  // namespace hp
