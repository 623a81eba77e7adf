// Instantiation unit: fused sum-factorised kernels for tet elements in float.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_tet_f32(int P, bool affine, int tile, const SFArgs<float>& a, cudaStream_t s) {
    return sf_dispatch<HP_TET, float>(P, affine, tile, a, s);
}
}  // namespace hp
