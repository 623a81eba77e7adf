// Instantiation unit: fused sum-factorised kernels for prism elements in double.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_prism_f64(int P, bool affine, int tile, const SFArgs<double>& a, cudaStream_t s) {
    return sf_dispatch<HP_PRISM, double>(P, affine, tile, a, s);
}
}  // namespace hp
