// Instantiation unit: fused sum-factorised kernels for pyr elements in double.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_pyr_f64(int P, bool affine, int tile, const SFArgs<double>& a, cudaStream_t s) {
    return sf_dispatch<HP_PYR, double>(P, affine, tile, a, s);
}
}  // namespace hp
