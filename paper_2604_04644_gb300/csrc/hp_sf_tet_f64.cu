// Instantiation unit: fused sum-factorised kernels for tet elements in double.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_tet_f64(int P, bool affine, int tile, const SFArgs<double>& a, cudaStream_t s) {
    return sf_dispatch<HP_TET, double>(P, affine, tile, a, s);
}
}  // namespace hp
