// Instantiation unit: fused sum-factorised kernels for hex elements in double.
#include "hp_sf.cuh"

namespace hp {
cudaError_t sf_launch_hex_f64(int P, bool affine, int tile, const SFArgs<double>& a, cudaStream_t s) {
    return sf_dispatch<HP_HEX, double>(P, affine, tile, a, s);
}
}  // namespace hp

namespace hp {
int sf_epb_host(int P, int tile, bool f64) { return f64 ? sf_epb<double>(P, tile) : sf_epb<float>(P, tile); }
}  // namespace hp
