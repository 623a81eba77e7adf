// Matrix-based strategy: stored per-element dense operator matrices H^e
// (Sec. 3.3, implementation strategies: the elemental matrices are assembled
// once and stored, and an apply is one dense matrix-vector product per
// element).
//
// Build: column m of every H^e of a block at once, by applying the FP64
// sum-factorised operator to the block's m-th unit coefficient vectors
// (mat_unit_kernel, then the operator, then mat_collect_kernel); the result is
// the matrix-free operator's own matrix, exact up to its rounding.
//
// Storage, per block: Ht[n][e][m] = H^e[m][n] (input mode n outermost, then
// element, then output mode), so that for a fixed n the threads of a warp,
// which own consecutive (e, m) pairs, read consecutive addresses: every load
// of the apply is a coalesced 128-byte (FP32) or 256-byte (FP64) warp access.
//
// Apply: HBM-bound streaming of the N_P^2 stored values per element (no
// reuse: each is read once per apply); the coefficients of the few elements a
// CTA covers are staged in shared memory.  At N_P <= 16 each thread computes
// four outputs, so that enough loads are in flight per thread.
#include "hp_internal.h"

namespace hp {
namespace {

__global__ void mat_unit_kernel(double* x, const int64_t* coeff_off, int64_t ne, int NP, int m) {
    const int64_t total = ne * NP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / NP;
        const int mm = (int)(i - e * NP);
        x[coeff_off[e] + mm] = mm == m ? 1.0 : 0.0;
    }
}

template <typename T>
__global__ void mat_collect_kernel(const double* y, const int64_t* coeff_off, int64_t ne, int NP, int m, T* Ht) {
    const int64_t total = ne * NP;
    T* col = Ht + (int64_t)m * total;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / NP;
        const int mm = (int)(i - e * NP);
        col[i] = (T)y[coeff_off[e] + mm];
    }
}

constexpr int kMatThreads = 256;
constexpr int kMatUnroll = 8;

// out[e][m] = sum_n H^e[m][n] in[e][n]; each thread takes K (e, m) pairs
// kMatThreads apart in a tile of K * kMatThreads consecutive pairs, so that at
// small N_P (few loads per output) K outputs' loads are in flight together;
// the coefficients of the tile's elements are staged in shared memory
template <typename T, int K>
__global__ void __launch_bounds__(kMatThreads) mat_apply_kernel(const T* __restrict__ Ht, const int64_t* __restrict__ coeff_off,
                                                                int64_t ne, int NP, const T* __restrict__ in, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    constexpr int TILE = K * kMatThreads;
    const int64_t total = ne * NP;
    const int64_t c0 = (int64_t)blockIdx.x * TILE;
    const int64_t e_first = c0 / NP;
    const int64_t c_last = min(c0 + TILE, total) - 1;
    const int n_el = (int)(c_last / NP - e_first + 1);
    for (int i = threadIdx.x; i < n_el * NP; i += kMatThreads) {
        const int le = i / NP;
        su[i] = in[coeff_off[e_first + le] + (i - le * NP)];
    }
    __syncthreads();
    if constexpr (K == 1) {
        const int64_t c = c0 + threadIdx.x;
        if (c >= total) return;
        const int64_t e = c / NP;
        const int mo = (int)(c - e * NP);
        const T* u = su + (e - e_first) * NP;
        const T* h = Ht + c;
        T acc[kMatUnroll];
#pragma unroll
        for (int k = 0; k < kMatUnroll; ++k) acc[k] = T(0);
        int n = 0;
        for (; n + kMatUnroll <= NP; n += kMatUnroll) {
            T hv[kMatUnroll];
#pragma unroll
            for (int k = 0; k < kMatUnroll; ++k) hv[k] = __ldcs(h + (int64_t)(n + k) * total);
#pragma unroll
            for (int k = 0; k < kMatUnroll; ++k) acc[k] += hv[k] * u[n + k];
        }
        for (; n < NP; ++n) acc[0] += __ldcs(h + (int64_t)n * total) * u[n];
        T s = T(0);
#pragma unroll
        for (int k = 0; k < kMatUnroll; ++k) s += acc[k];
        out[coeff_off[e] + mo] = s;
    } else {
        int64_t cc[K];
        const T* uu[K];
        T acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            cc[k] = c0 + threadIdx.x + k * kMatThreads;
            const int64_t e = (cc[k] < total ? cc[k] : c0) / NP;
            uu[k] = su + (e - e_first) * NP;
            acc[k] = T(0);
        }
        for (int n = 0; n < NP; ++n) {
            T hv[K];
#pragma unroll
            for (int k = 0; k < K; ++k) hv[k] = cc[k] < total ? __ldcs(Ht + (int64_t)n * total + cc[k]) : T(0);
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] += hv[k] * uu[k][n];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (cc[k] >= total) break;
            const int64_t e = cc[k] / NP;
            out[coeff_off[e] + (cc[k] - e * NP)] = acc[k];
        }
    }
}

int grid_for(int64_t n) {
    const int64_t b = (n + kMatThreads - 1) / kMatThreads;
    return (int)(b < 1 ? 1 : (b > 65535 * 4 ? 65535 * 4 : b));
}

}  // namespace

cudaError_t mat_unit(double* x, const int64_t* coeff_off, int64_t ne, int NP, int m, cudaStream_t s) {
    mat_unit_kernel<<<grid_for(ne * NP), kMatThreads, 0, s>>>(x, coeff_off, ne, NP, m);
    return cudaGetLastError();
}

cudaError_t mat_collect(const double* y, const int64_t* coeff_off, int64_t ne, int NP, int m, void* Ht, bool f64,
                        cudaStream_t s) {
    if (f64) mat_collect_kernel<double><<<grid_for(ne * NP), kMatThreads, 0, s>>>(y, coeff_off, ne, NP, m, (double*)Ht);
    else mat_collect_kernel<float><<<grid_for(ne * NP), kMatThreads, 0, s>>>(y, coeff_off, ne, NP, m, (float*)Ht);
    return cudaGetLastError();
}

cudaError_t mat_apply(const void* Ht, const int64_t* coeff_off, int64_t ne, int NP, const void* in, void* out, bool f64,
                      cudaStream_t s) {
    const int64_t total = ne * NP;
    if (total <= 0) return cudaSuccess;
    // small matrices: four outputs a thread (more loads in flight per thread)
    const int K = NP <= 16 ? 4 : 1;
    const int64_t tile = (int64_t)K * kMatThreads;
    const int64_t blocks = (total + tile - 1) / tile;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    // a CTA covers at most tile / NP + 2 elements
    const size_t smem = (size_t)(tile / NP + 2) * NP * (f64 ? 8 : 4);
    if (f64) {
        if (K == 4)
            mat_apply_kernel<double, 4><<<(unsigned)blocks, kMatThreads, smem, s>>>((const double*)Ht, coeff_off, ne, NP,
                                                                                (const double*)in, (double*)out);
        else
            mat_apply_kernel<double, 1><<<(unsigned)blocks, kMatThreads, smem, s>>>((const double*)Ht, coeff_off, ne, NP,
                                                                                (const double*)in, (double*)out);
    } else {
        if (K == 4)
            mat_apply_kernel<float, 4><<<(unsigned)blocks, kMatThreads, smem, s>>>((const float*)Ht, coeff_off, ne, NP,
                                                                              (const float*)in, (float*)out);
        else
            mat_apply_kernel<float, 1><<<(unsigned)blocks, kMatThreads, smem, s>>>((const float*)Ht, coeff_off, ne, NP,
                                                                              (const float*)in, (float*)out);
    }
    return cudaGetLastError();
}

}  // namespace hp
