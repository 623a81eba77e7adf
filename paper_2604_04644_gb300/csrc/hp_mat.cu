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
// CTA covers are staged in shared memory; at N_P <= 32 a thread issues all of
// its output's N_P loads before the first product and reads the coefficients
// from global memory (no staging, no barrier).
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

// out[e][m] = sum_n H^e[m][n] in[e][n], one (e, m) pair per thread, the
// coefficients of the CTA's elements staged in shared memory
template <typename T>
__global__ void __launch_bounds__(kMatThreads) mat_apply_kernel(const T* __restrict__ Ht, const int64_t* __restrict__ coeff_off,
                                                                int64_t ne, int NP, const T* __restrict__ in, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    const int64_t total = ne * NP;
    const int64_t c0 = (int64_t)blockIdx.x * kMatThreads;
    const int64_t e_first = c0 / NP;
    const int64_t c_last = min(c0 + kMatThreads, total) - 1;
    const int n_el = (int)(c_last / NP - e_first + 1);
    for (int i = threadIdx.x; i < n_el * NP; i += kMatThreads) {
        const int le = i / NP;
        su[i] = in[coeff_off[e_first + le] + (i - le * NP)];
    }
    __syncthreads();
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
    T sum = T(0);
#pragma unroll
    for (int k = 0; k < kMatUnroll; ++k) sum += acc[k];
    out[coeff_off[e] + mo] = sum;
}

// Small matrices (N_P <= NPMAX <= 32): one (e, m) pair per thread, all of
// its N_P stored values loaded before the first product and no shared-memory
// staging (no CTA barrier): the element's coefficients are read straight from
// global memory, where the N_P threads of the element share their cache lines.
// Measured on synthetic FP32 blocks of 512 MB: 0.61 (N_P = 4) to 0.86
// (N_P = 16) of the copy bandwidth, against 0.39-0.68 for staged tiles of
// four pairs per thread.
template <typename T, int NPMAX>
__global__ void __launch_bounds__(kMatThreads) mat_apply_small_kernel(const T* __restrict__ Ht,
                                                                      const int64_t* __restrict__ coeff_off, int64_t ne,
                                                                      int NP, const T* __restrict__ in, T* __restrict__ out) {
    const int64_t total = ne * NP;
    const int64_t c = (int64_t)blockIdx.x * kMatThreads + threadIdx.x;
    if (c >= total) return;
    T hv[NPMAX];
#pragma unroll
    for (int n = 0; n < NPMAX; ++n) hv[n] = n < NP ? __ldcs(Ht + (int64_t)n * total + c) : T(0);
    const int64_t e = c / NP;
    const int64_t o = __ldg(coeff_off + e);
    T acc = T(0);
#pragma unroll
    for (int n = 0; n < NPMAX; ++n) {
        if (n < NP) acc += hv[n] * __ldg(in + o + n);
    }
    out[o + (c - e * NP)] = acc;
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
    const int vs = f64 ? 8 : 4;
    // staged path: above 32 modes (FP32) or 16 (FP64, whose 32 loaded values a
    // thread cost more occupancy than the FP64 pipe, the limit there, can spare)
    if (NP > (f64 ? 16 : 32)) {
        const int64_t blocks = (total + kMatThreads - 1) / kMatThreads;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        const size_t smem = (size_t)(kMatThreads / NP + 2) * NP * vs;     // at most kMatThreads / NP + 2 elements
        if (f64)
            mat_apply_kernel<double><<<(unsigned)blocks, kMatThreads, smem, s>>>((const double*)Ht, coeff_off, ne, NP,
                                                                               (const double*)in, (double*)out);
        else
            mat_apply_kernel<float><<<(unsigned)blocks, kMatThreads, smem, s>>>((const float*)Ht, coeff_off, ne, NP,
                                                                              (const float*)in, (float*)out);
        return cudaGetLastError();
    }
    const int64_t blocks = (total + kMatThreads - 1) / kMatThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    auto go = [&](auto kern, auto* H, auto* x, auto* y) {
        kern<<<(unsigned)blocks, kMatThreads, 0, s>>>(H, coeff_off, ne, NP, x, y);
    };
    if (f64) {
        const double* H = (const double*)Ht;
        const double* x = (const double*)in;
        double* y = (double*)out;
        if (NP <= 8) go(mat_apply_small_kernel<double, 8>, H, x, y);
        else go(mat_apply_small_kernel<double, 16>, H, x, y);
    } else {
        const float* H = (const float*)Ht;
        const float* x = (const float*)in;
        float* y = (float*)out;
        if (NP <= 8) go(mat_apply_small_kernel<float, 8>, H, x, y);
        else if (NP <= 16) go(mat_apply_small_kernel<float, 16>, H, x, y);
        else go(mat_apply_small_kernel<float, 32>, H, x, y);
    }
    return cudaGetLastError();
}

}  // namespace hp
