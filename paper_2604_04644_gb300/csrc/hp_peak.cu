// Measured FP64 fused multiply-add rate of the current GPU: the denominator
// of the FP64 pipe's roofline.  Every thread runs kChains independent FMA
// recurrences x <- a x + b (a < 1, so the values stay bounded and normal) for
// `iters` steps; the grid fills every SM with several CTAs, so the pipe, not
// the latency of one chain, sets the time.
#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * threadIdx.x + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * (int64_t)kPeakThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" hp_status hp_peak_fp64(int device, int iters, double* tflops, double* ms, void* stream) {
    if (!tflops || iters < 1 || iters > (1 << 24)) {
        set_error("hp_peak_fp64: tflops must be non-null and iters in 1..2^24");
        return HP_ERR_ARG;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) {
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) return cuda_fail(e, "hp_peak_fp64");
    }
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fma_peak_kernel, kPeakThreads, 0);
    const int grid = sms * (per > 0 ? per : 1);
    cudaStream_t s = (cudaStream_t)stream;
    double* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * (size_t)grid * kPeakThreads);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 1e30f;
    // one warm-up launch, then the fastest of three
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
        cudaEventRecord(a, s);
        fma_peak_kernel<<<grid, kPeakThreads, 0, s>>>(out, iters, 0.999999, 1e-7);
        e = cudaGetLastError();
        cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&t, a, b);
        if (r > 0 && t < best) best = t;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(out);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "hp_peak_fp64");
    const double flops = 2.0 * kChains * (double)iters * grid * kPeakThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return HP_OK;
}
