// Device helpers shared by the kernels: collapsed-coordinate maps, the
// chain-rule factor d eta / d xi, and the bulk-copy (TMA) staging of the
// reference tables into shared memory with bounded mbarrier waits.
#pragma once
#include <atomic>
#include <cstdint>

#include "hp_internal.h"

namespace hp {

// Launch set-up of a persistent kernel on the current device: raises its
// dynamic shared-memory limit to `smem` there and returns in *cap its grid
// cap (SMs x resident CTAs).  The result is cached per device ordinal in
// `caps` (one zero-initialised array per kernel), so a second device gets its
// own attribute call; two threads that race only repeat the same idempotent
// calls.
constexpr int kMaxDevices = 64;
template <typename K>
cudaError_t persistent_grid_cap(K kern, int threads, int smem, std::atomic<int>* caps, int* cap) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int c = caps[dev].load(std::memory_order_acquire);
    if (c == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int sms = 0, per = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
        if (e != cudaSuccess) return e;
        c = sms * (per > 0 ? per : 1);
        caps[dev].store(c, std::memory_order_release);
    }
    *cap = c;
    return cudaSuccess;
}

// xi(eta) of the collapsed coordinates (paper Sec. 2.3, Duffy transformation;
// repeated for the 3-D shapes): prism collapses xi1 by xi3, pyramid xi1 and
// xi2 by xi3, tetrahedron xi1 by (xi2, xi3) and xi2 by xi3.
template <int SHAPE>
__device__ __forceinline__ void xi_from_eta(double e1, double e2, double e3, double* xi) {
    if (SHAPE == HP_HEX) {
        xi[0] = e1; xi[1] = e2; xi[2] = e3;
    } else if (SHAPE == HP_PRISM) {
        xi[0] = 0.5 * (1.0 + e1) * (1.0 - e3) - 1.0; xi[1] = e2; xi[2] = e3;
    } else if (SHAPE == HP_PYR) {
        xi[0] = 0.5 * (1.0 + e1) * (1.0 - e3) - 1.0;
        xi[1] = 0.5 * (1.0 + e2) * (1.0 - e3) - 1.0;
        xi[2] = e3;
    } else {
        xi[0] = 0.25 * (1.0 + e1) * (1.0 - e2) * (1.0 - e3) - 1.0;
        xi[1] = 0.5 * (1.0 + e2) * (1.0 - e3) - 1.0;
        xi[2] = e3;
    }
}

// T[d][a] = d eta_d / d xi_a at a point given in eta (the G of Sec. 2.3 in 3-D).
template <int SHAPE, typename R>
__host__ __device__ __forceinline__ void deta_dxi(R e1, R e2, R e3, R T[3][3]) {
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a) T[d][a] = (d == a) ? R(1) : R(0);
    if (SHAPE == HP_PRISM) {
        R r3 = R(1) / (R(1) - e3);
        T[0][0] = R(2) * r3;
        T[0][2] = (R(1) + e1) * r3;
    } else if (SHAPE == HP_PYR) {
        R r3 = R(1) / (R(1) - e3);
        T[0][0] = R(2) * r3;
        T[0][2] = (R(1) + e1) * r3;
        T[1][1] = R(2) * r3;
        T[1][2] = (R(1) + e2) * r3;
    } else if (SHAPE == HP_TET) {
        R r3 = R(1) / (R(1) - e3);
        R r23 = R(2) / ((R(1) - e2) * (R(1) - e3));   // 1 / (-xi2 - xi3)
        T[0][0] = R(2) * r23;
        T[0][1] = (R(1) + e1) * r23;
        T[0][2] = (R(1) + e1) * r23;
        T[1][1] = R(2) * r3;
        T[1][2] = (R(1) + e2) * r3;
    }
}

// ------------------------------------------------------------ mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared (TMA engine).  dst, src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for `phase` of the barrier for at most `limit_ns`; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, uint64_t limit_ns) {
    uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: far beyond any legitimate copy

// Stage `bytes` of `src` into shared memory `dst` with one bulk copy issued by
// thread 0; every thread waits on the barrier.  Returns false (and latches
// DERR_TIMEOUT) if the copy did not land within the limit; in that case the
// caller must not touch `dst` and should return (after a second bounded wait
// for the copy, done here, so no copy is left in flight).
__device__ __forceinline__ bool stage_tables(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                             unsigned int* err) {
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes);
        bulk_g2s(dst, src, bytes, bar);
    }
    bool ok = mbar_wait_bounded(bar, 0, kWaitLimitNs);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(err, DERR_TIMEOUT);
        mbar_wait_bounded(bar, 0, kWaitLimitNs);
    }
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// The same with a barrier the caller initialised once (count 1) and reuses:
// each staging waits on `phase`, which then flips for the next one.  Every
// thread must have finished with the previous tables (a CTA barrier) before
// the call.
__device__ __forceinline__ bool stage_tables_phase(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                   uint32_t& phase, unsigned int* err) {
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar, bytes);
        bulk_g2s(dst, src, bytes, bar);
    }
    bool ok = mbar_wait_bounded(bar, phase, kWaitLimitNs);
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(err, DERR_TIMEOUT);
        mbar_wait_bounded(bar, phase, kWaitLimitNs);
    }
    phase ^= 1u;
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

}  // namespace hp
