// Fifth-generation tensor-core primitives (sm_100 family, tcgen05) as inline
// PTX: tensor-memory allocation, shared-memory matrix descriptors, the
// instruction descriptor of kind::tf32 / kind::f16 MMAs with FP32
// accumulation, commit to an mbarrier, and tensor-memory loads.
//
// Operand layouts: swizzled, K-major or (for the BF16 backward operand)
// MN-major: rows of 128 / 64 / 32 bytes in 8-row atoms at 1024-byte aligned
// bases; with the 128-byte swizzle the 16-byte chunk c of row r sits at chunk
// c ^ (r mod 8), with the 64-byte one at c ^ ((r / 2) mod 4), so that the
// tensor core reads the rows of an atom from different shared-memory banks.
#pragma once
#include <cstdint>
#include "hp_device.cuh"

namespace hp {
namespace tc {

// byte offset of 4-byte element (r, k) in a K-major tile with the 64-byte
// swizzle (k < 16)
__host__ __device__ constexpr uint32_t sw64_offset(uint32_t r, uint32_t k) {
    return r * 64 + ((((k * 4) >> 4) ^ ((r >> 1) & 3)) << 4) + ((k * 4) & 15);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {   // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {   // one full warp
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // the allocating warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Descriptor of a swizzled K-major operand: start address (a K step of the
// MMA moves it by 32 bytes inside the swizzle row), SBO = 8-row atom stride,
// mode 2 = 128-byte swizzle, 4 = 64-byte swizzle; the leading offset is unused.
constexpr uint32_t kSw128 = 2, kSw64 = 4, kSw32 = 6;
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t saddr, uint32_t sbo, uint32_t mode) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)mode << 61;
    return d;
}

// Swizzled descriptor with an explicit leading offset (MN-major operands:
// LBO = stride between swizzle atoms along MN, SBO = stride between 8-row
// groups along K)
__device__ __forceinline__ uint64_t smem_desc_sw_lbo(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t mode) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)mode << 61;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt`
// (kind::f16: 0 = F16, 1 = BF16; kind::tf32: 2 = TF32), both K-major,
// N (multiple of 16 for M = 128, 8..256) and M (64 or 128).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
constexpr uint32_t kFmtBF16 = 1, kFmtTF32 = 2;

// D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// arrive once on `bar` when every MMA issued so far by this thread has completed
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// Warp-issued forms: every lane of a converged warp makes the call with the
// same operands and one lane, chosen by elect.sync, issues.  A single lane
// issuing from a divergent branch with a run-time instruction descriptor
// waits about 150 clocks per MMA whatever its N (measured on GB300: M = 128,
// K = 16); issued this way an MMA takes what its operands cost, 48 / 64 / 128
// clocks for N = 64 / 128 / 256 (the last at the peak rate).
__device__ __forceinline__ void mma_tf32_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_bf16_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// commit by the lane that elect.sync picks (the same lane as the MMAs': the
// first active one)
__device__ __forceinline__ void commit_w(uint64_t* bar) {
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp-collective load of 32 lanes x 16 consecutive 32-bit columns: thread i
// of the warp receives lane (lane base + i) of the accumulator.  The warp may
// only address the lane quarter (warp id mod 4) * 32 .. + 31.
__device__ __forceinline__ void ld_32x16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// four 32 x 8 loads at columns taddr + i * stride (i = 0..3) and one wait:
// v[i] receives the i-th group
__device__ __forceinline__ void ld_32x8_x4(uint32_t taddr, uint32_t stride, float (&v)[4][8]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr), "r"(taddr + stride), "r"(taddr + 2 * stride), "r"(taddr + 3 * stride)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i / 8][i % 8] = __uint_as_float(r[i]);
}

// four 32 x 4 loads at columns taddr + i * stride (i = 0..3) and one wait
__device__ __forceinline__ void ld_32x4_x4(uint32_t taddr, uint32_t stride, float (&v)[4][4]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%17];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%18];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [%19];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr), "r"(taddr + stride), "r"(taddr + 2 * stride), "r"(taddr + 3 * stride)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i / 4][i % 4] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld_x4(uint32_t taddr, uint32_t stride, float (&v)[4][4]) { ld_32x4_x4(taddr, stride, v); }
__device__ __forceinline__ void ld_x4(uint32_t taddr, uint32_t stride, float (&v)[4][8]) { ld_32x8_x4(taddr, stride, v); }

// round to the TF32 grid (10-bit mantissa, nearest, ties away)
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace hp
