// Elemental-matrix strategy on the fifth-generation tensor cores (TF32 inputs,
// FP32 accumulation in tensor memory).
//
// The operator of the elemental-matrix form (paper Sec. 3.2; Eq. (helm1) with
// the reference matrices of Sec. 2.2):
//   out_e = sum_{c,c'} A_c^T  diag(M_{cc'}(e))  A_c' uhat_e,
// A_0 = B (basis at the points), A_d = dB/d eta_d, M_00 = lambda w|J| (mass
// term), M_dd' = G_dd' (the six metric factors), M_0d = 0.  Mass uses c = 0
// only (M_00 = w|J|), the Laplacian c = 1..3.
//
// Organisation (one CTA per SM, persistent over work items = a tile of 128
// elements and a range of its point chunks):
//   forward  [V_0..V_3][128 elem x 4*16] = U[128 x K_P] * [F_0; ..; F_3]^T      (tcgen05, TMEM;
//            one MMA per K step covers the components, so U is read once)
//   metric   V'_c = sum_c' M_cc' V_c'  pointwise, by the eight warps that read the TMEM lanes
//   backward O[128 elem x N_P]       += V'_c[128 x 16] * R_c[N_P x 16]^T     (tcgen05, TMEM)
// over chunks of 16 quadrature points.  U (the element coefficients) stays in
// shared memory for the work item; the reference tiles F_c, R_c are laid out
// on the host in the tensor core's shared-memory order and streamed by 1-D
// bulk copies (TMA) through a ring of stages (TF32: the forward operand in K
// slices of 32 modes, the backward tiles one component at a time; BF16: one
// stage per chunk holding its whole forward operand, which the backward MMAs
// read again as an MN-major operand, so no backward tiles are streamed).  Three forward
// accumulators are in flight and the V' tiles are double-buffered, so the
// forward MMAs run two chunks ahead of the metric and the metric of chunk k
// overlaps the backward MMAs of chunk k-1.
// Roles: warps 0-7 gather U, run the metric and write the outputs (warp w
// reads TMEM lanes 32 (w mod 4).. and half w / 4 of each chunk's points);
// warp 8 issues the bulk copies; warp 9 issues the MMAs.  Every wait is
// bounded; a timeout latches DERR_TIMEOUT, stops every role, drains the
// copies and MMAs in flight and frees the tensor memory before the CTA exits.
#include <cuda_bf16.h>

#include "hp_tc.cuh"

namespace hp {
namespace {

constexpr int kNPT = 16;          // quadrature points per chunk
constexpr int kHalf = kNPT / 2;   // points per epilogue thread
constexpr int kMaxStages = 8;     // bulk-copy ring: as many stages (2..8) as fit in shared memory
constexpr int kTmemCols = 512;
constexpr int kFwdBufs = 3;       // forward accumulators in flight: the forward MMAs run two chunks ahead
constexpr int kOutCol = kFwdBufs * 4 * 16;   // TMEM column of the output accumulator
constexpr int kEpi = 256;         // epilogue threads
constexpr int kThreads = kEpi + 64;
constexpr int kSliceBytes = 4 * kNPT * 128;   // forward operand slice: 64 rows x 128 bytes of modes

// Operand element type: TF32 (ES = 4, kind::tf32, K = 8 per MMA) or BF16
// (ES = 2, kind::f16, K = 16 per MMA); every MMA K step is 32 bytes.  The
// 16-point tiles (V', backward R) have rows of 16 ES bytes: 64-byte swizzle
// for TF32, 32-byte swizzle for BF16.
template <int ES>
struct Op {
    static constexpr int KR = 128 / ES;                   // modes per 128-byte row (slice width)
    static constexpr int VROW = kNPT * ES;                // bytes per row of a 16-point tile
    static constexpr int VBYTES = 128 * VROW;             // one V' tile
    static constexpr uint32_t VSW = ES == 4 ? tc::kSw64 : tc::kSw32;
    static constexpr uint32_t FMT = ES == 4 ? tc::kFmtTF32 : tc::kFmtBF16;
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        if constexpr (ES == 4) tc::mma_tf32(d, a, b, id, acc);
        else tc::mma_bf16(d, a, b, id, acc);
    }
    // byte offset of element (r, k) in a 128-byte swizzled row block
    __device__ static uint32_t off128(uint32_t r, uint32_t k) {
        return r * 128 + ((((k * ES) >> 4) ^ (r & 7)) << 4) + ((k * ES) & 15);
    }
    // byte offset of the 16-byte chunk holding points p..p+16/ES-1 of row r of a 16-point tile
    __device__ static uint32_t offv(uint32_t r, uint32_t p) {
        if constexpr (ES == 4) return tc::sw64_offset(r, p);
        else return r * 32 + ((((p * 2) >> 4) ^ ((r >> 2) & 1)) << 4);
    }
    // 16 bytes of operands from 16 / ES floats
    __device__ static uint4 pack(const float* x) {
        uint4 u;
        if constexpr (ES == 4) {
            u.x = __float_as_uint(tc::to_tf32(x[0])); u.y = __float_as_uint(tc::to_tf32(x[1]));
            u.z = __float_as_uint(tc::to_tf32(x[2])); u.w = __float_as_uint(tc::to_tf32(x[3]));
        } else {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
                w[i] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            u = make_uint4(w[0], w[1], w[2], w[3]);
        }
        return u;
    }
};

struct Bars {
    uint64_t full[kMaxStages], empty[kMaxStages];
    uint64_t u_full, fwd_full[kFwdBufs], fwd_empty[kFwdBufs], vp_full[2], vp_empty[2], out_full, out_empty, drain;
    uint32_t tmem;
    int abort;
};

// wait for `parity` of `bar`, giving up when another role aborted or after the
// time limit (then this role aborts every role)
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, Bars* B, unsigned int* err) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*reinterpret_cast<volatile int*>(&B->abort)) return false;
        if (global_ns() - t0 > kWaitLimitNs) {
            atomicExch(&B->abort, 1);
            atomicOr(err, DERR_TIMEOUT);
            return false;
        }
    }
    return true;
}
// epilogue warps take the decision warp-wide (the tensor-memory loads that
// follow are warp-collective)
__device__ __forceinline__ bool wait_warp(uint64_t* bar, uint32_t parity, Bars* B, unsigned int* err) {
    return __all_sync(0xffffffffu, wait_bar(bar, parity, B, err));
}
__device__ __forceinline__ void arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int ES>
__global__ void __launch_bounds__(kThreads, 1) tc_emat_kernel(const __grid_constant__ TCArgs a) {
    using O = Op<ES>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzle patterns are taken from shared-memory address bits: align to 1 KB
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    Bars* B = reinterpret_cast<Bars*>(smem);
    unsigned char* sU = smem + 1024;                                   // KP/32 blocks [128 x 32] tf32, 128 B swizzle
    unsigned char* sV = sU + 128 * a.KP * ES;                          // [2][4][128 x 16], 64 / 32 B swizzle
    unsigned char* sR = sV + 8 * O::VBYTES;                            // ring
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nst = a.stages;
    // work items: (tile of 128 elements, part of its point chunks); parts of one
    // tile add their partial outputs (the output was zeroed first)
    const int64_t nwork = (a.n_elem + 127) / 128 * a.nsplit;
    auto chunk_range = [&](int64_t w, int& kb, int& ke) {
        const int part = (int)(w % a.nsplit);
        kb = (int)((int64_t)a.nch * part / a.nsplit);
        ke = (int)((int64_t)a.nch * (part + 1) / a.nsplit);
    };

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) { mbar_init(&B->full[s], 1); mbar_init(&B->empty[s], 1); }
        mbar_init(&B->u_full, kEpi);
        for (int b = 0; b < kFwdBufs; ++b) {
            mbar_init(&B->fwd_full[b], 1);
            mbar_init(&B->fwd_empty[b], kEpi);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B->vp_full[b], kEpi);
            mbar_init(&B->vp_empty[b], 1);
        }
        mbar_init(&B->out_full, 1);
        mbar_init(&B->out_empty, kEpi);
        mbar_init(&B->drain, 1);
        B->abort = 0;
    }
    if (warp == 0) { tc::tmem_alloc(&B->tmem, kTmemCols); tc::tmem_relinquish(); }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = B->tmem;

    if (warp == 8) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int slot = 0;
            uint32_t pass = 0;
            uint32_t last_parity[kMaxStages];
            bool used[kMaxStages];
            for (int i = 0; i < kMaxStages; ++i) { last_parity[i] = 0; used[i] = false; }
            bool ok = true;
            auto put = [&](const unsigned char* src, uint32_t bytes) {
                if (!wait_bar(&B->empty[slot], pass ^ 1u, B, a.err)) { ok = false; return; }
                mbar_expect_tx(&B->full[slot], bytes);
                bulk_g2s(sR + (size_t)slot * a.stage_bytes, src, bytes, &B->full[slot]);
                used[slot] = true;
                last_parity[slot] = pass;
                if (++slot == nst) { slot = 0; pass ^= 1u; }
            };
            for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
                int kb, ke;
                chunk_range(w, kb, ke);
                // the MMA issuer's order: forward of chunk t, backward of chunk t - (kFwdBufs - 1);
                // BF16: one stage per chunk (all forward slices), read again by the backward
                if constexpr (ES == 2) {
                    for (int t = kb; t < ke && ok; ++t) put(a.img + (size_t)t * a.chunk_bytes, (uint32_t)a.fwd_bytes);
                    continue;
                }
                for (int t = kb; t < ke + kFwdBufs - 1 && ok; ++t) {
                    if (t < ke) {
                        const unsigned char* base = a.img + (size_t)t * a.chunk_bytes;
                        for (int sl = 0; sl * O::KR < a.KP && ok; ++sl) put(base + (size_t)sl * kSliceBytes, kSliceBytes);
                    }
                    const int kbw = t - (kFwdBufs - 1);
                    if (kbw >= kb) {
                        const unsigned char* base = a.img + (size_t)kbw * a.chunk_bytes + (size_t)a.fwd_bytes;
                        for (int c = a.c0; c < a.c1 && ok; ++c) put(base + (size_t)c * a.bwd_bytes, a.bwd_bytes);
                    }
                }
            }
            // no copy may still be landing when the CTA leaves
            for (int s = 0; s < nst; ++s)
                if (used[s]) {
                    const uint64_t t0 = global_ns();
                    while (!mbar_try_wait(&B->full[s], last_parity[s]) && global_ns() - t0 < kWaitLimitNs) {}
                }
        }
        __syncwarp();
    } else if (warp == 9) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id_f = tc::instr_desc(O::FMT, 128, kNPT * (a.c1 - a.c0));
            const uint32_t id_b = tc::instr_desc(O::FMT, 128, a.NPpad);
            int slot = 0;
            uint32_t pass = 0, nout = 0, ntile = 0, g0 = 0;   // g: chunks processed by this CTA
            bool ok = true;
            for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++ntile) {
                int kb, ke;
                chunk_range(w, kb, ke);
                if (!wait_bar(&B->u_full, ntile & 1u, B, a.err)) { ok = false; break; }
                if constexpr (ES == 2) {
                    // one ring stage per chunk: forward MMAs read its slices K-major;
                    // kFwdBufs - 1 chunks later the backward MMAs read the same stage
                    // MN-major (N = modes: 64-mode atoms one slice apart; K = the
                    // component's 16 points) and release it
                    const uint32_t id_bt = id_b | (1u << 16);                     // B operand MN-major
                    for (int t = kb; t < ke + kFwdBufs - 1 && ok; ++t) {
                        if (t < ke) {
                            const uint32_t g = g0 + (uint32_t)(t - kb), b = g % kFwdBufs, use = g / kFwdBufs;
                            const uint32_t st = g % nst, par = (g / nst) & 1u;
                            if (!wait_bar(&B->fwd_empty[b], (use & 1u) ^ 1u, B, a.err)) { ok = false; break; }
                            if (!wait_bar(&B->full[st], par, B, a.err)) { ok = false; break; }
                            tc::fence_after();
                            const uint32_t d = tbase + (uint32_t)((b * 4 + a.c0) * kNPT);
                            const uint32_t stage = smem_addr(sR + (size_t)st * a.stage_bytes);
                            for (int sl = 0; sl * O::KR < a.KP; ++sl) {
                                const uint32_t sa = smem_addr(sU) + sl * 128 * 128;
                                const uint32_t sb = stage + sl * kSliceBytes + a.c0 * 2 * 1024;
                                for (int s = 0; s < 4; ++s)
                                    O::mma(d, tc::smem_desc_sw(sa + s * 32, 1024, tc::kSw128),
                                           tc::smem_desc_sw(sb + s * 32, 1024, tc::kSw128), id_f, sl > 0 || s > 0);
                            }
                            tc::commit(&B->fwd_full[b]);
                        }
                        const int k = t - (kFwdBufs - 1);
                        if (k >= kb && ok) {
                            const uint32_t g = g0 + (uint32_t)(k - kb), b = g & 1u, use = g >> 1;
                            const uint32_t st = g % nst;
                            if (!wait_bar(&B->vp_full[b], use & 1u, B, a.err)) { ok = false; break; }
                            if (k == kb) {
                                if (!wait_bar(&B->out_empty, (nout & 1u) ^ 1u, B, a.err)) { ok = false; break; }
                                ++nout;
                            }
                            tc::fence_after();
                            const uint32_t stage = smem_addr(sR + (size_t)st * a.stage_bytes);
                            for (int c = a.c0; c < a.c1; ++c) {
                                const uint32_t sa = smem_addr(sV + (size_t)(b * 4 + c) * O::VBYTES);
                                // LBO: next 64-mode atom (next slice); SBO: next 8 points
                                const uint64_t db = tc::smem_desc_sw_lbo(stage + c * 2 * 1024, kSliceBytes, 1024, tc::kSw128);
                                O::mma(tbase + kOutCol, tc::smem_desc_sw(sa, 8 * O::VROW, O::VSW), db, id_bt,
                                       !(k == kb && c == a.c0));
                            }
                            tc::commit(&B->empty[st]);
                            tc::commit(&B->vp_empty[b]);
                        }
                    }
                    if (ok) tc::commit(&B->out_full);
                    g0 += (uint32_t)(ke - kb);
                    continue;
                }
                for (int t = kb; t < ke + kFwdBufs - 1 && ok; ++t) {
                    if (t < ke) {
                        const int k = t;
                        const uint32_t g = g0 + (uint32_t)(k - kb), b = g % kFwdBufs, use = g / kFwdBufs;
                        if (!wait_bar(&B->fwd_empty[b], (use & 1u) ^ 1u, B, a.err)) { ok = false; break; }
                        tc::fence_after();
                        // columns (b*4 + c0)*16 .. of the accumulator = components c0..c1-1
                        const uint32_t d = tbase + (uint32_t)((b * 4 + a.c0) * kNPT);
                        for (int sl = 0; sl * O::KR < a.KP && ok; ++sl) {
                            if (!wait_bar(&B->full[slot], pass, B, a.err)) { ok = false; break; }
                            tc::fence_after();
                            // K block sl of U (128 rows x 128 B) and rows 16 c0.. of the slice
                            const uint32_t sa = smem_addr(sU) + sl * 128 * 128;
                            const uint32_t sb = smem_addr(sR + (size_t)slot * a.stage_bytes) + a.c0 * 2 * 1024;
                            for (int s = 0; s < 4; ++s)
                                O::mma(d, tc::smem_desc_sw(sa + s * 32, 1024, tc::kSw128),
                                       tc::smem_desc_sw(sb + s * 32, 1024, tc::kSw128), id_f, sl > 0 || s > 0);
                            tc::commit(&B->empty[slot]);
                            if (++slot == nst) { slot = 0; pass ^= 1u; }
                        }
                        tc::commit(&B->fwd_full[b]);
                    }
                    const int k = t - (kFwdBufs - 1);          // backward of chunk k
                    if (k >= kb && ok) {
                        const uint32_t g = g0 + (uint32_t)(k - kb), b = g & 1u, use = g >> 1;
                        if (!wait_bar(&B->vp_full[b], use & 1u, B, a.err)) { ok = false; break; }
                        if (k == kb) {
                            if (!wait_bar(&B->out_empty, (nout & 1u) ^ 1u, B, a.err)) { ok = false; break; }
                            ++nout;
                        }
                        tc::fence_after();
                        for (int c = a.c0; c < a.c1 && ok; ++c) {
                            if (!wait_bar(&B->full[slot], pass, B, a.err)) { ok = false; break; }
                            tc::fence_after();
                            const uint32_t sa = smem_addr(sV + (size_t)(b * 4 + c) * O::VBYTES);
                            const uint32_t sb = smem_addr(sR + (size_t)slot * a.stage_bytes);
                            for (int s = 0; s < O::VROW / 32; ++s)
                                O::mma(tbase + kOutCol, tc::smem_desc_sw(sa + s * 32, 8 * O::VROW, O::VSW),
                                       tc::smem_desc_sw(sb + s * 32, 8 * O::VROW, O::VSW), id_b,
                                       !(k == kb && c == a.c0 && s == 0));
                            tc::commit(&B->empty[slot]);
                            if (++slot == nst) { slot = 0; pass ^= 1u; }
                        }
                        tc::commit(&B->vp_empty[b]);
                    }
                }
                if (ok) tc::commit(&B->out_full);
                g0 += (uint32_t)(ke - kb);
            }
            // every MMA issued by this thread has completed before the CTA leaves
            tc::commit(&B->drain);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(&B->drain, 0) && global_ns() - t0 < kWaitLimitNs) {}
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue warps 0-7
        const int q = warp & 3, h = warp >> 2;
        const int r = q * 32 + lane;            // element row of the tile = TMEM lane
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        uint32_t ntile = 0, g0 = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++ntile) {
            int kb, ke;
            chunk_range(w, kb, ke);
            const int64_t tile = w / a.nsplit, e = tile * 128 + r;
            const bool valid = e < a.n_elem;
            // U row r (this thread: half h of it): coefficients, TF32, zero padded to KP
            {
                const float* src = valid ? a.in + a.coeff_off[e] : nullptr;
                const int half = a.KP / 2;
                constexpr int KC = 16 / ES;                   // modes per 16-byte chunk
                for (int m0 = h * half; m0 < (h + 1) * half; m0 += KC) {
                    float x[KC];
#pragma unroll
                    for (int i = 0; i < KC; ++i) x[i] = (valid && m0 + i < a.NP) ? src[m0 + i] : 0.f;
                    *reinterpret_cast<uint4*>(sU + (m0 / O::KR) * 128 * 128 + O::off128(r, m0 % O::KR)) = O::pack(x);
                }
            }
            tc::fence_async_smem();
            arrive(&B->u_full);
            // metric factors of a chunk: this thread's 8 points of each factor are
            // 32 contiguous bytes of the tile-major layout; the next chunk's are
            // fetched while the current one is processed
            float Gn[7][kHalf], Gc[7][kHalf];
            auto load_geom = [&](int k) {
                const float4* gt = reinterpret_cast<const float4*>(
                    a.geom + (((tile * a.nch + k) * 7) * 128 + r) * (int64_t)kNPT + h * kHalf);
#pragma unroll
                for (int f = 0; f < 7; ++f) {
                    float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
                    if (f == 6 || a.c1 > 1) {
                        x0 = __ldg(gt + f * 128 * kNPT / 4);
                        x1 = __ldg(gt + f * 128 * kNPT / 4 + 1);
                    }
                    Gn[f][0] = x0.x; Gn[f][1] = x0.y; Gn[f][2] = x0.z; Gn[f][3] = x0.w;
                    Gn[f][4] = x1.x; Gn[f][5] = x1.y; Gn[f][6] = x1.z; Gn[f][7] = x1.w;
                }
            };
            if (kb < ke) load_geom(kb);
            for (int k = kb; k < ke && ok; ++k) {
                const uint32_t g = g0 + (uint32_t)(k - kb), b = g & 1u, use = g >> 1;
                const uint32_t bf = g % kFwdBufs, usef = g / kFwdBufs;     // forward accumulator buffer
#pragma unroll
                for (int f = 0; f < 7; ++f)
#pragma unroll
                    for (int p = 0; p < kHalf; ++p) Gc[f][p] = Gn[f][p];
                if (k + 1 < ke) load_geom(k + 1);
                if (!wait_warp(&B->fwd_full[bf], usef & 1u, B, a.err)) { ok = false; break; }
                tc::fence_after();
                float v[4][kHalf];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c >= a.c0 && c < a.c1) tc::ld_32x8(tbase + lane_base + (uint32_t)((bf * 4 + c) * kNPT + h * kHalf), v[c]);
                    else {
#pragma unroll
                        for (int p = 0; p < kHalf; ++p) v[c][p] = 0.f;
                    }
                }
                tc::fence_before();
                arrive(&B->fwd_empty[bf]);
                float o[4][kHalf];
#pragma unroll
                for (int p = 0; p < kHalf; ++p) {
                    // padded points and elements hold zeros in the tile-major layout
                    float G[6];
#pragma unroll
                    for (int f = 0; f < 6; ++f) G[f] = Gc[f][p];
                    const float wJ = Gc[6][p];
                    const float v1 = v[1][p], v2 = v[2][p], v3 = v[3][p];
                    o[0][p] = (a.op == HP_MASS ? 1.f : a.lambda) * wJ * v[0][p];
                    o[1][p] = G[0] * v1 + G[1] * v2 + G[2] * v3;
                    o[2][p] = G[1] * v1 + G[3] * v2 + G[4] * v3;
                    o[3][p] = G[2] * v1 + G[4] * v2 + G[5] * v3;
                }
                // the V' tile b is free once the backward MMAs that last read it completed
                if (!wait_warp(&B->vp_empty[b], (use & 1u) ^ 1u, B, a.err)) { ok = false; break; }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c < a.c0 || c >= a.c1) continue;
                    unsigned char* dst = sV + (size_t)(b * 4 + c) * O::VBYTES;
#pragma unroll
                    for (int p0 = 0; p0 < kHalf; p0 += 16 / ES)
                        *reinterpret_cast<uint4*>(dst + O::offv(r, h * kHalf + p0)) = O::pack(&o[c][p0]);
                }
                tc::fence_async_smem();
                arrive(&B->vp_full[b]);
            }
            if (!ok) break;
            g0 += (uint32_t)(ke - kb);
            // outputs: row r of the accumulator = element e, columns = modes (half h of them)
            if (!wait_warp(&B->out_full, ntile & 1u, B, a.err)) { ok = false; break; }
            tc::fence_after();
            float* dst = valid ? a.out + a.coeff_off[e] : nullptr;
            const int nh = a.NPpad / 2;
            for (int c0 = h * nh; c0 < (h + 1) * nh; c0 += 8) {
                float v[8];
                tc::ld_32x8(tbase + lane_base + (uint32_t)(kOutCol + c0), v);
                if (valid) {
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (c0 + j < a.NP) {
                            if (a.nsplit > 1) atomicAdd(dst + c0 + j, v[j]);
                            else dst[c0 + j] = v[j];
                        }
                }
            }
            tc::fence_before();
            arrive(&B->out_empty);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, kTmemCols);
}

// zero the block's output coefficients (the parts of a tile add into them)
__global__ void zero_coeffs_kernel(float* out, const int64_t* coeff_off, int64_t n_elem, int NP) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_elem * NP) return;
    const int64_t e = i / NP;
    out[coeff_off[e] + (i - e * NP)] = 0.f;
}

// FP64 curved geometry [n][7][NQp] -> FP32 tile-major [tile][chunk][7][128 elem][16 pts],
// zeros at padded points and elements
__global__ void tc_geom_kernel(const double* g, float* out, int64_t n_elem, int NQ, int NQp, int nch) {
    const int64_t ntiles = (n_elem + 127) / 128;
    const int64_t total = ntiles * nch * 7 * kNPT * 128;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i % kNPT);
        int64_t t = i / kNPT;
        const int r = (int)(t & 127);
        t >>= 7;
        const int f = (int)(t % 7);
        t /= 7;
        const int k = (int)(t % nch);
        const int64_t tile = t / nch, e = tile * 128 + r;
        const int l = k * kNPT + p;
        out[i] = (e < n_elem && l < NQ) ? (float)g[(e * 7 + f) * (int64_t)NQp + l] : 0.f;
    }
}

// Affine elements: the factors at every point from the element record [16]
// (|J| J^-1 J^-T, |J|, J^-1) and d eta / d xi at the point, in FP64, stored in
// the same tile-major FP32 layout as the curved factors.
template <int SHAPE>
__global__ void tc_geom_affine_kernel(const double* rec, const double* z, const double* w, int Q, float* out,
                                      int64_t n_elem, int nch) {
    const int NQ = Q * Q * Q, QQ = Q * Q;
    const int64_t ntiles = (n_elem + 127) / 128;
    const int64_t total = ntiles * nch * kNPT * 128;          // one thread per (tile, chunk, element, point)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = (int)(i % kNPT);
        int64_t t = i / kNPT;
        const int r = (int)(t & 127);
        t >>= 7;
        const int k = (int)(t % nch);
        const int64_t tile = t / nch, e = tile * 128 + r;
        const int l = k * kNPT + p;
        double G[7] = {0, 0, 0, 0, 0, 0, 0};
        if (e < n_elem && l < NQ) {
            const int ii = l / QQ, jj = (l / Q) % Q, kk = l % Q;
            double Tm[3][3];
            deta_dxi<SHAPE, double>(z[ii], z[Q + jj], z[2 * Q + kk], Tm);
            const double wl = w[ii] * w[Q + jj] * w[2 * Q + kk];
            const double* R = rec + e * 16;
            const double Km[3][3] = {{R[0], R[1], R[2]}, {R[1], R[3], R[4]}, {R[2], R[4], R[5]}};
            double M[3][3];
            for (int d = 0; d < 3; ++d)
                for (int j = 0; j < 3; ++j) M[d][j] = Tm[d][0] * Km[0][j] + Tm[d][1] * Km[1][j] + Tm[d][2] * Km[2][j];
            auto gg = [&](int d, int d2) { return wl * (M[d][0] * Tm[d2][0] + M[d][1] * Tm[d2][1] + M[d][2] * Tm[d2][2]); };
            G[0] = gg(0, 0); G[1] = gg(0, 1); G[2] = gg(0, 2); G[3] = gg(1, 1); G[4] = gg(1, 2); G[5] = gg(2, 2);
            G[6] = wl * R[6];
        }
        for (int f = 0; f < 7; ++f) out[(((tile * nch + k) * 7 + f) * 128 + r) * (int64_t)kNPT + p] = (float)G[f];
    }
}

}  // namespace

int tc_stages(int KP, int stage_bytes, int es) {
    const int base = 2048 + 128 * KP * es + 8 * 128 * kNPT * es;      // alignment slack + barriers + U + V'
    for (int st = kMaxStages; st >= 2; --st)
        if (base + st * stage_bytes <= 227 * 1024) return st;
    return 0;
}

int tc_smem_bytes(int KP, int stage_bytes, int es) {
    int b = 2048 + 128 * KP * es + 8 * 128 * kNPT * es + tc_stages(KP, stage_bytes, es) * stage_bytes;
    return b < 116 * 1024 ? 116 * 1024 : b;    // at most one CTA (and one TMEM allocation) per SM
}

int tc_chunk_points() { return kNPT; }

int64_t tc_geom_floats(int64_t n_elem, int nch) { return (n_elem + 127) / 128 * nch * 7 * kNPT * 128; }

cudaError_t tc_geom_layout(const double* g, float* out, int64_t n_elem, int NQ, int NQp, int nch, cudaStream_t s) {
    tc_geom_kernel<<<1024, 256, 0, s>>>(g, out, n_elem, NQ, NQp, nch);
    return cudaGetLastError();
}

cudaError_t tc_geom_layout_affine(int shape, const double* rec, const double* z, const double* w, int Q, float* out,
                                  int64_t n_elem, int nch, cudaStream_t s) {
    switch (shape) {
        case HP_HEX: tc_geom_affine_kernel<HP_HEX><<<1024, 256, 0, s>>>(rec, z, w, Q, out, n_elem, nch); break;
        case HP_PRISM: tc_geom_affine_kernel<HP_PRISM><<<1024, 256, 0, s>>>(rec, z, w, Q, out, n_elem, nch); break;
        case HP_PYR: tc_geom_affine_kernel<HP_PYR><<<1024, 256, 0, s>>>(rec, z, w, Q, out, n_elem, nch); break;
        default: tc_geom_affine_kernel<HP_TET><<<1024, 256, 0, s>>>(rec, z, w, Q, out, n_elem, nch); break;
    }
    return cudaGetLastError();
}

cudaError_t tc_emat_launch(const TCArgs& a, cudaStream_t s) {
    const int64_t ntiles = (a.n_elem + 127) / 128;
    if (ntiles <= 0) return cudaSuccess;
    TCArgs b = a;
    b.stages = tc_stages(a.KP, a.stage_bytes, a.es);
    // BF16 holds a chunk's stage until its backward MMAs, kFwdBufs - 1 chunks later
    if (b.stages < (a.es == 2 ? kFwdBufs + 1 : 2)) return cudaErrorInvalidValue;
    const int smem = tc_smem_bytes(a.KP, a.stage_bytes, a.es);
    auto kern = a.es == 2 ? tc_emat_kernel<2> : tc_emat_kernel<4>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // split the point chunks of a tile over CTAs until the grid covers the SMs
    // (at least 4 chunks per part)
    int64_t ns = (sms + ntiles - 1) / ntiles;
    const int64_t cap = a.nch / 4 > 1 ? a.nch / 4 : 1;
    b.nsplit = (int)(ns < cap ? ns : cap);
    if (b.nsplit > 1) {
        const int64_t n = a.n_elem * a.NP;
        zero_coeffs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.out, a.coeff_off, a.n_elem, a.NP);
    }
    const int64_t nwork = ntiles * b.nsplit;
    const int grid = (int)(nwork < sms ? nwork : sms);
    kern<<<grid, kThreads, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace hp
