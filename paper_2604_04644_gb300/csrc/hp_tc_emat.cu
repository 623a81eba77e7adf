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
// overlaps the backward MMAs of chunk k-1 (the BF16 blocks of 257..320 modes:
// two accumulators and one V' tile, so that their larger stages fit).
// Roles: warps 0..EW-1 gather U, run the metric and write the outputs (warp
// w reads TMEM lanes 32 (w mod 4).. and points kPts (w / 4).. of each chunk;
// EW = 16, one CTA per SM: four warps per lane quarter, 4 points each, so each
// scheduler holds four of them to hide the tensor-memory and factor loads;
// EW = 8, two CTAs per SM for BF16 blocks of at most 64 modes: two pipelines
// per SM overlap their hand-offs); warp EW issues the bulk copies; warp EW + 1
// issues the MMAs.  Every wait is
// bounded; a timeout latches DERR_TIMEOUT, stops every role, drains the
// copies and MMAs in flight and frees the tensor memory before the CTA exits.
#include <algorithm>
#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>

#include "hp_tc.cuh"

namespace hp {
namespace {

constexpr int kNPT = 16;          // quadrature points per chunk
constexpr int kMaxStages = 16;    // bulk-copy ring: as many stages (2..16) as fit in shared memory
constexpr int kFwdBufs = 3;       // forward accumulators in flight: the forward MMAs run two chunks ahead
constexpr int kOutCol = kFwdBufs * 4 * 16;   // TMEM column of the output accumulator (three forward buffers)
constexpr int kOutColMax = 512 - kOutCol;    // output columns beside the forward accumulators
constexpr int kSliceBytes = 4 * kNPT * 128;   // forward operand slice: 64 rows x 128 bytes of modes
// metric-factor layout: runs of kGeoPts points, kGeoGroups runs per chunk
constexpr int kGeoGroups = 4, kGeoPts = kNPT / kGeoGroups;

// Epilogue shape: EW epilogue warps, EW / 4 per TMEM lane quarter, each thread
// taking kPts points of a chunk.  EW = 16: one CTA per SM holding all 512 TMEM
// columns; EW = 8: two CTAs per SM with 256 columns each (blocks of at most 64
// modes, whose output accumulator fits beside the forward ones), so that two
// MMA / epilogue pipelines overlap their hand-offs on one SM.
template <int EW>
struct Epi {
    static constexpr int kGroups = EW / 4;
    static constexpr int kPts = kNPT / kGroups;      // points of a chunk per epilogue thread
    static constexpr int kRows = 128 / EW;           // tile rows per warp (coefficient gather and output)
    static constexpr int kEpi = 32 * EW;             // epilogue threads
    static constexpr int kThreads = kEpi + 64;       // + the producer warp and the MMA warp
    static constexpr int kCtas = EW == 16 ? 1 : 2;   // CTAs per SM
    static constexpr int kTmemCols = 512 / kCtas;
};

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
    // issued by a whole converged warp (one elected lane issues)
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        if constexpr (ES == 4) tc::mma_tf32_w(d, a, b, id, acc);
        else tc::mma_bf16_w(d, a, b, id, acc);
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
    // NPTS consecutive points p.. of row r of a 16-point tile
    template <int NPTS>
    __device__ static void put_pts(unsigned char* tile, uint32_t r, uint32_t p, const float* x) {
        if constexpr (ES * NPTS >= 16) {
#pragma unroll
            for (int p0 = 0; p0 < NPTS; p0 += 16 / ES) *reinterpret_cast<uint4*>(tile + offv(r, p + p0)) = pack(x + p0);
        } else {      // BF16, 4 points: the half of a 16-byte chunk at (p mod 8) * 2
            const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]), h1 = __floats2bfloat162_rn(x[2], x[3]);
            *reinterpret_cast<uint2*>(tile + offv(r, p) + (p & 7) * 2) =
                make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
        }
    }
    // one operand element
    __device__ static void put(unsigned char* p, float x) {
        if constexpr (ES == 4) *reinterpret_cast<float*>(p) = tc::to_tf32(x);
        else *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(x);
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

// position in a ring of n buffers and the parity of its current pass
struct Ring {
    uint32_t n, i = 0, ph = 0;
    __device__ void next() {
        if (++i == n) { i = 0; ph ^= 1u; }
    }
};

// 8 bytes of the metric-factor stream: read once, so not kept in L1 (whose
// storage shares the SM's shared-memory banks with the operand tiles)
__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
// an epilogue thread's NP FP16 metric factors of one factor: 8 bytes (4 points) or 16 (8 points)
template <int NP>
using GVt = std::conditional_t<NP == 8, uint4, uint2>;
__device__ __forceinline__ uint32_t gv_word(const uint4& g, int i) { return i == 0 ? g.x : i == 1 ? g.y : i == 2 ? g.z : g.w; }
__device__ __forceinline__ uint32_t gv_word(const uint2& g, int i) { return i == 0 ? g.x : g.y; }

struct Bars {
    uint64_t full[kMaxStages], empty[kMaxStages];
    uint64_t epi;                      // the epilogue warps among themselves
    uint64_t u_full[2], fwd_full[kFwdBufs], fwd_empty[kFwdBufs], vp_full[2], vp_empty[2], out_full, out_empty, drain;
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(Bars) <= 1024, "the barriers sit in the first kilobyte of shared memory");

// wait for `parity` of `bar`, giving up when another role aborted or after the
// time limit (then this role aborts every role)
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, Bars* B, unsigned int* err) {
    if (mbar_try_wait(bar, parity)) return true;        // the common case reads no timer
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
// one arrival for the whole warp: every lane's earlier writes (and fences) are
// ordered before lane 0's arrival by the warp barrier
__device__ __forceinline__ void arrive_warp(uint64_t* bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) arrive(bar);
}


// VAR (BF16 only): 0 the default (kFwdBufs forward accumulators, two V' tiles,
// the backward reading each chunk's forward stage); 2 the lean form for blocks
// of 257..320 modes, whose forward stages are too large to hold kFwdBufs - 1
// chunks: two forward accumulators and one V' tile, so that the stages of two
// chunks fit beside U (the output, N_P > 256, takes two backward MMAs of N =
// 256 and 64, and is staged through U's buffer); 1 streams the backward tiles
// R_c like TF32 (the mode parts past 320 modes)
template <int ES, int EW, int VAR = 0>
__global__ void __launch_bounds__(Epi<EW>::kThreads, Epi<EW>::kCtas) tc_emat_kernel(const __grid_constant__ TCArgs a) {
    using O = Op<ES>;
    using E = Epi<EW>;
    constexpr bool SB = VAR == 1;
    constexpr bool kReuse = ES == 2 && !SB;   // the backward reads the forward stage (MN-major)
    constexpr int kFB = VAR == 2 ? 2 : kFwdBufs;     // forward accumulators in flight
    constexpr int kVB = VAR == 2 ? 1 : 2;            // V' tiles
    constexpr int kOC = kFB * 4 * kNPT;              // TMEM column of the output accumulator
    static_assert(kOC + (VAR == 2 ? 320 : 256) <= 512, "output accumulator beside the forward ones");
    constexpr int kGroups = E::kGroups, kPts = E::kPts, kRows = E::kRows;
    using GV = GVt<kPts>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the swizzle patterns are taken from shared-memory address bits: align to 1 KB
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    Bars* B = reinterpret_cast<Bars*>(smem);
    unsigned char* sU = smem + 1024;                                   // [ubufs][KP / KR][128 x 128 B], 128 B swizzle
    unsigned char* sV = sU + a.ubufs * 128 * a.KP * ES;                // [2][4][128 x 16], 64 / 32 B swizzle
    unsigned char* sR = sV + kVB * 4 * O::VBYTES;                      // ring
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nst = a.stages;
    // work items: (tile of 128 elements, part of its point chunks, range of
    // output modes); chunk parts of one tile add their partial outputs (the
    // output was zeroed first), mode parts write disjoint modes (BF16 past 320
    // modes: each recomputes the forward and the metric of its chunks)
    const int64_t per_tile = (int64_t)a.nsplit * a.nmpart;
    const int64_t nwork = (a.n_elem + 127) / 128 * per_tile;
    auto wtile = [&](int64_t w) { return w / per_tile; };
    auto wpart = [&](int64_t w) { return (int)((w % per_tile) % a.nsplit); };
    auto wmode0 = [&](int64_t w) { return (int)((w % per_tile) / a.nsplit) * a.mwidth; };
    auto chunk_range = [&](int64_t w, int& kb, int& ke) {
        const int part = wpart(w);
        kb = (int)((int64_t)a.nch * part / a.nsplit);
        ke = (int)((int64_t)a.nch * (part + 1) / a.nsplit);
    };

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) { mbar_init(&B->full[s], 1); mbar_init(&B->empty[s], 1); }
        for (int j = 0; j < 2; ++j) mbar_init(&B->u_full[j], EW);
        for (int b = 0; b < kFB; ++b) {
            mbar_init(&B->fwd_full[b], 1);
            mbar_init(&B->fwd_empty[b], EW);
        }
        for (int b = 0; b < kVB; ++b) {
            mbar_init(&B->vp_full[b], EW);
            mbar_init(&B->vp_empty[b], 1);
        }
        mbar_init(&B->out_full, 1);
        mbar_init(&B->out_empty, EW);
        mbar_init(&B->drain, 1);
        mbar_init(&B->epi, EW);
        B->abort = 0;
    }
    if (warp == 0) { tc::tmem_alloc(&B->tmem, E::kTmemCols); tc::tmem_relinquish(); }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = B->tmem;

    if (warp == EW) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int slot = 0;
            uint32_t pass = 0;
            uint32_t last_parity = 0, used = 0;     // bit s: stage s's last pass, whether it was filled
            bool ok = true;
            auto put = [&](const unsigned char* src, uint32_t bytes) {
                if (!wait_bar(&B->empty[slot], pass ^ 1u, B, a.err)) { ok = false; return; }
                mbar_expect_tx(&B->full[slot], bytes);
                bulk_g2s(sR + (size_t)slot * a.stage_bytes, src, bytes, &B->full[slot]);
                used |= 1u << slot;
                last_parity = (last_parity & ~(1u << slot)) | (pass << slot);
                if (++slot == nst) { slot = 0; pass ^= 1u; }
            };
            for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
                int kb, ke;
                chunk_range(w, kb, ke);
                // the MMA issuer's order: forward of chunk t, backward of chunk t - (kFB - 1);
                // BF16: one stage per chunk (all forward slices), read again by the backward
                if constexpr (kReuse) {
                    for (int t = kb; t < ke && ok; ++t) put(a.img + (size_t)t * a.chunk_bytes, (uint32_t)a.fwd_bytes);
                    continue;
                }
                for (int t = kb; t < ke + kFB - 1 && ok; ++t) {
                    if (t < ke) {
                        const unsigned char* base = a.img + (size_t)t * a.chunk_bytes;
                        for (int sl = 0; sl * O::KR < a.KP && ok; ++sl) put(base + (size_t)sl * kSliceBytes, kSliceBytes);
                    }
                    const int kbw = t - (kFB - 1);
                    if (kbw >= kb) {
                        const unsigned char* base = a.img + (size_t)kbw * a.chunk_bytes + (size_t)a.fwd_bytes;
                        for (int c = a.c0; c < a.c1 && ok; ++c) put(base + (size_t)c * a.bwd_bytes, a.bwd_bytes);
                    }
                }
            }
            // no copy may still be landing when the CTA leaves
            for (int s = 0; s < nst; ++s)
                if ((used >> s) & 1u) {
                    const uint64_t t0 = global_ns();
                    while (!mbar_try_wait(&B->full[s], (last_parity >> s) & 1u) && global_ns() - t0 < kWaitLimitNs) {}
                }
        }
        __syncwarp();
    } else if (warp == EW + 1) {
        // ---------------------------------------------------------------- MMA issuer
        // the whole warp runs the loop (its waits warp-wide, so every decision
        // is uniform) and one elected lane issues each MMA and commit
        {
            const uint32_t id_f = tc::instr_desc(O::FMT, 128, kNPT * (a.c1 - a.c0));
            // BF16 backward from the forward stage (B operand MN-major): N = N_P, or
            // past 256 modes N = 256 and then 64 (the fifth 64-mode atom, zero past N_P)
            const uint32_t id_bt = tc::instr_desc(O::FMT, 128, a.NPpad > 256 ? 256 : a.NPpad) | (1u << 16);
            const uint32_t id_bt1 = tc::instr_desc(O::FMT, 128, 64) | (1u << 16);
            // streamed backward: a work item's output modes m0 .. m0 + mw - 1, as
            // N = min(mw, 256) then N = mw - 256, reading the tile from its row m0
            // (and m0 + 256) on (K-major rows of VROW bytes)
            constexpr uint32_t kHalf16 = (256 * O::VROW) >> 4;
            // descriptors are built once: an operand x bytes past a base adds x / 16
            // to the start-address field (shared addresses stay below 256 KB, so
            // the 14-bit field never carries)
            const uint64_t dU = tc::smem_desc_sw(smem_addr(sU), 1024, tc::kSw128);
            const uint64_t dF = tc::smem_desc_sw(smem_addr(sR) + a.c0 * 2 * 1024, 1024, tc::kSw128);
            const uint64_t dV = tc::smem_desc_sw(smem_addr(sV), 8 * O::VROW, O::VSW);
            // BF16 backward: the chunk's stage read MN-major (N = modes: 64-mode atoms
            // one slice apart, LBO; K = the component's 16 points, 8-point groups 1 KB
            // apart, SBO); TF32 backward: streamed K-major tiles
            const uint64_t dRt = tc::smem_desc_sw_lbo(smem_addr(sR), kSliceBytes, 1024, tc::kSw128);
            const uint64_t dRb = tc::smem_desc_sw(smem_addr(sR), 8 * O::VROW, O::VSW);
            const uint32_t nsl = (uint32_t)((a.KP + O::KR - 1) / O::KR);
            const uint32_t st16 = (uint32_t)a.stage_bytes >> 4, u16 = (uint32_t)(128 * a.KP * ES) >> 4;
            constexpr uint32_t v16 = O::VBYTES >> 4, sl16 = kSliceBytes >> 4;
            // fb: forward accumulators, vb: V' tiles, fs / bs: ring stages taken by
            // the forward / released by the backward (BF16), ub: U buffers
            Ring fb{kFB}, vb{kVB}, fs{(uint32_t)nst}, bs{(uint32_t)nst}, ub{(uint32_t)a.ubufs};
            uint32_t nout = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
                int kb, ke;
                chunk_range(w, kb, ke);
                const uint32_t m0w = (uint32_t)wmode0(w), mww = (uint32_t)min(a.mwidth, a.NPpad - (int)m0w);
                const uint32_t nb0 = mww > 256 ? 256u : mww, nb1 = mww - nb0;
                const uint32_t id_b0 = tc::instr_desc(O::FMT, 128, nb0), id_b1 = tc::instr_desc(O::FMT, 128, nb1 > 0 ? nb1 : 16);
                const uint32_t mo16 = (m0w * O::VROW) >> 4;
                if (!wait_warp(&B->u_full[ub.i], ub.ph, B, a.err)) { ok = false; break; }
                const uint64_t dUw = dU + ub.i * u16;
                ub.next();
                // forward of chunk t, then backward of chunk t - (kFB - 1)
                for (int t = kb; t < ke + kFB - 1 && ok; ++t) {
                    if (t < ke) {
                        if (!wait_warp(&B->fwd_empty[fb.i], fb.ph ^ 1u, B, a.err)) { ok = false; break; }
                        // columns (fb*4 + c0)*16 .. of the accumulator = components c0..c1-1
                        const uint32_t d = tbase + (fb.i * 4 + (uint32_t)a.c0) * kNPT;
                        if constexpr (kReuse) {
                            // one ring stage per chunk holding every K slice
                            if (!wait_warp(&B->full[fs.i], fs.ph, B, a.err)) { ok = false; break; }
                            tc::fence_after();
                            const uint64_t dFs = dF + fs.i * st16;
                            for (uint32_t sl = 0; sl < nsl; ++sl)
#pragma unroll
                                for (uint32_t s = 0; s < 4; ++s)
                                    O::mma(d, dUw + (sl * 1024 + s * 2), dFs + (sl * sl16 + s * 2), id_f, sl > 0 || s > 0);
                            fs.next();
                        } else {
                            // one ring stage per K slice, released as soon as it is read
                            for (uint32_t sl = 0; sl < nsl && ok; ++sl) {
                                if (!wait_warp(&B->full[fs.i], fs.ph, B, a.err)) { ok = false; break; }
                                tc::fence_after();
                                const uint64_t dFs = dF + fs.i * st16;
#pragma unroll
                                for (uint32_t s = 0; s < 4; ++s)
                                    O::mma(d, dUw + (sl * 1024 + s * 2), dFs + s * 2, id_f, sl > 0 || s > 0);
                                tc::commit_w(&B->empty[fs.i]);
                                fs.next();
                            }
                            if (!ok) break;
                        }
                        tc::commit_w(&B->fwd_full[fb.i]);
                        fb.next();
                    }
                    const int k = t - (kFB - 1);
                    if (k >= kb) {
                        if (!wait_warp(&B->vp_full[vb.i], vb.ph, B, a.err)) { ok = false; break; }
                        if (k == kb) {
                            if (!wait_warp(&B->out_empty, (nout & 1u) ^ 1u, B, a.err)) { ok = false; break; }
                            ++nout;
                        }
                        tc::fence_after();
                        const uint64_t dVb = dV + vb.i * 4 * v16;
                        if constexpr (kReuse) {
                            const uint64_t dRs = dRt + bs.i * st16;
                            for (int c = a.c0; c < a.c1; ++c) {
                                const uint32_t acc = !(k == kb && c == a.c0);
                                O::mma(tbase + kOC, dVb + (uint32_t)c * v16, dRs + (uint32_t)c * 128, id_bt, acc);
                                if (a.NPpad > 256)
                                    O::mma(tbase + kOC + 256, dVb + (uint32_t)c * v16, dRs + (uint32_t)c * 128 + 4 * sl16,
                                           id_bt1, acc);
                            }
                            tc::commit_w(&B->empty[bs.i]);
                            bs.next();
                        } else {
                            for (int c = a.c0; c < a.c1 && ok; ++c) {
                                if (!wait_warp(&B->full[fs.i], fs.ph, B, a.err)) { ok = false; break; }
                                tc::fence_after();
                                const uint64_t dRs = dRb + fs.i * st16 + mo16;
#pragma unroll
                                for (uint32_t s = 0; s < O::VROW / 32; ++s) {
                                    const uint32_t acc = !(k == kb && c == a.c0 && s == 0);
                                    O::mma(tbase + kOC, dVb + (uint32_t)c * v16 + s * 2, dRs + s * 2, id_b0, acc);
                                    if (nb1 > 0)
                                        O::mma(tbase + kOC + 256, dVb + (uint32_t)c * v16 + s * 2, dRs + kHalf16 + s * 2,
                                               id_b1, acc);
                                }
                                tc::commit_w(&B->empty[fs.i]);
                                fs.next();
                            }
                            if (!ok) break;
                        }
                        tc::commit_w(&B->vp_empty[vb.i]);
                        vb.next();
                    }
                }
                if (ok) tc::commit_w(&B->out_full);
            }
            // every MMA issued by this warp has completed before the CTA leaves
            tc::commit_w(&B->drain);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(&B->drain, 0) && global_ns() - t0 < kWaitLimitNs) {}
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue warps
        // warp w reads TMEM lane quarter q = w mod 4 and points h kPts .. of each chunk
        const int q = warp & 3, h = warp >> 2;
        const int r = q * 32 + lane;            // element row of the tile = TMEM lane
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        constexpr uint32_t kAll = 0xffffffffu;
        // coefficient offsets of rows kRows warp .. of work item wi's tile: lane
        // i < kRows holds row kRows warp + i's (-1 past the last element)
        auto row_offsets = [&](int64_t wi) -> int64_t {
            const int64_t e = wtile(wi) * 128 + warp * kRows + lane;
            return (lane < kRows && e < a.n_elem) ? a.coeff_off[e] : (int64_t)-1;
        };
        // U of a tile into buffer j, coalesced: each warp copies the coefficient
        // rows of its kRows elements (offsets `offs`, lanes along the modes; RB
        // rows of up to 32 JJ modes with all their loads in flight at a time),
        // rounded to the operand type and zero padded to KP
        auto gather_rows = [&](auto RBc, auto JJc, unsigned char* dU, int64_t offs) {
            constexpr int RB = decltype(RBc)::value, JJ = decltype(JJc)::value;
            for (int i0 = 0; i0 < kRows; i0 += RB) {
                float x[RB][JJ];
#pragma unroll
                for (int ii = 0; ii < RB; ++ii) {
                    const int64_t off = __shfl_sync(kAll, offs, i0 + ii);
#pragma unroll
                    for (int jj = 0; jj < JJ; ++jj) {
                        const int m = lane + 32 * jj;
                        x[ii][jj] = (off >= 0 && m < a.NP) ? __ldg(a.in + off + m) : 0.f;
                    }
                }
#pragma unroll
                for (int ii = 0; ii < RB; ++ii) {
                    const int row = warp * kRows + i0 + ii;
#pragma unroll
                    for (int jj = 0; jj < JJ; ++jj) {
                        const int m = lane + 32 * jj;
                        if (32 * jj < a.KP) O::put(dU + (m / O::KR) * 128 * 128 + O::off128(row, m % O::KR), x[ii][jj]);
                    }
                }
            }
        };
        auto gather_u = [&](int j, int64_t offs) {
            unsigned char* dU = sU + (size_t)j * 128 * a.KP * ES;
            if (a.KP <= 128) gather_rows(std::integral_constant<int, 8>{}, std::integral_constant<int, 4>{}, dU, offs);
            else if (a.KP <= 256) gather_rows(std::integral_constant<int, 4>{}, std::integral_constant<int, 8>{}, dU, offs);
            else if constexpr (ES == 2) {      // past 256 modes (BF16 only)
                if (a.KP <= 320) gather_rows(std::integral_constant<int, 4>{}, std::integral_constant<int, 10>{}, dU, offs);
                else gather_rows(std::integral_constant<int, 1>{}, std::integral_constant<int, kTcMaxModes16 / 32>{}, dU, offs);
            }
            tc::fence_async_smem();
            arrive_warp(&B->u_full[j]);
        };
        // barrier of the epilogue warps alone, bounded like every other wait (a
        // warp that left after a timeout never arrives; the others see the abort)
        uint32_t nepi = 0;
        auto epi_sync = [&]() -> bool {
            arrive_warp(&B->epi);
            return wait_warp(&B->epi, (nepi++) & 1u, B, a.err);
        };
        const float lam = a.op == HP_MASS ? 1.f : a.lambda;
        uint32_t ntile = 0, g0 = 0;
        bool ok = true;
        // row offsets of the current work item, and of the next one fetched a tile ahead
        int64_t offs = blockIdx.x < nwork ? row_offsets(blockIdx.x) : (int64_t)-1;
        for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x, ++ntile) {
            int kb, ke;
            chunk_range(w, kb, ke);
            const int64_t tile = wtile(w);
            const int m0 = wmode0(w), mw = min(a.mwidth, a.NPpad - m0);   // this item's output modes
            const bool more = w + gridDim.x < nwork;
            const int64_t offs_next = more ? row_offsets(w + gridDim.x) : (int64_t)-1;
            // one U buffer: gathered once the previous tile's MMAs completed; two:
            // the next tile's U is gathered while this tile's last MMAs run
            if (a.ubufs == 1 || ntile == 0) gather_u(0, offs);
            // 2^-k of element r's FP16 Laplacian factors and of its w|J| (0: padding)
            const float2 isc2 = *reinterpret_cast<const float2*>(a.gscale + 2 * (tile * 128 + r));
            const float isc = isc2.x, iscm = isc2.y;
            // this thread's points h kPts.. are kPts / kGeoPts runs of the factor layout
            const uint2* gt = reinterpret_cast<const uint2*>(a.geom16) +
                              (tile * a.nch * 7 * kGeoGroups + h * (kPts / kGeoPts)) * 128 + r;
            // the seven factors of chunk k at this thread's kPts points (kPts halves each)
            auto load_geom = [&](int k, GV (&G)[7]) {
#pragma unroll
                for (int f = 0; f < 7; ++f) {
                    const uint2* q = gt + ((int64_t)k * 7 + f) * (kGeoGroups * 128);
                    const bool need = f == 6 || a.c1 > 1;
                    if constexpr (kPts == kGeoPts) {
                        G[f] = need ? ld_stream(q) : uint2{0u, 0u};
                    } else {
                        const uint2 lo = need ? ld_stream(q) : uint2{0u, 0u}, hi = need ? ld_stream(q + 128) : uint2{0u, 0u};
                        G[f] = make_uint4(lo.x, lo.y, hi.x, hi.y);
                    }
                }
            };
            // metric of chunk k: forward accumulator -> V' tile (components
            // outside [c0, c1) are computed from unused columns and discarded)
            // after_metric runs once the factors Gh are consumed (one-set rotation)
            auto process = [&](int k, GV (&Gh)[7], auto&& after_metric) -> bool {
                const uint32_t g = g0 + (uint32_t)(k - kb), b = g % kVB, use = g / kVB;
                const uint32_t bf = g % kFB, usef = g / kFB;     // forward accumulator buffer
                if (!wait_warp(&B->fwd_full[bf], usef & 1u, B, a.err)) return false;
                tc::fence_after();
                float v[4][kPts];
                tc::ld_x4(tbase + lane_base + (uint32_t)(bf * 4 * kNPT + h * kPts), kNPT, v);
                tc::fence_before();
                arrive_warp(&B->fwd_empty[bf]);
                float o[4][kPts];
#pragma unroll
                for (int p2 = 0; p2 < kPts / 2; ++p2) {
                    float2 G[7];
#pragma unroll
                    for (int f = 0; f < 7; ++f) {
                        const uint32_t wd = gv_word(Gh[f], p2);
                        G[f] = __half22float2(*reinterpret_cast<const __half2*>(&wd));
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int p = 2 * p2 + j;
                        auto gf = [&](int f) { return j ? G[f].y : G[f].x; };
                        const float v1 = v[1][p], v2 = v[2][p], v3 = v[3][p];
                        o[0][p] = lam * iscm * gf(6) * v[0][p];
                        o[1][p] = isc * (gf(0) * v1 + gf(1) * v2 + gf(2) * v3);
                        o[2][p] = isc * (gf(1) * v1 + gf(3) * v2 + gf(4) * v3);
                        o[3][p] = isc * (gf(2) * v1 + gf(4) * v2 + gf(5) * v3);
                    }
                }
                after_metric();
                // the V' tile b is free once the backward MMAs that last read it completed
                if (!wait_warp(&B->vp_empty[b], (use & 1u) ^ 1u, B, a.err)) return false;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c < a.c0 || c >= a.c1) continue;
                    O::template put_pts<kPts>(sV + (size_t)(b * 4 + c) * O::VBYTES, r, h * kPts, o[c]);
                }
                tc::fence_async_smem();
                arrive_warp(&B->vp_full[b]);
                return true;
            };
            auto none = [] {};
            if constexpr (EW == 8) {
                // one register set (two CTAs per SM leave 96 registers a thread): the
                // next chunk's factors are loaded as soon as the metric consumed these
                GV ga[7];
                if (kb < ke) load_geom(kb, ga);
                for (int k = kb; k < ke; ++k) {
                    if (!(ok = process(k, ga, [&] { if (k + 1 < ke) load_geom(k + 1, ga); }))) break;
                }
            } else if constexpr (ES == 2) {
                // factors one chunk ahead: two register sets in rotation (with
                // sixteen epilogue warps the shorter BF16 chunks hide the load,
                // and the registers saved avoid spills)
                GV ga[7], gb[7];
                if (kb < ke) load_geom(kb, ga);
                for (int k = kb; k < ke; k += 2) {
                    if (k + 1 < ke) load_geom(k + 1, gb);
                    if (!(ok = process(k, ga, none)) || k + 1 >= ke) break;
                    if (k + 2 < ke) load_geom(k + 2, ga);
                    if (!(ok = process(k + 1, gb, none))) break;
                }
            } else {
                // factors two chunks ahead: three register sets in rotation
                GV ga[7], gb[7], gc[7];
                if (kb < ke) load_geom(kb, ga);
                if (kb + 1 < ke) load_geom(kb + 1, gb);
                for (int k = kb; k < ke; k += 3) {
                    if (k + 2 < ke) load_geom(k + 2, gc);
                    if (!(ok = process(k, ga, none)) || k + 1 >= ke) break;
                    if (k + 3 < ke) load_geom(k + 3, ga);
                    if (!(ok = process(k + 1, gb, none)) || k + 2 >= ke) break;
                    if (k + 4 < ke) load_geom(k + 4, gb);
                    if (!(ok = process(k + 2, gc, none))) break;
                }
            }
            if (!ok) break;
            g0 += (uint32_t)(ke - kb);
            if (a.ubufs == 2 && more) gather_u((int)((ntile + 1) & 1u), offs_next);
            // outputs: row r of the accumulator = element r of the tile, columns =
            // modes; staged CB columns at a time through the V' tiles (free from
            // the tile's last backward MMA to the next tile's first V' write) so
            // that each warp stores whole coefficient rows (coalesced)
            if (!wait_warp(&B->out_full, ntile & 1u, B, a.err)) { ok = false; break; }
            tc::fence_after();
            // staged through the two V' tiles, or (one V' tile) through this
            // tile's U buffer, free once its MMAs completed (a next tile's U goes
            // into the other buffer, or is gathered after the output)
            float* stage = kVB == 2 ? reinterpret_cast<float*>(sV)
                                    : reinterpret_cast<float*>(sU + (size_t)(a.ubufs == 2 ? (ntile & 1u) : 0u) * 128 * a.KP * ES);
            constexpr int CB = 8 * O::VBYTES / (128 * 4);
            const int part = wpart(w);
            for (int cb = 0; cb < mw; cb += CB) {
                // row r, columns h CB / kGroups .. of the pass; 16-byte chunks XOR-swizzled by row
#pragma unroll
                for (int c = 0; c < CB / kGroups; c += 16) {
                    const int cc = h * (CB / kGroups) + c;
                    if (cb + cc < mw) {                  // warp-uniform; mw is a multiple of 16
                        float v[16];
                        tc::ld_32x16(tbase + lane_base + (uint32_t)(kOC + cb + cc), v);
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            *reinterpret_cast<float4*>(stage + r * CB + ((((cc + i) >> 2) ^ (r & 7)) << 2)) =
                                make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                    }
                }
                if (!(ok = epi_sync())) break;
                // every row and column of the pass unrolled, so that the loads and
                // the stores or atomics of different rows are in flight together
                // (one row at a time spent ~400 clocks a row waiting)
#pragma unroll
                for (int i = 0; i < kRows; ++i) {
                    const int64_t off = __shfl_sync(kAll, offs, i);
                    const int row = warp * kRows + i;
#pragma unroll
                    for (int j = 0; j < CB / 32; ++j) {
                        const int m = lane + 32 * j, mo = m0 + cb + m;
                        const float val = stage[row * CB + (((m >> 2) ^ (row & 7)) << 2) + (m & 3)];
                        if (off < 0 || cb + m >= mw || mo >= a.NP) continue;
                        if (a.nsplit == 1) a.out[off + mo] = val;
                        else if (a.part_out)   // fixed-order sum later: this part's own slot
                            a.part_out[((int64_t)part * a.n_elem + tile * 128 + row) * a.NP + mo] = val;
                        else atomicAdd(a.out + off + mo, val);
                    }
                }
                if (!(ok = epi_sync())) break;
            }
            if (!ok) break;
            tc::fence_before();
            arrive_warp(&B->out_empty);
            offs = offs_next;
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, E::kTmemCols);
}

// Hybrid strategy on the tensor cores: the two dense contractions with the
// reference basis, u = B uhat (MODE 0, modes -> points) and out = B^T u'
// (MODE 1, points -> modes), for tiles of 128 elements (the MMA's M, one
// element per TMEM lane), on component 0 (B) of the elemental-matrix image;
// the collocated derivatives and the metric between them run on the CUDA
// cores.  The point chunks of a tile are software pipelined: component 0's
// operand of chunk k (its 16 rows of every 128-byte K slice, packed 2 KB
// apart) is bulk-copied into stage k mod S of a ring S (2 or 3) deep, issued
// as soon as the MMA that read the stage's previous chunk has completed; the
// MMA of chunk k runs while MODE 0 stores chunk k-1's 16 point values per
// element from the other of two TMEM buffers, and while MODE 1 loads chunk
// k+1's point values into registers for the other of two V' tiles.  MODE 1
// accumulates all chunks into N_P columns (two MMAs of at most 256 columns
// each past 256 modes).  128 threads, warp 0 issuing (one elected lane); every wait bounded,
// and copies or MMAs still in flight after a timeout are waited for (bounded)
// before the CTA frees its tensor memory.
constexpr int kHybSlice = kNPT * 128;       // component 0 of one K slice: 16 rows x 128 bytes
constexpr int kHybMaxStages = 3;

struct HybBars {
    uint64_t full[kHybMaxStages], mma[2];
    uint32_t tmem;
};

template <int ES, int MODE>
__global__ void __launch_bounds__(128) tc_hyb_kernel(const __grid_constant__ HybArgs a) {
    using O = Op<ES>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    HybBars* B = reinterpret_cast<HybBars*>(smem);
    // MODE 0: U [KP / KR][128 x 128 B]; MODE 1: V' [2][128 x 16 points]; then the ring
    unsigned char* sOp = smem + 1024;
    const size_t op_bytes = MODE == 0 ? (size_t)128 * a.KP * ES : (size_t)2 * O::VBYTES;
    unsigned char* sSt = sOp + (op_bytes + 1023) / 1024 * 1024;
    const int S = a.stages;
    const uint32_t stb = (uint32_t)a.stage_bytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = MODE == 0 ? 32u : (a.NPpad > 256 ? 512u : 256u);
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&B->full[s], 1);
        mbar_init(&B->mma[0], 1);
        mbar_init(&B->mma[1], 1);
    }
    if (warp == 0) { tc::tmem_alloc(&B->tmem, ncols); tc::tmem_relinquish(); }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = B->tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    // barrier bookkeeping, identical in every thread: next phase, and whether a
    // copy (full) or an MMA group (mma) was issued and not yet waited for
    // (bit s of a mask per array, so that the bookkeeping stays in registers:
    // an array indexed by the stage would live in local memory)
    uint32_t ph_full = 0, ph_mma = 0, fl = 0, ml = 0;
    bool ok = true;
    auto wait_full = [&](int s) {
        const bool w = mbar_wait_bounded(&B->full[s], (ph_full >> s) & 1u, kWaitLimitNs);
        if (w) { ph_full ^= 1u << s; fl &= ~(1u << s); }
        else if (tid == 0) atomicOr(a.err, DERR_TIMEOUT);
        ok = (__syncthreads_and(w ? 1 : 0) != 0) && ok;
    };
    auto wait_mma = [&](int b) {
        const bool w = mbar_wait_bounded(&B->mma[b], (ph_mma >> b) & 1u, kWaitLimitNs);
        if (w) { ph_mma ^= 1u << b; ml &= ~(1u << b); }
        else if (tid == 0) atomicOr(a.err, DERR_TIMEOUT);
        ok = (__syncthreads_and(w ? 1 : 0) != 0) && ok;
    };
    const uint32_t nsl = (uint32_t)((a.KP + O::KR - 1) / O::KR);
    // copy of chunk k's operand into stage k mod S (thread 0 issues; all threads book it)
    auto issue = [&](int k) {
        const int s = k % S;
        if (tid == 0) {
            const unsigned char* src = a.img + (size_t)k * a.chunk_bytes;
            unsigned char* dst = sSt + (size_t)s * stb;
            if (MODE == 1 && ES == 4) {     // TF32 backward: component 0's tile R_0[mode][point]
                mbar_expect_tx(&B->full[s], (uint32_t)a.bwd_bytes);
                bulk_g2s(dst, src + a.fwd_bytes, (uint32_t)a.bwd_bytes, &B->full[s]);
            } else {
                mbar_expect_tx(&B->full[s], nsl * (uint32_t)kHybSlice);
                for (uint32_t sl = 0; sl < nsl; ++sl)
                    bulk_g2s(dst + sl * kHybSlice, src + (size_t)sl * kSliceBytes, kHybSlice, &B->full[s]);
            }
        }
        fl |= 1u << s;
    };
    const int64_t ntiles = (a.n_elem + 127) / 128;
    constexpr uint32_t hs16 = kHybSlice >> 4;
    const uint32_t st16 = stb >> 4;
    // MODE 0: A = U (K-major, 128-byte swizzle), B = the packed slices (K-major)
    const uint64_t dU = tc::smem_desc_sw(smem_addr(sOp), 1024, tc::kSw128);
    const uint64_t dF = tc::smem_desc_sw(smem_addr(sSt), 1024, tc::kSw128);
    // MODE 1: A = V' (K = the 16 points); B = BF16: the packed slices read MN-major
    // (64-mode atoms one packed slice apart, 8-point groups 1 KB apart);
    // TF32: the component's backward tile R_0[mode][point] (K-major)
    const uint64_t dV = tc::smem_desc_sw(smem_addr(sOp), 8 * O::VROW, O::VSW);
    const uint64_t dRt = tc::smem_desc_sw_lbo(smem_addr(sSt), kHybSlice, 1024, tc::kSw128);
    const uint64_t dRb = tc::smem_desc_sw(smem_addr(sSt), 8 * O::VROW, O::VSW);
    constexpr uint32_t v16 = O::VBYTES >> 4;
    const uint32_t id_f = tc::instr_desc(O::FMT, 128, kNPT);
    const uint32_t n0 = a.NPpad > 256 ? 256u : (uint32_t)a.NPpad, n1 = (uint32_t)a.NPpad - n0;
    // BF16 backward: B operand MN-major (bit 16 of the instruction descriptor)
    const uint32_t mn = ES == 2 ? (1u << 16) : 0u;
    const uint32_t id_b0 = tc::instr_desc(O::FMT, 128, n0) | mn, id_b1 = tc::instr_desc(O::FMT, 128, n1 > 0 ? n1 : 16) | mn;
    // start of modes 256.. in the backward operand (16-byte units)
    const uint32_t half16 = ES == 2 ? (256 / 64) * hs16 : (256 * O::VROW) >> 4;
    const int nch = a.nch, npre = nch < S ? nch : S;
    bool pre = false;               // the tile's first chunks were issued at the end of the previous tile
    float x[kNPT];                  // MODE 1: the next chunk's point values of this thread's element
    auto load_pts = [&](int64_t tl, int k) {
        const int64_t e = tl * 128 + tid;
        const bool v = e < a.n_elem;
        const float* src = v ? a.in + __ldg(a.phys_off + e) : nullptr;
#pragma unroll
        for (int p = 0; p < kNPT; ++p) {
            const int l = k * kNPT + p;
            x[p] = (v && l < a.NQ) ? __ldg(src + l) : 0.f;
        }
    };
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t e = tile * 128 + tid;              // this thread's element = TMEM lane
        const bool valid = e < a.n_elem;
        const int64_t next = tile + gridDim.x;
        if (MODE == 0) {
            // U: the tile's coefficient rows, read coalesced (a warp takes 32 rows,
            // its lanes consecutive modes), rounded to the operand type, zero padded to KP
            const int per_warp = 32 * a.KP;
            for (int base = lane; base < per_warp; base += 32 * 8) {
                float v[8];
                int row[8], col[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = base + 32 * u;
                    v[u] = 0.f;
                    row[u] = -1;
                    col[u] = 0;
                    if (idx < per_warp) {
                        const int rr = idx / a.KP, m = idx - rr * a.KP;
                        const int64_t er = tile * 128 + warp * 32 + rr;
                        row[u] = warp * 32 + rr;
                        col[u] = m;
                        if (er < a.n_elem && m < a.NP) v[u] = __ldg(a.in + __ldg(a.coeff_off + er) + m);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (row[u] >= 0)
                        O::put(sOp + (col[u] / O::KR) * 128 * 128 + O::off128((uint32_t)row[u], (uint32_t)(col[u] % O::KR)), v[u]);
            }
            tc::fence_async_smem();
            __syncthreads();
        } else if (!pre) {
            load_pts(tile, 0);
        }
        if (!pre)
            for (int k = 0; k < npre; ++k) issue(k);
        const int64_t po = valid ? __ldg(a.phys_off + e) : 0;
        auto store_chunk = [&](int j) {       // MODE 0: chunk j's point values from TMEM buffer j & 1
            float v[16];
            tc::ld_32x16(tbase + lane_base + (uint32_t)((j & 1) * kNPT), v);
            if (valid) {
                float* o = a.out + po + j * kNPT;
#pragma unroll
                for (int p = 0; p < kNPT; ++p)
                    if (j * kNPT + p < a.NQ) o[p] = v[p];
            }
        };
        for (int k = 0; k < nch && ok; ++k) {
            const int s = k % S;
            if (MODE == 1) {
                O::template put_pts<kNPT>(sOp + (size_t)(k & 1) * O::VBYTES, (uint32_t)tid, 0, x);
                tc::fence_async_smem();
                if (k + 1 < nch) load_pts(tile, k + 1);
            }
            wait_full(s);
            if (!ok) break;
            if (warp == 0) {         // warp-issued MMAs (one elected lane)
                tc::fence_after();
                const uint64_t dFs = dF + (uint32_t)s * st16;
                if (MODE == 0) {
                    const uint32_t d = tbase + (uint32_t)((k & 1) * kNPT);
                    for (uint32_t sl = 0; sl < nsl; ++sl)
#pragma unroll
                        for (uint32_t st = 0; st < 4; ++st)
                            O::mma(d, dU + (sl * 1024 + st * 2), dFs + (sl * hs16 + st * 2), id_f, sl > 0 || st > 0);
                } else {
                    const uint64_t dVk = dV + (uint32_t)(k & 1) * v16;
                    if (ES == 2) {
                        const uint64_t dRs = dRt + (uint32_t)s * st16;
                        O::mma(tbase, dVk, dRs, id_b0, k > 0);
                        if (n1 > 0) O::mma(tbase + 256, dVk, dRs + half16, id_b1, k > 0);
                    } else {
                        const uint64_t dRs = dRb + (uint32_t)s * st16;
#pragma unroll
                        for (uint32_t st = 0; st < O::VROW / 32; ++st) {
                            O::mma(tbase, dVk + st * 2, dRs + st * 2, id_b0, k > 0 || st > 0);
                            if (n1 > 0) O::mma(tbase + 256, dVk + st * 2, dRs + half16 + st * 2, id_b1, k > 0 || st > 0);
                        }
                    }
                }
                tc::commit_w(&B->mma[k & 1]);
            }
            ml |= 1u << (k & 1);
            if (k >= 1) {
                // MMA k-1 done: its stage takes chunk k-1+S; MODE 0 stores its points
                wait_mma((k - 1) & 1);
                if (!ok) break;
                if (k - 1 + S < nch) issue(k - 1 + S);
                if (MODE == 0) {
                    tc::fence_after();
                    store_chunk(k - 1);
                    tc::fence_before();
                    __syncthreads();
                }
            }
        }
        if (!ok) break;
        wait_mma((nch - 1) & 1);
        if (!ok) break;
        // every stage is free: the next tile's first chunks go in flight now
        pre = next < ntiles;
        if (pre) {
            for (int k = 0; k < npre; ++k) issue(k);
            if (MODE == 1) load_pts(next, 0);
        }
        tc::fence_after();
        if (MODE == 0) {
            store_chunk(nch - 1);
        } else {
            // the row's offset read once (a load per pass would wait behind the stores)
            const int64_t ce = valid ? __ldg(a.coeff_off + e) : 0;
            for (int c = 0; c < a.NPpad; c += 16) {
                float v[16];
                tc::ld_32x16(tbase + lane_base + (uint32_t)c, v);
                if (valid) {
                    float* o = a.out + ce + c;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c + i < a.NP) o[i] = v[i];
                }
            }
        }
        tc::fence_before();
        __syncthreads();
    }
    if (!ok) {      // nothing may still write shared or tensor memory when the CTA leaves
        for (int s = 0; s < S; ++s)
            if ((fl >> s) & 1u) mbar_wait_bounded(&B->full[s], (ph_full >> s) & 1u, kWaitLimitNs);
        for (int b = 0; b < 2; ++b)
            if ((ml >> b) & 1u) mbar_wait_bounded(&B->mma[b], (ph_mma >> b) & 1u, kWaitLimitNs);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// deterministic split-tile sum: out = part 0 + part 1 + ... in part order
__global__ void sum_parts_kernel(float* out, const int64_t* coeff_off, const float* part_out, int64_t n_elem, int NP,
                                 int nsplit) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_elem * NP) return;
    const int64_t e = i / NP;
    float acc = part_out[i];
    for (int p = 1; p < nsplit; ++p) acc += part_out[(int64_t)p * n_elem * NP + i];
    out[coeff_off[e] + (i - e * NP)] = acc;
}

// zero the block's output coefficients (the parts of a tile add into them)
__global__ void zero_coeffs_kernel(float* out, const int64_t* coeff_off, int64_t n_elem, int NP) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_elem * NP) return;
    const int64_t e = i / NP;
    out[coeff_off[e] + (i - e * NP)] = 0.f;
}

// Metric factors for the tensor-core forms: the seven factors of every point
// (the six unique entries of G and w|J|) in FP16 with two power-of-two scales
// per element.  The operands round to 11 (TF32) or 8 (BF16) significant bits,
// so FP16's 11 keep the factors as accurate as the operands at half the bytes
// of FP32.  Element e's six Laplacian factors are multiplied by 2^k with
// k = 14 - floor(log2 max|G|), its w|J| by 2^k' from its own maximum (the two
// differ by h^2, so one scale would push w|J| into FP16's subnormals on small
// elements): each group's largest lies in [2^14, 2^15) (FP16 ends at 65504)
// and only entries below 2^-28 of it are subnormal; the epilogue multiplies
// its outputs by 2^-k, 2^-k' (exact in FP32).
// Layout [tile][chunk][7 factors][kGeoGroups point runs][128 elements][kGeoPts
// points], an epilogue thread's run of a factor contiguous and a warp's 32
// elements adjacent; padded points and elements stay zero
// (the buffer is cleared first), and so does the scale of a padded element.
__host__ __device__ constexpr int64_t geom16_index(int64_t tile, int k, int f, int p, int r, int nch) {
    return ((((tile * nch + k) * 7 + f) * kGeoGroups + p / kGeoPts) * 128 + r) * kGeoPts + p % kGeoPts;
}

// factors of element e at point l: curved from the FP64 factors [n][7][NQp];
// affine from the element record [16] (|J| J^-1 J^-T, |J|, J^-1) and
// d eta / d xi at the point, in FP64
template <int SHAPE, bool CURVED>
__device__ __forceinline__ void point_factors(const double* g, int NQp, const double* z, const double* w, int Q,
                                              int64_t e, int l, double (&G)[7]) {
    if constexpr (CURVED) {
#pragma unroll
        for (int f = 0; f < 7; ++f) G[f] = g[(e * 7 + f) * (int64_t)NQp + l];
    } else {
        const int QQ = Q * Q;
        const int ii = l / QQ, jj = (l / Q) % Q, kk = l % Q;
        double Tm[3][3];
        deta_dxi<SHAPE, double>(z[ii], z[Q + jj], z[2 * Q + kk], Tm);
        const double wl = w[ii] * w[Q + jj] * w[2 * Q + kk];
        const double* R = g + e * 16;
        const double Km[3][3] = {{R[0], R[1], R[2]}, {R[1], R[3], R[4]}, {R[2], R[4], R[5]}};
        double M[3][3];
        for (int d = 0; d < 3; ++d)
            for (int j = 0; j < 3; ++j) M[d][j] = Tm[d][0] * Km[0][j] + Tm[d][1] * Km[1][j] + Tm[d][2] * Km[2][j];
        auto gg = [&](int d, int d2) { return wl * (M[d][0] * Tm[d2][0] + M[d][1] * Tm[d2][1] + M[d][2] * Tm[d2][2]); };
        G[0] = gg(0, 0); G[1] = gg(0, 1); G[2] = gg(0, 2); G[3] = gg(1, 1); G[4] = gg(1, 2); G[5] = gg(2, 2);
        G[6] = wl * R[6];
    }
}

// one warp per element: the largest of its six Laplacian factors and its
// largest w|J|, each group scaled by its own power of two (w|J| ~ h^3 and the
// G ~ h differ by h^2, which one scale would push into FP16's subnormals on
// small elements), then the scaled values; isc[2e], isc[2e + 1] undo the scales
template <int SHAPE, bool CURVED>
__global__ void tc_geom16_kernel(const double* g, int NQp, int NQ, const double* z, const double* w, int Q,
                                 uint16_t* out, float* isc, int64_t n_elem, int nch) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t e = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32; e < n_elem; e += nw) {
        double mg = 0.0, mm = 0.0;
        for (int l = lane; l < NQ; l += 32) {
            double G[7];
            point_factors<SHAPE, CURVED>(g, NQp, z, w, Q, e, l, G);
            for (int f = 0; f < 6; ++f) mg = fmax(mg, fabs(G[f]));
            mm = fmax(mm, fabs(G[6]));
        }
        for (int o = 16; o > 0; o >>= 1) {
            mg = fmax(mg, __shfl_xor_sync(0xffffffffu, mg, o));
            mm = fmax(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        }
        const int kg = mg > 0.0 ? 14 - ilogb(mg) : 0, km = mm > 0.0 ? 14 - ilogb(mm) : 0;
        const int64_t tile = e >> 7;
        const int r = (int)(e & 127);
        for (int l = lane; l < NQ; l += 32) {
            double G[7];
            point_factors<SHAPE, CURVED>(g, NQp, z, w, Q, e, l, G);
            for (int f = 0; f < 7; ++f)
                out[geom16_index(tile, l / kNPT, f, l % kNPT, r, nch)] =
                    __half_as_ushort(__float2half_rn((float)ldexp(G[f], f < 6 ? kg : km)));
        }
        if (lane == 0) {
            isc[2 * e] = (float)ldexp(1.0, -kg);
            isc[2 * e + 1] = (float)ldexp(1.0, -km);
        }
    }
}

template <int SHAPE>
cudaError_t geom16_shape(bool curved, const double* g, int NQp, int NQ, const double* z, const double* w, int Q,
                         uint16_t* out, float* isc, int64_t n_elem, int nch, cudaStream_t s) {
    const int64_t blocks = (n_elem + 7) / 8;
    const unsigned grid = (unsigned)(blocks < 8192 ? blocks : 8192);
    if (curved) tc_geom16_kernel<SHAPE, true><<<grid, 256, 0, s>>>(g, NQp, NQ, z, w, Q, out, isc, n_elem, nch);
    else tc_geom16_kernel<SHAPE, false><<<grid, 256, 0, s>>>(g, NQp, NQ, z, w, Q, out, isc, n_elem, nch);
    return cudaGetLastError();
}

}  // namespace

// Shared memory a CTA may take: all of the SM's (one CTA per SM) or half of it
// (two).  The smallest request keeps the tensor-memory allocations of the CTAs
// that share an SM within its 512 columns: a one-CTA kernel (512 columns)
// leaves less than a two-CTA kernel's CTA (256 columns) needs, and two-CTA
// CTAs leave no room for a third.
constexpr int kSmemCap1 = 227 * 1024, kSmemCap2 = 113 * 1024;
constexpr int kSmemMin1 = 152 * 1024, kSmemMin2 = 77 * 1024;

// ring stages (2..kMaxStages) that fit beside ubufs U buffers and vbufs V' tiles
// (four components each)
int tc_stages(int KP, int stage_bytes, int es, int ubufs, int vbufs, int cap) {
    const int base = 2048 + ubufs * 128 * KP * es + vbufs * 4 * 128 * kNPT * es;   // alignment slack + barriers + U + V'
    for (int st = kMaxStages; st >= 2; --st)
        if (base + st * stage_bytes <= cap) return st;
    return 0;
}

// launch plan: CTAs per SM, U buffers, ring stages, dynamic shared memory.
// Two CTAs per SM (allow2: the block has at least two tiles per SM, so both
// slots fill without splitting tiles) for BF16 blocks whose output accumulator
// fits beside the forward ones in 256 columns (N_P <= 64) and whose buffers
// fit half the SM;
// a second U buffer where it leaves a deep ring (or costs no stage).
struct TcPlan {
    int ctas, ubufs, stages, smem;
};
TcPlan tc_plan(int KP, int NPpad, int stage_bytes, int es, bool allow2, int variant = 0) {
    // BF16 reading the forward stage again holds a stage through kFB - 1 chunks:
    // kFB + 1 stages (kFB = 2 in the lean variant)
    const int need = (es == 2 && variant != 1) ? (variant == 2 ? 3 : kFwdBufs + 1) : 2;
    const int vbufs = variant == 2 ? 1 : 2;
    for (int ctas = 2; ctas >= 1; --ctas) {
        if (ctas == 2 && !(allow2 && es == 2 && variant == 0 && NPpad <= kOutCol / 3 && kOutCol + NPpad <= 256)) continue;
        const int cap = ctas == 2 ? kSmemCap2 : kSmemCap1;
        const int s1 = tc_stages(KP, stage_bytes, es, 1, vbufs, cap);
        if (s1 < need) continue;
        const int s2 = tc_stages(KP, stage_bytes, es, 2, vbufs, cap);
        const int ub = (s2 >= 6 || (s2 == s1 && s2 >= need)) ? 2 : 1;
        const int st = ub == 2 ? s2 : s1;
        int smem = 2048 + ub * 128 * KP * es + vbufs * 4 * 128 * kNPT * es + st * stage_bytes;
        const int mn = ctas == 2 ? kSmemMin2 : kSmemMin1;
        if (smem < mn) smem = mn;
        return {ctas, ub, st, smem};
    }
    return {1, 1, 0, 0};
}

// BF16 variant of a block (`TCArgs::variant`): 0 up to 256 modes; 2, the lean
// form, up to 320 modes where its plan fits an SM; 1 (streamed backward tiles,
// mode parts) otherwise.  TF32: 0.
int tc_variant(int KP, int NPpad, int fwd_bytes, int es) {
    if (es != 2 || NPpad <= kTcMaxModes) return 0;
    if (NPpad <= kOutColMax && tc_plan(KP, NPpad, fwd_bytes, es, false, 2).stages >= 3) return 2;
    return 1;
}

int tc_chunk_points() { return kNPT; }

int64_t tc_geom_halves(int64_t n_elem, int nch) { return (n_elem + 127) / 128 * nch * 7 * kNPT * 128; }

cudaError_t tc_geom_layout16(int shape, bool curved, const double* g, int NQp, int NQ, const double* z, const double* w, int Q,
                             uint16_t* out, float* isc, int64_t n_elem, int nch, cudaStream_t s) {
    if (n_elem <= 0) return cudaSuccess;
    const int64_t ntiles = (n_elem + 127) / 128;
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)tc_geom_halves(n_elem, nch) * sizeof(uint16_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(isc, 0, (size_t)ntiles * 128 * 2 * sizeof(float), s);
    if (e != cudaSuccess) return e;
    switch (shape) {
        case HP_HEX: return geom16_shape<HP_HEX>(curved, g, NQp, NQ, z, w, Q, out, isc, n_elem, nch, s);
        case HP_PRISM: return geom16_shape<HP_PRISM>(curved, g, NQp, NQ, z, w, Q, out, isc, n_elem, nch, s);
        case HP_PYR: return geom16_shape<HP_PYR>(curved, g, NQp, NQ, z, w, Q, out, isc, n_elem, nch, s);
        default: return geom16_shape<HP_TET>(curved, g, NQp, NQ, z, w, Q, out, isc, n_elem, nch, s);
    }
}

// point-chunk parts per tile: split until the grid covers the CTA slots (at
// least 4 chunks per part); 0 on error
// output-mode parts of a tile: BF16 past 320 modes splits its N_P output
// columns into parts of at most 320 (multiples of 16) that fit the tensor
// memory beside the forward accumulators; one part otherwise
void tc_mode_parts(const TCArgs& a, int* nmp, int* mw) {
    if (a.variant != 1 || a.NPpad <= kOutColMax) {
        *nmp = 1;
        *mw = a.NPpad;
        return;
    }
    *nmp = (a.NPpad + kOutColMax - 1) / kOutColMax;
    *mw = ((a.NPpad + *nmp - 1) / *nmp + 15) & ~15;
}

int tc_emat_nsplit(const TCArgs& a) {
    const int64_t ntiles = (a.n_elem + 127) / 128;
    if (ntiles <= 0) return 1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const TcPlan pl = tc_plan(a.KP, a.NPpad, a.stage_bytes, a.es, ntiles >= 2 * (int64_t)sms, a.variant);
    if (pl.stages == 0) return 0;
    // parts per tile: as many as keep every work item in one wave of the
    // launch's CTA slots (a ceiling would leave some CTAs a second item, and
    // the launch twice an item's time), at least four chunks a part
    // (a block launched with others in a graph splits for its share of the slots)
    int nmp = 1, mw = 0;
    tc_mode_parts(a, &nmp, &mw);
    const double slots = (double)sms * pl.ctas * (a.slot_share > 0.0 ? a.slot_share : 1.0);
    const int64_t ns = std::max<int64_t>(1, (int64_t)(slots / (double)(ntiles * nmp)));
    const int64_t cap = a.nch / 4 > 1 ? a.nch / 4 : 1;
    return (int)(ns < cap ? ns : cap);
}

// shared memory of a hybrid launch with `stages` ring stages (0: the plan's
// choice, 3 if it fits, else 2); *stages_out, *stage_bytes_out receive the plan
int tc_hyb_smem(int mode, int es, int KP, int NPpad, int bwd_bytes, int* stages_out, int* stage_bytes_out) {
    const int kr = 128 / es, nsl = (KP + kr - 1) / kr;
    const int op_bytes = mode == 0 ? 128 * KP * es : 2 * 128 * kNPT * es;
    const int stb = (((mode == 1 && es == 4) ? bwd_bytes : nsl * kHybSlice) + 1023) & ~1023;
    int st = kHybMaxStages, smem = 0;
    for (; st >= 2; --st) {
        smem = 1024 + (op_bytes + 1023) / 1024 * 1024 + st * stb + 1024;
        if (smem <= 227 * 1024) break;
    }
    // MODE 1 holds 256 (N_P <= 256) or 512 TMEM columns: shared memory keeps
    // at most two CTAs, or one, on an SM, so that every allocation succeeds at once
    if (mode == 1) smem = std::max(smem, NPpad > 256 ? 120 * 1024 : 80 * 1024);
    if (stages_out) *stages_out = st;
    if (stage_bytes_out) *stage_bytes_out = stb;
    return st >= 2 ? smem : 0;
}

cudaError_t tc_hyb_launch(const HybArgs& a0, int mode, cudaStream_t s) {
    const int64_t ntiles = (a0.n_elem + 127) / 128;
    if (ntiles <= 0) return cudaSuccess;
    if (a0.NPpad > kTcHybMaxModes || a0.NPpad % 16 || (a0.es != 2 && a0.es != 4) || a0.nch < 1)
        return cudaErrorInvalidValue;
    HybArgs a = a0;
    const int smem = tc_hyb_smem(mode, a.es, a.KP, a.NPpad, a.bwd_bytes, &a.stages, &a.stage_bytes);
    if (smem <= 0 || smem > 227 * 1024) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM: shared memory (228 KB an SM, 1 KB reserved per CTA),
    // at most 8, and the tensor memory the CTAs hold (512 columns an SM)
    const int ncols = mode == 0 ? 32 : (a.NPpad > 256 ? 512 : 256);
    const int per = std::max(1, std::min({228 * 1024 / (smem + 1024), 8, 512 / ncols}));
    auto launch = [&](auto kern) -> cudaError_t {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e2 != cudaSuccess) return e2;
        const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms * per);
        kern<<<grid, 128, smem, s>>>(a);
        return cudaGetLastError();
    };
    if (a.es == 4) return mode == 0 ? launch(tc_hyb_kernel<4, 0>) : launch(tc_hyb_kernel<4, 1>);
    return mode == 0 ? launch(tc_hyb_kernel<2, 0>) : launch(tc_hyb_kernel<2, 1>);
}

cudaError_t tc_emat_launch(const TCArgs& a, cudaStream_t s) {
    const int64_t ntiles = (a.n_elem + 127) / 128;
    if (ntiles <= 0) return cudaSuccess;
    TCArgs b = a;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (a.NPpad > (a.variant ? kTcMaxModes16 : kTcMaxModes) || (a.variant && a.es != 2) || a.variant < 0 || a.variant > 2)
        return cudaErrorInvalidValue;
    const TcPlan pl = tc_plan(a.KP, a.NPpad, a.stage_bytes, a.es, ntiles >= 2 * (int64_t)sms, a.variant);
    if (pl.stages == 0) return cudaErrorInvalidValue;
    b.ubufs = pl.ubufs;
    b.stages = pl.stages;
    auto kern = a.es == 4 ? tc_emat_kernel<4, 16> : a.variant == 2 ? tc_emat_kernel<2, 16, 2>
              : a.variant == 1 ? tc_emat_kernel<2, 16, 1>
              : pl.ctas == 2 ? tc_emat_kernel<2, 8> : tc_emat_kernel<2, 16>;
    const int threads = pl.ctas == 2 ? Epi<8>::kThreads : Epi<16>::kThreads;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
    if (e != cudaSuccess) return e;
    const int slots = sms * pl.ctas;
    b.nsplit = tc_emat_nsplit(a);
    if (b.nsplit < 1) return cudaErrorInvalidValue;
    tc_mode_parts(a, &b.nmpart, &b.mwidth);
    const int64_t n = a.n_elem * a.NP;
    if (b.nsplit == 1) b.part_out = nullptr;
    if (b.nsplit > 1 && !b.part_out)   // atomics: the parts add into a zeroed output
        zero_coeffs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.out, a.coeff_off, a.n_elem, a.NP);
    const int64_t nwork = ntiles * b.nsplit * b.nmpart;
    const int grid = (int)(nwork < slots ? nwork : slots);
    kern<<<grid, threads, pl.smem, s>>>(b);
    e = cudaGetLastError();
    if (e == cudaSuccess && b.part_out) {
        sum_parts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.out, a.coeff_off, b.part_out, a.n_elem, a.NP,
                                                                    b.nsplit);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace hp
