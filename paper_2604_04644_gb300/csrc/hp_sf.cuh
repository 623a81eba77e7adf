// Fused sum-factorised element operators (one kernel per block of elements
// of equal shape and order).
//
// Collocated Helmholtz (paper Sec. 2.2 Eq. (helm1); Sec. 3.3, algorithm
// "Helmholtz implementation by collocated approach"):
//   u = B uhat                          BwdTrans, three 1-D passes (Sec. 3.3.2)
//   v_d = D_d u                         StdDeriv, collocation differentiation (Eq. dphitodh)
//   w_d = sum_d' G_dd' v_d',  t = lambda w|J| u     ApplyMetric (includes W)
//   u' = sum_d D_d^T w_d + t            SumStdDeriv
//   out = B^T u'                        Restrict (IProductWRTBase), three 1-D passes
// Mass skips the derivative steps; the building blocks are the pieces.
//
// Collapsed shapes (Sec. 2.3): the modes are generalised tensor products
// phi = A_a(eta1) F^{t(a)}_b(eta2) F^{s(a,b)}_c(eta3), evaluated on a padded
// (P+1)^3 slot tensor whose 1-D factor tables depend on the family indices
// t(a), s(a,b) (zero rows pad the triangular index ranges).  Modes that are
// constant in eta1 (or eta1 and eta2) -- the collapsed-vertex modes -- occupy
// 2 (or 4) slots: BwdTrans copies their coefficient into each slot and the
// restriction sums the slots.
//
// GPU organisation (a GB300 design, not the paper's): a persistent grid of
// CTAs, each staging the reference tables once into shared memory with a
// 1-D bulk copy (TMA) and then looping over groups of EPB elements; every
// pass assigns one output entry per thread over the whole group
// (threaded on output point across EPB elements) with intermediates in
// shared memory; geometric factors stream from HBM in the metric pass.
#pragma once
#include "hp_device.cuh"

namespace hp {

// Tile variants (chosen per block by the autotuner): the shared-memory budget
// for the element group, hence elements per CTA (EPB) and CTAs per SM.
constexpr int kTileBudget[3] = {56 * 1024, 20 * 1024, 110 * 1024};
constexpr int kNumTiles = 3;

template <int P, typename T, int TILE = 0>
struct SFCfg {
    static constexpr int n = P + 1, Q = P + 2, QQ = Q * Q, NQ = Q * Q * Q, N3 = n * n * n;
    static constexpr int NT = 256;
    static constexpr int per_elem_bytes = 5 * NQ * (int)sizeof(T);
    static constexpr int budget = kTileBudget[TILE];
    static constexpr int epb0 = budget / per_elem_bytes;
    static constexpr int EPB = epb0 < 1 ? 1 : (epb0 > 64 ? 64 : epb0);
};

template <int SHAPE, int P, typename T, int TILE>
__host__ __device__ constexpr int sf_smem_bytes() {
    return 16 + blob_layout_c(SHAPE, P, (int)sizeof(T)).total_bytes +
           SFCfg<P, T, TILE>::EPB * 5 * SFCfg<P, T, TILE>::NQ * (int)sizeof(T);
}

// FP32: as many CTAs per SM as the tile's shared memory admits (at most four, 64
// registers a thread), so that the loads batched per thread do not take
// registers from occupancy; FP64: no target
template <int SHAPE, int P, typename T, int TILE>
__host__ __device__ constexpr int sf_min_blocks() {
    if (sizeof(T) != 4) return 0;
    const int b = (228 * 1024) / (sf_smem_bytes<SHAPE, P, T, TILE>() + 1024);
    return b < 1 ? 1 : (b > 4 ? 4 : b);
}

// One CTA's share of a block of (SHAPE, P): stage the block's reference
// tables into shared memory (one bulk copy on the CTA's barrier at smem[0],
// initialised by the caller, waiting on `phase`, which then flips), then
// process the element groups g_first, g_first + g_step, ... below g_end.
// Returns false (error word set) if the copy did not land in time.  A is
// SFArgs<T> or any struct with the same fields the instantiation reads.
template <int SHAPE, int P, typename T, bool AFFINE, int TILE, typename A>
__device__ __forceinline__ bool sf_groups(const A& args, unsigned char* smem, int64_t g_first, int64_t g_step,
                                          int64_t g_end, uint32_t& phase) {
    using C = SFCfg<P, T, TILE>;
    constexpr int n = C::n, Q = C::Q, QQ = C::QQ, NQ = C::NQ, N3 = C::N3, EPB = C::EPB, NT = C::NT;
    constexpr int NN = n * n, Qh = (Q + 1) / 2;   // Qh: even-odd pairs (i, Q-1-i) along eta1
    constexpr BlobLayout L = blob_layout_c(SHAPE, P, (int)sizeof(T));
    constexpr int NP = n_modes_c(SHAPE, P);
    constexpr int NQp = (NQ + 3) & ~3;
    // FP32: register-blocked line passes with constant-bank tables (the shared
    // memory load pipe is the limit); FP64: one output per thread (more parallel
    // tasks to keep the FP64 pipe, the limit there, busy)
    constexpr bool LINES = sizeof(T) == 4;
    constexpr int kU = 4;      // FP32: loop iterations per thread whose global loads are issued together
    constexpr int kUG = 8;     // the same for the coefficient gather (one batch for most blocks)

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    unsigned char* tab = smem + 16;
    if (!stage_tables_phase(tab, args.blob, L.total_bytes, bar, phase, args.err)) return false;

    const T* Ta = reinterpret_cast<const T*>(tab) + L.Ta;   // parity form {1/2, -z/2, psi_2..}
    const T* Td = reinterpret_cast<const T*>(tab) + L.Td;   // its eta1 derivative
    const T* Tb = reinterpret_cast<const T*>(tab) + L.Tb;
    const T* Tc = reinterpret_cast<const T*>(tab) + L.Tc;
    const T* D0 = reinterpret_cast<const T*>(tab) + L.D;
    const T* D1 = D0 + QQ;
    const T* D2 = D0 + 2 * QQ;
    const T* zt = reinterpret_cast<const T*>(tab) + L.z;
    const T* wt = reinterpret_cast<const T*>(tab) + L.w;
    const T* rzt = reinterpret_cast<const T*>(tab) + L.rz;
    const uint8_t* famb = tab + L.famb;
    const uint8_t* famc = tab + L.famc;
    const int16_t* slot2mode = reinterpret_cast<const int16_t*>(tab + L.slot2mode);
    const int16_t* mode_slots = reinterpret_cast<const int16_t*>(tab + L.mode_slots);
    // valid index sets of the collapsed shapes (the hexahedron indexes directly)
    constexpr int NPR = npairs_c(SHAPE, P), NVL = nvalid_c(SHAPE, P);
    const int32_t* pairs = reinterpret_cast<const int32_t*>(tab + L.pairs);
    const int32_t* valid = reinterpret_cast<const int32_t*>(tab + L.valid);
    const int16_t* poff = reinterpret_cast<const int16_t*>(tab + L.poff);
    const uint8_t* porder = tab + L.porder;
    T* S1 = reinterpret_cast<T*>(tab + L.total_bytes);   // [EPB][4*NQ]: u, v1, v2, v3
    T* S2 = S1 + EPB * 4 * NQ;                            // [EPB][NQ]

    const int tid = threadIdx.x;
    const int op = args.op;
    const bool adr = op == HP_ADVECTION_DIFFUSION_REACTION;
    const bool coeff_in = (op == HP_MASS || op == HP_LAPLACIAN || op == HP_HELMHOLTZ || op == HP_BWDTRANS || adr);
    const bool deriv = (op == HP_LAPLACIAN || op == HP_HELMHOLTZ || op == HP_PHYSDERIV || adr);
    const bool sumderiv = (op == HP_LAPLACIAN || op == HP_HELMHOLTZ || op == HP_IPRODUCT_WRT_DERIV_BASE || adr);
    const bool merged = !LINES && deriv && coeff_in;   // v1 comes out of the eta1 pass
    bool point_io = false;                             // FP32: point values in and out (no B, B^T)
    if constexpr (LINES) point_io = args.point_io != 0;

    for (int64_t g = g_first; g < g_end; g += g_step) {
        const int64_t e0 = g * EPB;
        const int ne = (int)min((int64_t)EPB, args.n_elem - e0);

        if (coeff_in && !point_io) {
            // gather modal coefficients into the slot tensor
            // (slots a = 0, 1 take the sum and the difference of the two coefficients,
            // the inputs of the parity-form eta1 table)
            if constexpr (LINES) {
                // FP32 (the passes are cheap, the memory latency is not): kUG slots
                // per thread have their loads issued before any is stored
                for (int base = tid; base < EPB * N3; base += NT * kUG) {
                    T v[kUG];
#pragma unroll
                    for (int u = 0; u < kUG; ++u) {
                        const int idx = base + u * NT;
                        v[u] = T(0);
                        if (idx < EPB * N3) {
                            const int e = idx / N3, sl = idx - e * N3, m = slot2mode[sl];
                            if (e < ne && m >= 0) {
                                const T* cin = args.in + __ldg(args.coeff_off + e0 + e);
                                if (sl >= 2 * NN) v[u] = __ldg(cin + m);
                                else if (sl < NN) v[u] = __ldg(cin + m) + __ldg(cin + slot2mode[sl + NN]);
                                else v[u] = __ldg(cin + slot2mode[sl - NN]) - __ldg(cin + m);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kUG; ++u) {
                        const int idx = base + u * NT;
                        if (idx < EPB * N3) {
                            const int e = idx / N3;
                            S2[e * NQ + idx - e * N3] = v[u];
                        }
                    }
                }
            } else
            for (int idx = tid; idx < EPB * N3; idx += NT) {
                int e = idx / N3, sl = idx - e * N3;
                T v = T(0);
                if (e < ne) {
                    int m = slot2mode[sl];
                    if (m >= 0) {
                        const T* cin = args.in + args.coeff_off[e0 + e];
                        if (sl >= 2 * NN) v = cin[m];
                        else if (sl < NN) v = cin[m] + cin[slot2mode[sl + NN]];
                        else v = cin[slot2mode[sl - NN]] - cin[m];
                    }
                }
                S2[e * NQ + sl] = v;
            }
            __syncthreads();
            // eta3 pass over the valid (a,b) pairs p (compact, a-major):
            // f[p][k] = sum_{c < len(p)} Tc[s(a,b)][c][k] uhat[a][b][c]; pairs taken
            // in order of decreasing length so that a warp's loops end together
            for (int idx = tid; idx < EPB * NPR * Q; idx += NT) {
                int e = idx / (NPR * Q), r = idx - e * (NPR * Q);
                int pp = r / Q, k = r - pp * Q;
                T acc = T(0);
                if constexpr (SHAPE == 0) {
                    const T* tc = Tc + k;
                    const T* x = S2 + e * NQ + pp * n;
#pragma unroll
                    for (int c = 0; c < n; ++c) acc += tc[c * Q] * x[c];
                    S1[e * 4 * NQ + pp * Q + k] = acc;
                } else {
                    const int p = porder[pp], pr = pairs[p];
                    const int len = pr >> 24;
                    const T* tc = Tc + ((pr >> 16) & 0xff) * n * Q + k;
                    const T* x = S2 + e * NQ + (pr & 0xffff) * n;
#pragma unroll
                    for (int c = 0; c < n; ++c) {
                        if (c >= len) break;
                        acc += tc[c * Q] * x[c];
                    }
                    S1[e * 4 * NQ + p * Q + k] = acc;
                }
            }
            __syncthreads();
            // eta2 pass: g[a][j][k] = sum_{b < len_b(a)} Tb[t(a)][b][j] f[p(a,b)][k]
            for (int idx = tid; idx < EPB * n * QQ; idx += NT) {
                int e = idx / (n * QQ), r = idx - e * (n * QQ);
                int a = r / QQ, jk = r - a * QQ, j = jk / Q, k = jk - j * Q;
                T acc = T(0);
                if constexpr (SHAPE != HP_TET) {       // every (a, b) pair is valid
                    const T* tb = Tb + j;
                    const T* x = S1 + e * 4 * NQ + a * n * Q + k;
#pragma unroll
                    for (int b = 0; b < n; ++b) acc += tb[b * Q] * x[b * Q];
                } else {
                    const int p0 = poff[a], lb = poff[a + 1] - p0;
                    const T* tb = Tb + famb[a] * n * Q + j;
                    const T* x = S1 + e * 4 * NQ + p0 * Q + k;
#pragma unroll
                    for (int b = 0; b < n; ++b) {
                        if (b >= lb) break;
                        acc += tb[b * Q] * x[b * Q];
                    }
                }
                S2[e * NQ + r] = acc;
            }
            __syncthreads();
            if constexpr (LINES) {
            // eta1 pass: u[i][j][k] = sum_a Ta[a][i] g[a][j][k]; one (j,k) line per
            // thread, the table as constant-bank operands
            for (int idx = tid; idx < EPB * QQ; idx += NT) {
                int e = idx / QQ, jk = idx - e * QQ;
                const T* x = S2 + e * NQ + jk;
                T g[n];
#pragma unroll
                for (int a = 0; a < n; ++a) g[a] = x[a * QQ];
                T* u = S1 + e * 4 * NQ + jk;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    T acc = T(0);
#pragma unroll
                    for (int a = 0; a < n; ++a) acc += args.cTa[a * Q + i] * g[a];
                    u[i * QQ] = acc;
                }
            }
            __syncthreads();
            } else {
            // eta1 pass in even-odd pairs (i, Q-1-i): row a of the parity table has
            // parity (-1)^a, so u_i = E + O and u_{Q-1-i} = E - O with E, O the sums
            // over the even and odd rows; the derivative operators take
            // v1 = du/d eta1 = sum_a Td[a][i] g[a] in the same pass (exact for the
            // degree-P rows, replaces the collocation derivative along eta1)
            for (int idx = tid; idx < EPB * Qh * QQ; idx += NT) {
                int e = idx / (Qh * QQ), r = idx - e * (Qh * QQ);
                int i = r / QQ, jk = r - i * QQ, i2 = Q - 1 - i;
                const T* x = S2 + e * NQ + jk;
                T ev = T(0), od = T(0);
#pragma unroll
                for (int a = 0; a < n; a += 2) ev += Ta[a * Q + i] * x[a * QQ];
#pragma unroll
                for (int a = 1; a < n; a += 2) od += Ta[a * Q + i] * x[a * QQ];
                T* u = S1 + e * 4 * NQ + jk;
                u[i * QQ] = ev + od;
                if (i2 != i) u[i2 * QQ] = ev - od;
                if (merged) {
                    T dv = T(0), dd = T(0);
#pragma unroll
                    for (int a = 1; a < n; a += 2) dv += Td[a * Q + i] * x[a * QQ];
#pragma unroll
                    for (int a = 2; a < n; a += 2) dd += Td[a * Q + i] * x[a * QQ];
                    u[NQ + i * QQ] = dv + dd;
                    if (i2 != i) u[NQ + i2 * QQ] = dv - dd;
                }
            }
            __syncthreads();
            }
            if (op == HP_BWDTRANS) {
                for (int idx = tid; idx < EPB * NQ; idx += NT) {
                    int e = idx / NQ, r = idx - e * NQ;
                    if (e < ne) args.out[args.phys_off[e0 + e] + r] = S1[e * 4 * NQ + r];
                }
                __syncthreads();
                continue;
            }
        } else {
            const int nc = (op == HP_IPRODUCT_WRT_DERIV_BASE) ? 3 : 1;
            const int dst = (op == HP_IPRODUCT_WRT_DERIV_BASE) ? 1 : 0;
            for (int idx = tid; idx < EPB * NQ; idx += NT) {
                int e = idx / NQ, r = idx - e * NQ;
                for (int c = 0; c < nc; ++c) {
                    T v = T(0);
                    if (e < ne) v = args.in[c * args.n_phys_total + args.phys_off[e0 + e] + r];
                    S1[e * 4 * NQ + (dst + c) * NQ + r] = v;
                }
            }
            __syncthreads();
        }

        if constexpr (LINES) {
        if (deriv) {
            // v_d = D_d u (collocation differentiation), one line per thread and
            // direction, D as constant-bank operands
            for (int idx = tid; idx < EPB * QQ; idx += NT) {     // eta1 lines (j,k)
                int e = idx / QQ, jk = idx - e * QQ;
                const T* u = S1 + e * 4 * NQ + jk;
                T x[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) x[m] = u[m * QQ];
                T* v = S1 + e * 4 * NQ + NQ + jk;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    T acc = T(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc += args.cD[0][i * Q + m] * x[m];
                    v[i * QQ] = acc;
                }
            }
            for (int idx = tid; idx < EPB * QQ; idx += NT) {     // eta2 lines (i,k)
                int e = idx / QQ, ik = idx - e * QQ, i = ik / Q, k = ik - i * Q;
                const T* u = S1 + e * 4 * NQ + i * QQ + k;
                T x[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) x[m] = u[m * Q];
                T* v = S1 + e * 4 * NQ + 2 * NQ + i * QQ + k;
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    T acc = T(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc += args.cD[1][j * Q + m] * x[m];
                    v[j * Q] = acc;
                }
            }
            for (int idx = tid; idx < EPB * QQ; idx += NT) {     // eta3 lines (i,j)
                int e = idx / QQ, ij = idx - e * QQ;
                const T* u = S1 + e * 4 * NQ + ij * Q;
                T x[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) x[m] = u[m];
                T* v = S1 + e * 4 * NQ + 3 * NQ + ij * Q;
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    T acc = T(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc += args.cD[2][k * Q + m] * x[m];
                    v[k] = acc;
                }
            }
            __syncthreads();
        }

        } else {
        if (deriv) {
            // v_d = D_d u (collocation differentiation in eta_2, eta_3, and in eta_1
            // when v1 did not come out of the eta1 pass)
            for (int idx = tid; idx < EPB * NQ; idx += NT) {
                int e = idx / NQ, r = idx - e * NQ;
                int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q;
                const T* u = S1 + e * 4 * NQ;
                T a2 = T(0), a3 = T(0);
#pragma unroll
                for (int m = 0; m < Q; ++m) {
                    a2 += D1[j * Q + m] * u[i * QQ + m * Q + k];
                    a3 += D2[k * Q + m] * u[i * QQ + j * Q + m];
                }
                if (!merged) {
                    T a1 = T(0);
#pragma unroll
                    for (int m = 0; m < Q; ++m) a1 += D0[i * Q + m] * u[m * QQ + jk];
                    S1[e * 4 * NQ + NQ + r] = a1;
                }
                S1[e * 4 * NQ + 2 * NQ + r] = a2;
                S1[e * 4 * NQ + 3 * NQ + r] = a3;
            }
            __syncthreads();
        }

        }

        // pointwise metric
        bool metric_done = false;
        if constexpr (LINES && !AFFINE) {
            if (op == HP_MASS || op == HP_LAPLACIAN || op == HP_HELMHOLTZ) {
                // FP32: the factors of kU points per thread are loaded before any is
                // used, so their HBM latencies overlap
                const bool lap = op != HP_MASS;
                for (int base = tid; base < EPB * NQ; base += NT * kU) {
                    T G[kU][7];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int idx = base + u * NT, e = idx / NQ, r = idx - e * NQ;
#pragma unroll
                        for (int f = 0; f < 7; ++f) G[u][f] = T(0);
                        if (idx < EPB * NQ && e < ne) {
                            const T* gp = args.geom + (e0 + e) * 7 * (int64_t)NQp + r;
                            G[u][6] = __ldg(gp + 6 * NQp);
                            if (lap) {
#pragma unroll
                                for (int f = 0; f < 6; ++f) G[u][f] = __ldg(gp + f * NQp);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int idx = base + u * NT, e = idx / NQ, r = idx - e * NQ;
                        if (idx >= EPB * NQ) break;
                        T* uu = S1 + e * 4 * NQ + r;
                        if (e >= ne) {
                            S2[e * NQ + r] = T(0);
                            if (lap) { uu[NQ] = T(0); uu[2 * NQ] = T(0); uu[3 * NQ] = T(0); }
                            continue;
                        }
                        const T uval = uu[0];
                        if (!lap) {
                            S2[e * NQ + r] = G[u][6] * uval;
                            continue;
                        }
                        const T v1 = uu[NQ], v2 = uu[2 * NQ], v3 = uu[3 * NQ];
                        uu[NQ] = G[u][0] * v1 + G[u][1] * v2 + G[u][2] * v3;
                        uu[2 * NQ] = G[u][1] * v1 + G[u][3] * v2 + G[u][4] * v3;
                        uu[3 * NQ] = G[u][2] * v1 + G[u][4] * v2 + G[u][5] * v3;
                        S2[e * NQ + r] = (op == HP_HELMHOLTZ) ? args.lambda * G[u][6] * uval : T(0);
                    }
                }
                metric_done = true;
            }
        }
        if (!metric_done)
        for (int idx = tid; idx < EPB * NQ; idx += NT) {
            int e = idx / NQ, r = idx - e * NQ;
            if (e >= ne) {
                S2[e * NQ + r] = T(0);
                if (sumderiv) {
                    S1[e * 4 * NQ + NQ + r] = T(0);
                    S1[e * 4 * NQ + 2 * NQ + r] = T(0);
                    S1[e * 4 * NQ + 3 * NQ + r] = T(0);
                }
                continue;
            }
            const int64_t eg = e0 + e;
            T G[6], wJ, Gx[3][3];
            const bool need_gx = (op == HP_PHYSDERIV || op == HP_IPRODUCT_WRT_DERIV_BASE || adr);
            if (AFFINE && (op == HP_LAPLACIAN || op == HP_HELMHOLTZ || adr)) {
                // affine element: w = wl T K T^T v with K = |J| (d xi/d x)(d xi/d x)^T
                // per element and T = d eta / d xi at the reference point, whose
                // collapse factors come from the reciprocal tables 1/(1 - z) (no
                // division and no per-point G: the product is applied factor by
                // factor); the same G_dd' = wl (T K T^T)_dd' as the curved path
                const T* rec = args.geom + eg * 16;
                const int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q;
                const T wl = wt[i] * wt[Q + j] * wt[2 * Q + k];
                T* u = S1 + e * 4 * NQ + r;
                const T uval = u[0], v0 = u[NQ], v1 = u[2 * NQ], v2 = u[3 * NQ];
                T g0 = v0, g1 = v1, g2 = v2;                 // g = T^T v
                T t00 = T(1), t01 = T(0), t02 = T(0), t11 = T(1), t12 = T(0);
                if constexpr (SHAPE != HP_HEX) {
                    const T r3 = rzt[2 * Q + k];
                    const T a1 = T(1) + zt[i];
                    if constexpr (SHAPE == HP_TET) {
                        const T r23 = T(2) * rzt[Q + j] * r3;
                        t00 = T(2) * r23; t01 = a1 * r23; t02 = t01;
                        t11 = T(2) * r3; t12 = (T(1) + zt[Q + j]) * r3;
                    } else {
                        t00 = T(2) * r3; t02 = a1 * r3;
                        if constexpr (SHAPE == HP_PYR) { t11 = T(2) * r3; t12 = (T(1) + zt[Q + j]) * r3; }
                    }
                    g0 = t00 * v0;
                    g1 = t01 * v0 + t11 * v1;
                    g2 = t02 * v0 + t12 * v1 + v2;
                }
                const T h0 = wl * (rec[0] * g0 + rec[1] * g1 + rec[2] * g2);
                const T h1 = wl * (rec[1] * g0 + rec[3] * g1 + rec[4] * g2);
                const T h2 = wl * (rec[2] * g0 + rec[4] * g1 + rec[5] * g2);
                u[NQ] = t00 * h0 + t01 * h1 + t02 * h2;     // w = T h
                u[2 * NQ] = t11 * h1 + t12 * h2;
                u[3 * NQ] = h2;
                T mass = (op == HP_HELMHOLTZ || adr) ? args.lambda * uval : T(0);
                if (adr) {
                    // advection a . grad u = c . v with c = T (d xi / d x) a, the
                    // velocity in eta coordinates (rec[7 + 3 a + i] = d xi_a / d x_i)
                    const T b0 = rec[7] * args.adv[0] + rec[8] * args.adv[1] + rec[9] * args.adv[2];
                    const T b1 = rec[10] * args.adv[0] + rec[11] * args.adv[1] + rec[12] * args.adv[2];
                    const T b2 = rec[13] * args.adv[0] + rec[14] * args.adv[1] + rec[15] * args.adv[2];
                    mass += (t00 * b0 + t01 * b1 + t02 * b2) * v0 + (t11 * b1 + t12 * b2) * v1 + b2 * v2;
                }
                S2[e * NQ + r] = wl * rec[6] * mass;
                continue;
            }
            if (AFFINE) {
                const T* rec = args.geom + eg * 16;
                int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q;
                T Tm[3][3];
                deta_dxi<SHAPE, T>(zt[i], zt[Q + j], zt[2 * Q + k], Tm);
                T wl = wt[i] * wt[Q + j] * wt[2 * Q + k];
                wJ = wl * rec[6];
                if (need_gx) {
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            Gx[d][c] = Tm[d][0] * rec[7 + c] + Tm[d][1] * rec[10 + c] + Tm[d][2] * rec[13 + c];
                }
            } else {
                const T* gp = args.geom + eg * 7 * (int64_t)NQp + r;
                wJ = gp[6 * NQp];
                if (op == HP_LAPLACIAN || op == HP_HELMHOLTZ || adr) {
#pragma unroll
                    for (int f = 0; f < 6; ++f) G[f] = gp[f * NQp];
                }
                if (need_gx) {
                    const T* hp_ = args.dgeom + eg * 9 * (int64_t)NQp + r;
#pragma unroll
                    for (int d = 0; d < 3; ++d)
#pragma unroll
                        for (int c = 0; c < 3; ++c) Gx[d][c] = hp_[(3 * d + c) * NQp];
                }
            }
            T* u = S1 + e * 4 * NQ + r;
            T uval = u[0];
            if (op == HP_MASS || op == HP_IPRODUCT_WRT_BASE) {
                S2[e * NQ + r] = wJ * uval;
            } else if (op == HP_LAPLACIAN || op == HP_HELMHOLTZ || adr) {
                T v1 = u[NQ], v2 = u[2 * NQ], v3 = u[3 * NQ];
                u[NQ] = G[0] * v1 + G[1] * v2 + G[2] * v3;
                u[2 * NQ] = G[1] * v1 + G[3] * v2 + G[4] * v3;
                u[3 * NQ] = G[2] * v1 + G[4] * v2 + G[5] * v3;
                T mass = (op == HP_HELMHOLTZ || adr) ? args.lambda * uval : T(0);
                if (adr) {   // a . grad u = sum_d c_d du / d eta_d, c_d = sum_i a_i d eta_d / d x_i
                    const T c1 = Gx[0][0] * args.adv[0] + Gx[0][1] * args.adv[1] + Gx[0][2] * args.adv[2];
                    const T c2 = Gx[1][0] * args.adv[0] + Gx[1][1] * args.adv[1] + Gx[1][2] * args.adv[2];
                    const T c3 = Gx[2][0] * args.adv[0] + Gx[2][1] * args.adv[1] + Gx[2][2] * args.adv[2];
                    mass += c1 * v1 + c2 * v2 + c3 * v3;
                }
                S2[e * NQ + r] = wJ * mass;
            } else if (op == HP_PHYSDERIV) {
                T v1 = u[NQ], v2 = u[2 * NQ], v3 = u[3 * NQ];
                const int64_t o = args.phys_off[eg] + r;
#pragma unroll
                for (int c = 0; c < 3; ++c) args.out[c * args.n_phys_total + o] = Gx[0][c] * v1 + Gx[1][c] * v2 + Gx[2][c] * v3;
            } else {   // HP_IPRODUCT_WRT_DERIV_BASE: w_d = w|J| sum_i Gx[d][i] f_i
                T f1 = u[NQ], f2 = u[2 * NQ], f3 = u[3 * NQ];
#pragma unroll
                for (int d = 0; d < 3; ++d) u[(d + 1) * NQ] = wJ * (Gx[d][0] * f1 + Gx[d][1] * f2 + Gx[d][2] * f3);
                S2[e * NQ + r] = T(0);
            }
        }
        __syncthreads();
        if (op == HP_PHYSDERIV) continue;

        if constexpr (LINES) {
        if (sumderiv) {
            // u' = t + sum_d D_d^T w_d: one accumulating line pass per direction
            for (int idx = tid; idx < EPB * QQ; idx += NT) {     // eta1 lines (j,k)
                int e = idx / QQ, jk = idx - e * QQ;
                const T* w = S1 + e * 4 * NQ + NQ + jk;
                T x[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) x[m] = w[m * QQ];
                T* o = S2 + e * NQ + jk;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    T acc = o[i * QQ];
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc += args.cD[0][m * Q + i] * x[m];
                    o[i * QQ] = acc;
                }
            }
            __syncthreads();
            for (int idx = tid; idx < EPB * QQ; idx += NT) {     // eta2 lines (i,k)
                int e = idx / QQ, ik = idx - e * QQ, i = ik / Q, k = ik - i * Q;
                const T* w = S1 + e * 4 * NQ + 2 * NQ + i * QQ + k;
                T x[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) x[m] = w[m * Q];
                T* o = S2 + e * NQ + i * QQ + k;
#pragma unroll
                for (int j = 0; j < Q; ++j) {
                    T acc = o[j * Q];
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc += args.cD[1][m * Q + j] * x[m];
                    o[j * Q] = acc;
                }
            }
            __syncthreads();
            for (int idx = tid; idx < EPB * QQ; idx += NT) {     // eta3 lines (i,j)
                int e = idx / QQ, ij = idx - e * QQ;
                const T* w = S1 + e * 4 * NQ + 3 * NQ + ij * Q;
                T x[Q];
#pragma unroll
                for (int m = 0; m < Q; ++m) x[m] = w[m];
                T* o = S2 + e * NQ + ij * Q;
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    T acc = o[k];
#pragma unroll
                    for (int m = 0; m < Q; ++m) acc += args.cD[2][m * Q + k] * x[m];
                    o[k] = acc;
                }
            }
            __syncthreads();
        }

        } else {
        if (sumderiv) {
            // y = t + D_2^T w_2 + D_3^T w_3 in even-odd pairs (i, Q-1-i) along eta1,
            // stored as sums at i and differences at Q-1-i, and the same sweep of
            // w_1; the eta1 restriction applies [Tp | Td] to (y, w_1), which takes
            // the place of D_1^T w_1 (u' = y + D_1^T w_1)
            for (int idx = tid; idx < EPB * Qh * QQ; idx += NT) {
                int e = idx / (Qh * QQ), r = idx - e * (Qh * QQ);
                int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q, i2 = Q - 1 - i;
                const T* w = S1 + e * 4 * NQ;
                T* ys = S2 + e * NQ + jk;
                T y1 = ys[i * QQ], y2 = ys[i2 * QQ];
#pragma unroll
                for (int m = 0; m < Q; ++m) {
                    y1 += D1[m * Q + j] * w[2 * NQ + i * QQ + m * Q + k];
                    y1 += D2[m * Q + k] * w[3 * NQ + i * QQ + j * Q + m];
                    y2 += D1[m * Q + j] * w[2 * NQ + i2 * QQ + m * Q + k];
                    y2 += D2[m * Q + k] * w[3 * NQ + i2 * QQ + j * Q + m];
                }
                if (i2 != i) {
                    T* w1 = S1 + e * 4 * NQ + NQ + jk;
                    const T wa = w1[i * QQ], wb = w1[i2 * QQ];
                    ys[i * QQ] = y1 + y2;
                    ys[i2 * QQ] = y1 - y2;
                    w1[i * QQ] = wa + wb;
                    w1[i2 * QQ] = wa - wb;
                } else {
                    ys[i * QQ] = y1;
                }
            }
            __syncthreads();
        }

        }

        if (point_io) {
            for (int idx = tid; idx < EPB * NQ; idx += NT) {
                const int e = idx / NQ, r = idx - e * NQ;
                if (e < ne) args.out[args.phys_off[e0 + e] + r] = S2[e * NQ + r];
            }
            __syncthreads();
            continue;
        }
        if constexpr (LINES) {
        // restriction B^T: eta1 pass g'[a][j][k] = sum_i Ta[a][i] u'[i][j][k], one (j,k) line per thread
        for (int idx = tid; idx < EPB * QQ; idx += NT) {
            int e = idx / QQ, jk = idx - e * QQ;
            const T* x = S2 + e * NQ + jk;
            T uq[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) uq[i] = x[i * QQ];
            T* g = S1 + e * 4 * NQ + jk;
#pragma unroll
            for (int a = 0; a < n; ++a) {
                T acc = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) acc += args.cTa[a * Q + i] * uq[i];
                g[a * QQ] = acc;
            }
        }
        __syncthreads();
        } else if (sumderiv) {
        // restriction B^T along eta1 from the even-odd sweeps:
        // g'[a] = sum_{i < Qh} Tp[a][i] y^{+-}_i + Td[a][i] w_1^{-+}_i, the sum or
        // difference taken by the parity of the row (the middle point of odd Q
        // meets an exact zero in the row of the wrong parity)
        for (int idx = tid; idx < EPB * n * QQ; idx += NT) {
            int e = idx / (n * QQ), r = idx - e * (n * QQ);
            int a = r / QQ, jk = r - a * QQ;
            const bool even = (a & 1) == 0;
            const T* ys = S2 + e * NQ + jk;
            const T* ws = S1 + e * 4 * NQ + NQ + jk;
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < Qh; ++i) {
                const int iy = even ? i : Q - 1 - i, iw = even ? Q - 1 - i : i;
                acc += Ta[a * Q + i] * ys[iy * QQ];
                acc += Td[a * Q + i] * ws[iw * QQ];
            }
            S1[e * 4 * NQ + r] = acc;
        }
        __syncthreads();
        } else {
        // restriction B^T: eta1 pass g'[a][j][k] = sum_i Ta[a][i] u'[i][j][k]
        for (int idx = tid; idx < EPB * n * QQ; idx += NT) {
            int e = idx / (n * QQ), r = idx - e * (n * QQ);
            int a = r / QQ, jk = r - a * QQ;
            const T* x = S2 + e * NQ + jk;
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) acc += Ta[a * Q + i] * x[i * QQ];
            S1[e * 4 * NQ + r] = acc;
        }
        __syncthreads();
        }
        // eta2 pass over the valid pairs p = (a,b): f'[p][k] = sum_j Tb[t(a)][b][j] g'[a][j][k]
        for (int idx = tid; idx < EPB * NPR * Q; idx += NT) {
            int e = idx / (NPR * Q), r = idx - e * (NPR * Q);
            int p = r / Q, k = r - p * Q;
            int ab = p;
            if constexpr (SHAPE != 0) ab = pairs[p] & 0xffff;
            const int a = ab / n, b = ab - a * n;
            const T* tb = Tb + (famb[a] * n + b) * Q;
            const T* x = S1 + e * 4 * NQ + a * QQ + k;
            T acc = T(0);
#pragma unroll
            for (int j = 0; j < Q; ++j) acc += tb[j] * x[j * Q];
            S2[e * NQ + r] = acc;
        }
        __syncthreads();
        // eta3 pass over the valid slots (a,b,c): r[a][b][c] = sum_k Tc[s(a,b)][c][k] f'[p(a,b)][k]
        for (int idx = tid; idx < EPB * NVL; idx += NT) {
            int e = idx / NVL, v = idx - e * NVL;
            int sl = v, p = v / n, sc = 0, c = v - p * n;
            if constexpr (SHAPE != 0) {
                const int vv = valid[v];
                sl = vv & 2047; p = (vv >> 11) & 127; sc = (vv >> 18) & 15; c = (vv >> 22) & 15;
            }
            const T* tc = Tc + (sc * n + c) * Q;
            const T* x = S2 + e * NQ + p * Q;
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) acc += tc[k] * x[k];
            S1[e * 4 * NQ + sl] = acc;
        }
        __syncthreads();
        // scatter slots to modes (collapsed modes sum their slots)
        auto mode_sum = [&](int e, int m) {
            const T* rs = S1 + e * 4 * NQ;
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int sl = mode_slots[m * 4 + q];
                if (sl < 0) continue;
                // slots a = 0, 1 hold the restrictions against 1/2 and -z/2:
                // L = 1/2 - z/2 takes their sum, R = 1/2 + z/2 their difference
                if (sl >= 2 * NN) acc += rs[sl];
                else if (sl < NN) acc += rs[sl] + rs[sl + NN];
                else acc += rs[sl - NN] - rs[sl];
            }
            return acc;
        };
        if constexpr (LINES) {
            // FP32: the output offsets of kU modes per thread are loaded together
            for (int base = tid; base < EPB * NP; base += NT * kU) {
                int64_t off[kU];
                T acc[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int idx = base + u * NT, e = idx / NP, m = idx - e * NP;
                    off[u] = -1;
                    acc[u] = T(0);
                    if (idx < EPB * NP && e < ne) {
                        off[u] = __ldg(args.coeff_off + e0 + e) + m;
                        acc[u] = mode_sum(e, m);
                    }
                }
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (off[u] >= 0) args.out[off[u]] = acc[u];
            }
        } else
        for (int idx = tid; idx < EPB * NP; idx += NT) {
            int e = idx / NP, m = idx - e * NP;
            if (e >= ne) continue;
            const T* rs = S1 + e * 4 * NQ;
            T acc = T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int sl = mode_slots[m * 4 + q];
                if (sl < 0) continue;
                if (sl >= 2 * NN) acc += rs[sl];
                else if (sl < NN) acc += rs[sl] + rs[sl + NN];
                else acc += rs[sl - NN] - rs[sl];
            }
            args.out[args.coeff_off[e0 + e] + m] = acc;
        }
        __syncthreads();
    }
    return true;
}

// One launch per block: a persistent grid of CTAs over the block's element groups.
template <int SHAPE, int P, typename T, bool AFFINE, int TILE>
__global__ void __launch_bounds__(256, (sf_min_blocks<SHAPE, P, T, TILE>())) sf_kernel(const __grid_constant__ SFArgs<T> args) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(smem), 1);
    __syncthreads();
    uint32_t phase = 0;
    const int64_t ngroups = (args.n_elem + SFCfg<P, T, TILE>::EPB - 1) / SFCfg<P, T, TILE>::EPB;
    sf_groups<SHAPE, P, T, AFFINE, TILE>(args, smem, blockIdx.x, gridDim.x, ngroups, phase);
}

template <int SHAPE, int P, typename T, bool AFFINE, int TILE>
cudaError_t sf_launch_one(const SFArgs<T>& a, cudaStream_t s) {
    using C = SFCfg<P, T, TILE>;
    constexpr int smem = sf_smem_bytes<SHAPE, P, T, TILE>();
    static std::atomic<int> caps[kMaxDevices];
    auto kern = sf_kernel<SHAPE, P, T, AFFINE, TILE>;
    int grid_cap = 0;
    cudaError_t e = persistent_grid_cap(kern, C::NT, smem, caps, &grid_cap);
    if (e != cudaSuccess) return e;
    int64_t groups = (a.n_elem + C::EPB - 1) / C::EPB;
    int grid = (int)(groups < grid_cap ? groups : grid_cap);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, C::NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SHAPE, int P, typename T, bool AFFINE>
cudaError_t sf_launch_tile(int tile, const SFArgs<T>& a, cudaStream_t s) {
    switch (tile) {
        case 1: return sf_launch_one<SHAPE, P, T, AFFINE, 1>(a, s);
        case 2: return sf_launch_one<SHAPE, P, T, AFFINE, 2>(a, s);
        default: return sf_launch_one<SHAPE, P, T, AFFINE, 0>(a, s);
    }
}

// elements per CTA of a tile variant (host side, for the autotuner)
template <typename T>
int sf_epb(int P, int tile) {
#define HP_EPB(PP) \
    case PP: return tile == 1 ? SFCfg<PP, T, 1>::EPB : tile == 2 ? SFCfg<PP, T, 2>::EPB : SFCfg<PP, T, 0>::EPB;
    switch (P) {
        HP_EPB(1) HP_EPB(2) HP_EPB(3) HP_EPB(4) HP_EPB(5) HP_EPB(6) HP_EPB(7) HP_EPB(8) HP_EPB(9) HP_EPB(10)
        default: return 1;
    }
#undef HP_EPB
}

template <int SHAPE, typename T>
cudaError_t sf_dispatch(int P, bool affine, int tile, const SFArgs<T>& a, cudaStream_t s) {
#define HP_CASE(PP)                                                                             \
    case PP:                                                                                    \
        return affine ? sf_launch_tile<SHAPE, PP, T, true>(tile, a, s) : sf_launch_tile<SHAPE, PP, T, false>(tile, a, s);
    switch (P) {
        HP_CASE(1) HP_CASE(2) HP_CASE(3) HP_CASE(4) HP_CASE(5)
        HP_CASE(6) HP_CASE(7) HP_CASE(8) HP_CASE(9) HP_CASE(10)
        default: return cudaErrorInvalidValue;
    }
#undef HP_CASE
}

}  // namespace hp
