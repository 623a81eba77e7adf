// Non-collocated sum-factorised Laplacian / Helmholtz in FP64: the form the
// paper's collocation study (Sec. 5, "Maximising collocation-based
// operations") compares the collocated approach against.
//
// The derivatives are taken by sum factorisation with the derivative tables
// instead of by collocation at the quadrature points:
//   u   = A  (B  (C  uhat))        v_1 = A' (B  (C  uhat))
//   v_2 = A  (B' (C  uhat))        v_3 = A  (B  (C' uhat))
// (A, B, C the eta1, eta2, eta3 factor tables, primes their derivatives), then
// the same pointwise metric as the collocated kernel, and the transposed
// passes
//   out = C^T [B^T (A^T t + A'^T w_1) + B'^T (A^T w_2)] + C'^T [B^T (A^T w_3)].
// The eta3 and eta2 contractions are shared where the products allow: two
// eta3 contractions (C, C') in one pass, three eta2 contractions (B f, B' f,
// B f') in one pass and four eta1 contractions in three passes forward; the
// mirror image backward.
// Collocated and non-collocated results agree up to rounding: each 1-D factor
// has degree <= P < Q, so collocation differentiation of its values is exact.
//
// One kernel per (shape, P, affine), FP64 only; one output entry per thread
// over a group of EPB elements, intermediates in shared memory; the eta1
// passes use the even-odd symmetry of the parity-form table (one product sum
// gives the values at i and Q-1-i) like the collocated FP64 kernel.
#include "hp_device.cuh"

namespace hp {
namespace {

constexpr int kNcBudget = 56 * 1024;   // shared memory for the element group

template <int P>
struct NCCfg {
    static constexpr int n = P + 1, Q = P + 2, QQ = Q * Q, NQ = Q * Q * Q, N3 = n * n * n;
    static constexpr int NT = 256;
    static constexpr int per_elem_bytes = 5 * NQ * 8;
    static constexpr int epb0 = kNcBudget / per_elem_bytes;
    static constexpr int EPB = epb0 < 1 ? 1 : (epb0 > 64 ? 64 : epb0);
    static constexpr int dtab_vals = 2 * (P + 1) * n * Q;   // [Tbd | Tcd]
};

template <int SHAPE, int P>
constexpr int nc_smem_bytes() {
    return 16 + blob_layout_c(SHAPE, P, 8).total_bytes + align16c(NCCfg<P>::dtab_vals * 8) +
           NCCfg<P>::EPB * 5 * NCCfg<P>::NQ * 8;
}

template <int SHAPE, int P, bool AFFINE>
__global__ void __launch_bounds__(256) sf_nc_kernel(const __grid_constant__ SFArgs<double> args, const double* dtab) {
    using C = NCCfg<P>;
    constexpr int n = C::n, Q = C::Q, QQ = C::QQ, NQ = C::NQ, N3 = C::N3, EPB = C::EPB, NT = C::NT;
    constexpr int NN = n * n, Qh = (Q + 1) / 2;
    constexpr BlobLayout L = blob_layout_c(SHAPE, P, 8);
    constexpr int NP = n_modes_c(SHAPE, P);
    constexpr int NQp = (NQ + 3) & ~3;
    constexpr int NPR = SHAPE == 0 ? n * n : npairs_c(SHAPE, P);
    constexpr int NVL = SHAPE == 0 ? N3 : nvalid_c(SHAPE, P);

    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    unsigned char* tab = smem + 16;
    if (!stage_tables(tab, args.blob, L.total_bytes, bar, args.err)) return;
    double* Tbd = reinterpret_cast<double*>(tab + L.total_bytes);
    double* Tcd = Tbd + (P + 1) * n * Q;
    for (int i = threadIdx.x; i < C::dtab_vals; i += NT) Tbd[i] = dtab[i];

    const double* Ta = reinterpret_cast<const double*>(tab) + L.Ta;   // parity form, row a of parity (-1)^a
    const double* Td = reinterpret_cast<const double*>(tab) + L.Td;   // its derivative, parity (-1)^(a+1)
    const double* Tb = reinterpret_cast<const double*>(tab) + L.Tb;
    const double* Tc = reinterpret_cast<const double*>(tab) + L.Tc;
    const double* zt = reinterpret_cast<const double*>(tab) + L.z;
    const double* wt = reinterpret_cast<const double*>(tab) + L.w;
    const uint8_t* famb = tab + L.famb;
    const int16_t* slot2mode = reinterpret_cast<const int16_t*>(tab + L.slot2mode);
    const int16_t* mode_slots = reinterpret_cast<const int16_t*>(tab + L.mode_slots);
    const int32_t* pairs = reinterpret_cast<const int32_t*>(tab + L.pairs);
    const int32_t* valid = reinterpret_cast<const int32_t*>(tab + L.valid);
    const int16_t* poff = reinterpret_cast<const int16_t*>(tab + L.poff);
    double* X = reinterpret_cast<double*>(tab + L.total_bytes + align16c(C::dtab_vals * 8));   // [EPB][5][NQ]
    __syncthreads();

    const int tid = threadIdx.x;
    const bool helm = args.op == HP_HELMHOLTZ;
    const int64_t ngroups = (args.n_elem + EPB - 1) / EPB;
    auto buf = [&](int e, int k) { return X + (e * 5 + k) * NQ; };

    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e0 = g * EPB;
        const int ne = (int)min((int64_t)EPB, args.n_elem - e0);

        // coefficients into the slot tensor (slots a = 0, 1: sum and difference
        // of the two coefficients, the inputs of the parity-form eta1 table) -> X4
        for (int idx = tid; idx < EPB * N3; idx += NT) {
            const int e = idx / N3, sl = idx - e * N3;
            double v = 0.0;
            const int m = slot2mode[sl];
            if (e < ne && m >= 0) {
                const double* cin = args.in + args.coeff_off[e0 + e];
                if (sl >= 2 * NN) v = cin[m];
                else if (sl < NN) v = cin[m] + cin[slot2mode[sl + NN]];
                else v = cin[slot2mode[sl - NN]] - cin[m];
            }
            buf(e, 4)[sl] = v;
        }
        __syncthreads();
        // eta3: f = C uhat -> X0, f' = C' uhat -> X1, per valid (a, b) pair
        for (int idx = tid; idx < EPB * NPR * Q; idx += NT) {
            const int e = idx / (NPR * Q), r = idx - e * (NPR * Q), p = r / Q, k = r - p * Q;
            int ab = p, sc = 0, len = n;
            if constexpr (SHAPE != 0) {
                const int pr = pairs[p];
                ab = pr & 0xffff; sc = (pr >> 16) & 0xff; len = pr >> 24;
            }
            const double* x = buf(e, 4) + ab * n;
            const double* tc = Tc + sc * n * Q + k;
            const double* td = Tcd + sc * n * Q + k;
            double f = 0.0, fd = 0.0;
#pragma unroll
            for (int c = 0; c < n; ++c) {
                if (c >= len) break;
                f += tc[c * Q] * x[c];
                fd += td[c * Q] * x[c];
            }
            buf(e, 0)[r] = f;
            buf(e, 1)[r] = fd;
        }
        __syncthreads();
        // eta2: g = B f -> X2, g2 = B' f -> X3, g3 = B f' -> X4, at [a][j][k]
        for (int idx = tid; idx < EPB * n * QQ; idx += NT) {
            const int e = idx / (n * QQ), r = idx - e * (n * QQ), a = r / QQ, jk = r - a * QQ;
            const int j = jk / Q, k = jk - j * Q;
            int p0 = a * n, lb = n;
            if constexpr (SHAPE != 0) { p0 = poff[a]; lb = poff[a + 1] - p0; }
            const double* tb = Tb + famb[a] * n * Q + j;
            const double* tbd = Tbd + famb[a] * n * Q + j;
            const double* f = buf(e, 0) + p0 * Q + k;
            const double* fd = buf(e, 1) + p0 * Q + k;
            double g0 = 0.0, g2 = 0.0, g3 = 0.0;
#pragma unroll
            for (int b = 0; b < n; ++b) {
                if (b >= lb) break;
                g0 += tb[b * Q] * f[b * Q];
                g2 += tbd[b * Q] * f[b * Q];
                g3 += tb[b * Q] * fd[b * Q];
            }
            buf(e, 2)[r] = g0;
            buf(e, 3)[r] = g2;
            buf(e, 4)[r] = g3;
        }
        __syncthreads();
        // eta1 in even-odd pairs (i, Q-1-i): u = A g -> X0 and v1 = A' g -> X1
        for (int idx = tid; idx < EPB * Qh * QQ; idx += NT) {
            const int e = idx / (Qh * QQ), r = idx - e * (Qh * QQ), i = r / QQ, jk = r - i * QQ, i2 = Q - 1 - i;
            const double* x = buf(e, 2) + jk;
            double ev = 0.0, od = 0.0, dv = 0.0, dd = 0.0;
#pragma unroll
            for (int a = 0; a < n; a += 2) ev += Ta[a * Q + i] * x[a * QQ];
#pragma unroll
            for (int a = 1; a < n; a += 2) od += Ta[a * Q + i] * x[a * QQ];
#pragma unroll
            for (int a = 1; a < n; a += 2) dv += Td[a * Q + i] * x[a * QQ];
#pragma unroll
            for (int a = 2; a < n; a += 2) dd += Td[a * Q + i] * x[a * QQ];
            double* u = buf(e, 0) + jk;
            double* v1 = buf(e, 1) + jk;
            u[i * QQ] = ev + od;
            v1[i * QQ] = dv + dd;
            if (i2 != i) { u[i2 * QQ] = ev - od; v1[i2 * QQ] = dv - dd; }
        }
        __syncthreads();
        // eta1: v2 = A g2 -> X2, then v3 = A g3 -> X3
        for (int pass = 0; pass < 2; ++pass) {
            for (int idx = tid; idx < EPB * Qh * QQ; idx += NT) {
                const int e = idx / (Qh * QQ), r = idx - e * (Qh * QQ), i = r / QQ, jk = r - i * QQ, i2 = Q - 1 - i;
                const double* x = buf(e, 3 + pass) + jk;
                double ev = 0.0, od = 0.0;
#pragma unroll
                for (int a = 0; a < n; a += 2) ev += Ta[a * Q + i] * x[a * QQ];
#pragma unroll
                for (int a = 1; a < n; a += 2) od += Ta[a * Q + i] * x[a * QQ];
                double* v = buf(e, 2 + pass) + jk;
                v[i * QQ] = ev + od;
                if (i2 != i) v[i2 * QQ] = ev - od;
            }
            __syncthreads();
        }
        // pointwise metric: w_d = sum_d' G_dd' v_d' in place (X1..X3), t = lambda w|J| u -> X4
        for (int idx = tid; idx < EPB * NQ; idx += NT) {
            const int e = idx / NQ, r = idx - e * NQ;
            double* u = buf(e, 0) + r;
            if (e >= ne) {
                u[NQ] = 0.0; u[2 * NQ] = 0.0; u[3 * NQ] = 0.0; u[4 * NQ] = 0.0;
                continue;
            }
            const int64_t eg = e0 + e;
            double G[6], wJ;
            if constexpr (AFFINE) {
                const double* rec = args.geom + eg * 16;
                const int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q;
                double Tm[3][3];
                deta_dxi<SHAPE, double>(zt[i], zt[Q + j], zt[2 * Q + k], Tm);
                const double wl = wt[i] * wt[Q + j] * wt[2 * Q + k];
                wJ = wl * rec[6];
                const double K[3][3] = {{rec[0], rec[1], rec[2]}, {rec[1], rec[3], rec[4]}, {rec[2], rec[4], rec[5]}};
                double M[3][3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int b = 0; b < 3; ++b) M[d][b] = Tm[d][0] * K[0][b] + Tm[d][1] * K[1][b] + Tm[d][2] * K[2][b];
                auto gg = [&](int d, int d2) { return wl * (M[d][0] * Tm[d2][0] + M[d][1] * Tm[d2][1] + M[d][2] * Tm[d2][2]); };
                G[0] = gg(0, 0); G[1] = gg(0, 1); G[2] = gg(0, 2); G[3] = gg(1, 1); G[4] = gg(1, 2); G[5] = gg(2, 2);
            } else {
                const double* gp = args.geom + eg * 7 * (int64_t)NQp + r;
#pragma unroll
                for (int f = 0; f < 6; ++f) G[f] = gp[f * NQp];
                wJ = gp[6 * NQp];
            }
            const double v1 = u[NQ], v2 = u[2 * NQ], v3 = u[3 * NQ];
            u[NQ] = G[0] * v1 + G[1] * v2 + G[2] * v3;
            u[2 * NQ] = G[1] * v1 + G[3] * v2 + G[4] * v3;
            u[3 * NQ] = G[2] * v1 + G[4] * v2 + G[5] * v3;
            u[4 * NQ] = helm ? args.lambda * wJ * u[0] : 0.0;
        }
        __syncthreads();
        // t, w1, w2, w3 along eta1 into sums (at i) and differences (at Q-1-i),
        // the inputs of the parity-form transposed tables
        for (int idx = tid; idx < EPB * 4 * (Q / 2) * QQ; idx += NT) {
            const int e = idx / (4 * (Q / 2) * QQ), r = idx - e * (4 * (Q / 2) * QQ);
            const int c = r / ((Q / 2) * QQ), r2 = r - c * ((Q / 2) * QQ), i = r2 / QQ, jk = r2 - i * QQ;
            double* y = buf(e, 1 + c) + jk;
            const double ya = y[i * QQ], yb = y[(Q - 1 - i) * QQ];
            y[i * QQ] = ya + yb;
            y[(Q - 1 - i) * QQ] = ya - yb;
        }
        __syncthreads();
        // transposed eta1: h0 = A^T t + A'^T w1 -> X0 (row a of A takes the sums
        // for even a and the differences for odd a, A' the other way round; the
        // middle point of odd Q meets an exact zero in the row of the wrong parity)
        for (int idx = tid; idx < EPB * n * QQ; idx += NT) {
            const int e = idx / (n * QQ), r = idx - e * (n * QQ), a = r / QQ, jk = r - a * QQ;
            const bool even = (a & 1) == 0;
            const double* t = buf(e, 4) + jk;
            const double* w1 = buf(e, 1) + jk;
            double acc = 0.0;
#pragma unroll
            for (int i = 0; i < Qh; ++i) {
                const int is = even ? i : Q - 1 - i, id = even ? Q - 1 - i : i;
                acc += Ta[a * Q + i] * t[is * QQ];
                acc += Td[a * Q + i] * w1[id * QQ];
            }
            buf(e, 0)[r] = acc;
        }
        __syncthreads();
        // transposed eta1: h2 = A^T w2 -> X1, h3 = A^T w3 -> X4
        for (int idx = tid; idx < EPB * n * QQ; idx += NT) {
            const int e = idx / (n * QQ), r = idx - e * (n * QQ), a = r / QQ, jk = r - a * QQ;
            const bool even = (a & 1) == 0;
            const double* w2 = buf(e, 2) + jk;
            const double* w3 = buf(e, 3) + jk;
            double h2 = 0.0, h3 = 0.0;
#pragma unroll
            for (int i = 0; i < Qh; ++i) {
                const int is = even ? i : Q - 1 - i;
                h2 += Ta[a * Q + i] * w2[is * QQ];
                h3 += Ta[a * Q + i] * w3[is * QQ];
            }
            buf(e, 1)[r] = h2;
            buf(e, 4)[r] = h3;
        }
        __syncthreads();
        // transposed eta2 over the valid pairs: k0 = B^T h0 + B'^T h2 -> X2, k3 = B^T h3 -> X3
        for (int idx = tid; idx < EPB * NPR * Q; idx += NT) {
            const int e = idx / (NPR * Q), r = idx - e * (NPR * Q), p = r / Q, k = r - p * Q;
            int ab = p;
            if constexpr (SHAPE != 0) ab = pairs[p] & 0xffff;
            const int a = ab / n, b = ab - a * n;
            const double* tb = Tb + (famb[a] * n + b) * Q;
            const double* tbd = Tbd + (famb[a] * n + b) * Q;
            const double* h0 = buf(e, 0) + a * QQ + k;
            const double* h2 = buf(e, 1) + a * QQ + k;
            const double* h3 = buf(e, 4) + a * QQ + k;
            double k0 = 0.0, k3 = 0.0;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                k0 += tb[j] * h0[j * Q] + tbd[j] * h2[j * Q];
                k3 += tb[j] * h3[j * Q];
            }
            buf(e, 2)[r] = k0;
            buf(e, 3)[r] = k3;
        }
        __syncthreads();
        // transposed eta3 over the valid slots: r = C^T k0 + C'^T k3 -> X0
        for (int idx = tid; idx < EPB * NVL; idx += NT) {
            const int e = idx / NVL, v = idx - e * NVL;
            int sl = v, p = v / n, sc = 0, c = v - p * n;
            if constexpr (SHAPE != 0) {
                const int vv = valid[v];
                sl = vv & 2047; p = (vv >> 11) & 127; sc = (vv >> 18) & 15; c = (vv >> 22) & 15;
            }
            const double* tc = Tc + (sc * n + c) * Q;
            const double* td = Tcd + (sc * n + c) * Q;
            const double* k0 = buf(e, 2) + p * Q;
            const double* k3 = buf(e, 3) + p * Q;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) acc += tc[k] * k0[k] + td[k] * k3[k];
            buf(e, 0)[sl] = acc;
        }
        __syncthreads();
        // slots to modes (the collapsed modes sum their slots; slots a = 0, 1 hold
        // the restrictions against 1/2 and -z/2: L takes their sum, R their difference)
        for (int idx = tid; idx < EPB * NP; idx += NT) {
            const int e = idx / NP, m = idx - e * NP;
            if (e >= ne) continue;
            const double* rs = buf(e, 0);
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sl = mode_slots[m * 4 + q];
                if (sl < 0) continue;
                if (sl >= 2 * NN) acc += rs[sl];
                else if (sl < NN) acc += rs[sl] + rs[sl + NN];
                else acc += rs[sl - NN] - rs[sl];
            }
            args.out[args.coeff_off[e0 + e] + m] = acc;
        }
        __syncthreads();
    }
}

template <int SHAPE, int P, bool AFFINE>
cudaError_t nc_launch_one(const SFArgs<double>& a, const double* dtab, cudaStream_t s) {
    constexpr int smem = nc_smem_bytes<SHAPE, P>();
    static_assert(smem <= 227 * 1024, "non-collocated kernel: shared memory above the per-CTA limit");
    static std::atomic<int> caps[kMaxDevices];
    auto kern = sf_nc_kernel<SHAPE, P, AFFINE>;
    int grid_cap = 0;
    cudaError_t e = persistent_grid_cap(kern, NCCfg<P>::NT, smem, caps, &grid_cap);
    if (e != cudaSuccess) return e;
    const int64_t groups = (a.n_elem + NCCfg<P>::EPB - 1) / NCCfg<P>::EPB;
    const int grid = (int)(groups < grid_cap ? groups : grid_cap);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, NCCfg<P>::NT, smem, s>>>(a, dtab);
    return cudaGetLastError();
}

template <int SHAPE>
cudaError_t nc_dispatch(int P, bool affine, const SFArgs<double>& a, const double* dtab, cudaStream_t s) {
#define HP_NC_CASE(PP) \
    case PP: return affine ? nc_launch_one<SHAPE, PP, true>(a, dtab, s) : nc_launch_one<SHAPE, PP, false>(a, dtab, s);
    switch (P) {
        HP_NC_CASE(1) HP_NC_CASE(2) HP_NC_CASE(3) HP_NC_CASE(4) HP_NC_CASE(5)
        HP_NC_CASE(6) HP_NC_CASE(7) HP_NC_CASE(8) HP_NC_CASE(9) HP_NC_CASE(10)
        default: return cudaErrorInvalidValue;
    }
#undef HP_NC_CASE
}

}  // namespace

cudaError_t sf_nc_launch(int shape, int P, bool affine, const SFArgs<double>& a, const double* dtab, cudaStream_t s) {
    if (a.op != HP_LAPLACIAN && a.op != HP_HELMHOLTZ) return cudaErrorInvalidValue;
    switch (shape) {
        case HP_HEX: return nc_dispatch<HP_HEX>(P, affine, a, dtab, s);
        case HP_PRISM: return nc_dispatch<HP_PRISM>(P, affine, a, dtab, s);
        case HP_PYR: return nc_dispatch<HP_PYR>(P, affine, a, dtab, s);
        case HP_TET: return nc_dispatch<HP_TET>(P, affine, a, dtab, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace hp
