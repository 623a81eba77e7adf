// Elemental-matrix (StdMat) and hybrid strategies.
//
// Elemental matrix (paper Sec. 3.3.1, StdMat with reference-element matrices,
// and the non-collocated Helmholtz algorithm of Sec. 3.3, which the paper
// adopts for StdMat because the dense D_d B is smaller than D_d):
//   [u; v1; v2; v3] = [B; D1 B; D2 B; D3 B] uhat        (one dense product, A4)
//   w_d = sum_d' G_dd' v_d',  t = lambda w|J| u           (pointwise metric)
//   out = B^T t + sum_d (D_d B)^T w_d                     (one dense product, A4^T)
// per block of elements, with the element index as the wide dimension.  The
// kernel streams the points in chunks of 32: the forward product for a chunk
// (each thread one (quantity, point) row for 8 elements at once, A4^T read
// coalesced from L2), the metric, then the transposed product accumulated
// per mode in shared memory -- so the 4 N_Q intermediate rows never leave the
// chip (a fused GEMM-metric-GEMM).
//
// Hybrid (not in the paper): the restriction/expansion B, B^T as dense
// products and the derivatives collocated (D_d at the points), i.e. the
// collocated algorithm of Sec. 3.3 with the two sum-factorised passes replaced
// by dense reference-matrix products.
#include "hp_device.cuh"

namespace hp {
namespace {

template <int SHAPE, typename T, bool AFFINE>
__device__ __forceinline__ void point_metric(const T* geom, int64_t eg, int l, int NQp, int Q, const T* zt,
                                             const T* wt, bool need_G, T G[6], T& wJ) {
    if (AFFINE) {
        const T* rec = geom + eg * 16;
        int i = l / (Q * Q), j = (l / Q) % Q, k = l % Q;
        T Tm[3][3];
        deta_dxi<SHAPE, T>(zt[i], zt[Q + j], zt[2 * Q + k], Tm);
        T wl = wt[i] * wt[Q + j] * wt[2 * Q + k];
        wJ = wl * rec[6];
        if (need_G) {
            T K[3][3] = {{rec[0], rec[1], rec[2]}, {rec[1], rec[3], rec[4]}, {rec[2], rec[4], rec[5]}};
            T M[3][3];
            for (int d = 0; d < 3; ++d)
                for (int b = 0; b < 3; ++b) M[d][b] = Tm[d][0] * K[0][b] + Tm[d][1] * K[1][b] + Tm[d][2] * K[2][b];
            auto gg = [&](int d, int d2) { return wl * (M[d][0] * Tm[d2][0] + M[d][1] * Tm[d2][1] + M[d][2] * Tm[d2][2]); };
            G[0] = gg(0, 0); G[1] = gg(0, 1); G[2] = gg(0, 2); G[3] = gg(1, 1); G[4] = gg(1, 2); G[5] = gg(2, 2);
        }
    } else {
        const T* gp = geom + eg * 7 * (int64_t)NQp + l;
        wJ = gp[6 * NQp];
        if (need_G)
            for (int f = 0; f < 6; ++f) G[f] = gp[f * NQp];
    }
}

constexpr int kE = 8;     // elements per CTA (elemental matrix)
constexpr int kPC = 32;   // points per chunk
constexpr int kNT = 256;

template <int SHAPE, typename T, bool AFFINE>
__global__ void __launch_bounds__(kNT) emat_kernel(const EMArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    unsigned char* tab = smem + 16;
    const BlobLayout L = blob_layout_c(SHAPE, a.P, (int)sizeof(T));
    if (!stage_tables(tab, a.blob, L.total_bytes, bar, a.err)) return;
    const T* zt = reinterpret_cast<const T*>(tab) + L.z;
    const T* wt = reinterpret_cast<const T*>(tab) + L.w;
    const int NP = a.NP, NQ = a.NQ, op = a.op;
    T* uhT = reinterpret_cast<T*>(tab + L.total_bytes);   // [NP][E]
    T* acc = uhT + NP * kE;                               // [NP][E]
    T* V = acc + NP * kE;                                 // [4][PC][E]
    const int tid = threadIdx.x;
    const int nq = (op == HP_MASS || op == HP_BWDTRANS || op == HP_IPRODUCT_WRT_BASE) ? 1 : 4;
    const bool need_G = (op == HP_LAPLACIAN || op == HP_HELMHOLTZ);
    const int64_t ngroups = (a.n_elem + kE - 1) / kE;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e0 = g * kE;
        const int ne = (int)min((int64_t)kE, a.n_elem - e0);
        if (op != HP_IPRODUCT_WRT_BASE)
            for (int idx = tid; idx < NP * kE; idx += kNT) {
                int e = idx / NP, m = idx - e * NP;
                uhT[m * kE + e] = e < ne ? a.in[a.coeff_off[e0 + e] + m] : T(0);
            }
        for (int idx = tid; idx < NP * kE; idx += kNT) acc[idx] = T(0);
        __syncthreads();
        for (int l0 = 0; l0 < NQ; l0 += kPC) {
            const int pc = min(kPC, NQ - l0);
            if (op == HP_IPRODUCT_WRT_BASE) {
                for (int idx = tid; idx < pc * kE; idx += kNT) {
                    int e = idx / pc, p = idx - e * pc;
                    V[p * kE + e] = e < ne ? a.in[a.phys_off[e0 + e] + l0 + p] : T(0);
                }
            } else {
                for (int r = tid; r < nq * pc; r += kNT) {
                    int q = r / pc, p = r - q * pc;
                    T s[kE];
#pragma unroll
                    for (int e = 0; e < kE; ++e) s[e] = T(0);
                    const T* col = a.A4T + (int64_t)q * NQ + l0 + p;
                    for (int m = 0; m < NP; ++m) {
                        T av = col[(int64_t)m * 4 * NQ];
#pragma unroll
                        for (int e = 0; e < kE; ++e) s[e] += av * uhT[m * kE + e];
                    }
#pragma unroll
                    for (int e = 0; e < kE; ++e) V[(q * kPC + p) * kE + e] = s[e];
                }
            }
            __syncthreads();
            if (op == HP_BWDTRANS) {
                for (int idx = tid; idx < pc * kE; idx += kNT) {
                    int e = idx / pc, p = idx - e * pc;
                    if (e < ne) a.out[a.phys_off[e0 + e] + l0 + p] = V[p * kE + e];
                }
                __syncthreads();
                continue;
            }
            for (int idx = tid; idx < pc * kE; idx += kNT) {
                int p = idx / kE, e = idx - p * kE;
                if (e >= ne) {
                    for (int q = 0; q < nq; ++q) V[(q * kPC + p) * kE + e] = T(0);
                    continue;
                }
                T G[6], wJ;
                point_metric<SHAPE, T, AFFINE>(a.geom, e0 + e, l0 + p, a.NQp, a.Q, zt, wt, need_G, G, wJ);
                T* v = V + p * kE + e;
                if (!need_G) {
                    v[0] = wJ * v[0];
                } else {
                    T v1 = v[kPC * kE], v2 = v[2 * kPC * kE], v3 = v[3 * kPC * kE];
                    v[kPC * kE] = G[0] * v1 + G[1] * v2 + G[2] * v3;
                    v[2 * kPC * kE] = G[1] * v1 + G[3] * v2 + G[4] * v3;
                    v[3 * kPC * kE] = G[2] * v1 + G[4] * v2 + G[5] * v3;
                    v[0] = (op == HP_HELMHOLTZ) ? a.lambda * wJ * v[0] : T(0);
                }
            }
            __syncthreads();
            for (int m = tid; m < NP; m += kNT) {
                T s[kE];
#pragma unroll
                for (int e = 0; e < kE; ++e) s[e] = T(0);
                for (int q = 0; q < nq; ++q) {
                    const T* rowp = a.A4 + ((int64_t)q * NQ + l0) * NP + m;
                    for (int p = 0; p < pc; ++p) {
                        T av = rowp[(int64_t)p * NP];
                        const T* vv = V + (q * kPC + p) * kE;
#pragma unroll
                        for (int e = 0; e < kE; ++e) s[e] += av * vv[e];
                    }
                }
#pragma unroll
                for (int e = 0; e < kE; ++e) acc[m * kE + e] += s[e];
            }
            __syncthreads();
        }
        if (op != HP_BWDTRANS) {
            for (int idx = tid; idx < NP * kE; idx += kNT) {
                int e = idx / NP, m = idx - e * NP;
                if (e < ne) a.out[a.coeff_off[e0 + e] + m] = acc[m * kE + e];
            }
        }
        __syncthreads();
    }
}

// Hybrid: dense B / B^T, collocated derivatives.  E elements per CTA (runtime).
template <int SHAPE, typename T, bool AFFINE>
__global__ void __launch_bounds__(kNT) hyb_kernel(const EMArgs<T> a, int E) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    unsigned char* tab = smem + 16;
    const BlobLayout L = blob_layout_c(SHAPE, a.P, (int)sizeof(T));
    if (!stage_tables(tab, a.blob, L.total_bytes, bar, a.err)) return;
    const T* D0 = reinterpret_cast<const T*>(tab) + L.D;
    const int Q = a.Q, QQ = Q * Q, NQ = a.NQ, NP = a.NP, op = a.op;
    const T* D1 = D0 + QQ;
    const T* D2 = D0 + 2 * QQ;
    const T* zt = reinterpret_cast<const T*>(tab) + L.z;
    const T* wt = reinterpret_cast<const T*>(tab) + L.w;
    T* uh = reinterpret_cast<T*>(tab + L.total_bytes);   // [E][NP]
    T* S1 = uh + E * NP;                                  // [E][4 NQ]
    T* S2 = S1 + E * 4 * NQ;                              // [E][NQ]
    const int tid = threadIdx.x;
    const bool deriv = (op == HP_LAPLACIAN || op == HP_HELMHOLTZ);
    const int64_t ngroups = (a.n_elem + E - 1) / E;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e0 = g * E;
        const int ne = (int)min((int64_t)E, a.n_elem - e0);
        if (op == HP_IPRODUCT_WRT_BASE) {
            for (int idx = tid; idx < E * NQ; idx += kNT) {
                int e = idx / NQ, l = idx - e * NQ;
                S1[e * 4 * NQ + l] = e < ne ? a.in[a.phys_off[e0 + e] + l] : T(0);
            }
        } else {
            for (int idx = tid; idx < E * NP; idx += kNT) {
                int e = idx / NP, m = idx - e * NP;
                uh[idx] = e < ne ? a.in[a.coeff_off[e0 + e] + m] : T(0);
            }
            __syncthreads();
            // u[l] = sum_m B[l][m] uhat[m]   (B^T rows coalesced over l)
            for (int idx = tid; idx < E * NQ; idx += kNT) {
                int e = idx / NQ, l = idx - e * NQ;
                const T* col = a.A4T + l;
                const T* x = uh + e * NP;
                T s = T(0);
                for (int m = 0; m < NP; ++m) s += col[(int64_t)m * 4 * NQ] * x[m];
                S1[e * 4 * NQ + l] = s;
            }
        }
        __syncthreads();
        if (op == HP_BWDTRANS) {
            for (int idx = tid; idx < E * NQ; idx += kNT) {
                int e = idx / NQ, l = idx - e * NQ;
                if (e < ne) a.out[a.phys_off[e0 + e] + l] = S1[e * 4 * NQ + l];
            }
            __syncthreads();
            continue;
        }
        if (deriv) {
            for (int idx = tid; idx < E * NQ; idx += kNT) {
                int e = idx / NQ, r = idx - e * NQ;
                int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q;
                const T* u = S1 + e * 4 * NQ;
                T a1 = T(0), a2 = T(0), a3 = T(0);
                for (int m = 0; m < Q; ++m) {
                    a1 += D0[i * Q + m] * u[m * QQ + jk];
                    a2 += D1[j * Q + m] * u[i * QQ + m * Q + k];
                    a3 += D2[k * Q + m] * u[i * QQ + j * Q + m];
                }
                S1[e * 4 * NQ + NQ + r] = a1;
                S1[e * 4 * NQ + 2 * NQ + r] = a2;
                S1[e * 4 * NQ + 3 * NQ + r] = a3;
            }
            __syncthreads();
        }
        for (int idx = tid; idx < E * NQ; idx += kNT) {
            int e = idx / NQ, r = idx - e * NQ;
            if (e >= ne) {
                S2[e * NQ + r] = T(0);
                if (deriv) S1[e * 4 * NQ + NQ + r] = S1[e * 4 * NQ + 2 * NQ + r] = S1[e * 4 * NQ + 3 * NQ + r] = T(0);
                continue;
            }
            T G[6], wJ;
            point_metric<SHAPE, T, AFFINE>(a.geom, e0 + e, r, a.NQp, Q, zt, wt, deriv, G, wJ);
            T* u = S1 + e * 4 * NQ + r;
            if (!deriv) {
                S2[e * NQ + r] = wJ * u[0];
            } else {
                T v1 = u[NQ], v2 = u[2 * NQ], v3 = u[3 * NQ];
                u[NQ] = G[0] * v1 + G[1] * v2 + G[2] * v3;
                u[2 * NQ] = G[1] * v1 + G[3] * v2 + G[4] * v3;
                u[3 * NQ] = G[2] * v1 + G[4] * v2 + G[5] * v3;
                S2[e * NQ + r] = (op == HP_HELMHOLTZ) ? a.lambda * wJ * u[0] : T(0);
            }
        }
        __syncthreads();
        if (deriv) {
            for (int idx = tid; idx < E * NQ; idx += kNT) {
                int e = idx / NQ, r = idx - e * NQ;
                int i = r / QQ, jk = r - i * QQ, j = jk / Q, k = jk - j * Q;
                const T* w = S1 + e * 4 * NQ;
                T s = S2[e * NQ + r];
                for (int m = 0; m < Q; ++m) {
                    s += D0[m * Q + i] * w[NQ + m * QQ + jk];
                    s += D1[m * Q + j] * w[2 * NQ + i * QQ + m * Q + k];
                    s += D2[m * Q + k] * w[3 * NQ + i * QQ + j * Q + m];
                }
                S2[e * NQ + r] = s;
            }
            __syncthreads();
        }
        // out[m] = sum_l B[l][m] u'[l]   (B rows coalesced over m)
        for (int idx = tid; idx < E * NP; idx += kNT) {
            int e = idx / NP, m = idx - e * NP;
            if (e >= ne) continue;
            const T* x = S2 + e * NQ;
            T s = T(0);
            for (int l = 0; l < NQ; ++l) s += a.A4[(int64_t)l * NP + m] * x[l];
            a.out[a.coeff_off[e0 + e] + m] = s;
        }
        __syncthreads();
    }
}

// diag of (lambda M + L) of each element: sum over points of
// lambda w|J| B_lm^2 + sum_dd' G_dd' (D_d B)_lm (D_d' B)_lm; one thread per (element, mode)
template <int SHAPE, bool AFFINE>
__global__ void elem_diag_kernel(int64_t n_elem, int P, int Q, int NP, int NQp, const int64_t* __restrict__ coeff_off,
                                 const double* __restrict__ geom, const double* __restrict__ A4,
                                 const double* __restrict__ zt, const double* __restrict__ wt, double lambda,
                                 double* __restrict__ diag) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_elem * NP) return;
    int64_t e = idx / NP;
    int m = (int)(idx % NP);
    const int NQ = Q * Q * Q;
    double acc = 0.0;
    for (int l = 0; l < NQ; ++l) {
        double G[6], wJ;
        point_metric<SHAPE, double, AFFINE>(geom, e, l, NQp, Q, zt, wt, true, G, wJ);
        double b = A4[(int64_t)l * NP + m];
        double d1 = A4[((int64_t)NQ + l) * NP + m], d2 = A4[((int64_t)2 * NQ + l) * NP + m],
               d3 = A4[((int64_t)3 * NQ + l) * NP + m];
        acc += lambda * wJ * b * b + G[0] * d1 * d1 + G[3] * d2 * d2 + G[5] * d3 * d3 +
               2.0 * (G[1] * d1 * d2 + G[2] * d1 * d3 + G[4] * d2 * d3);
    }
    diag[coeff_off[e] + m] = acc;
}

template <typename K>
int grid_for(K kern, int smem, int64_t groups) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kNT, smem);
    int64_t cap = (int64_t)sms * (per > 0 ? per : 1);
    return (int)(groups < cap ? groups : cap);
}

template <int SHAPE, typename T, bool AFFINE>
cudaError_t launch_shape(bool hybrid, const EMArgs<T>& a, cudaStream_t s) {
    const BlobLayout L = blob_layout_c(SHAPE, a.P, (int)sizeof(T));
    if (!hybrid) {
        int smem = 16 + L.total_bytes + (2 * a.NP * kE + 4 * kPC * kE) * (int)sizeof(T);
        auto kern = emat_kernel<SHAPE, T, AFFINE>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int grid = grid_for(kern, smem, (a.n_elem + kE - 1) / kE);
        if (grid <= 0) return cudaSuccess;
        kern<<<grid, kNT, smem, s>>>(a);
        return cudaGetLastError();
    }
    const int per_elem = (a.NP + 5 * a.NQ) * (int)sizeof(T);
    int E = (64 * 1024) / per_elem;
    E = E < 1 ? 1 : (E > 32 ? 32 : E);
    int smem = 16 + L.total_bytes + E * per_elem;
    auto kern = hyb_kernel<SHAPE, T, AFFINE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int grid = grid_for(kern, smem, (a.n_elem + E - 1) / E);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, kNT, smem, s>>>(a, E);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_any(bool hybrid, bool affine, const EMArgs<T>& a, cudaStream_t s) {
    switch (a.shape * 2 + (affine ? 1 : 0)) {
        case 0: return launch_shape<HP_HEX, T, false>(hybrid, a, s);
        case 1: return launch_shape<HP_HEX, T, true>(hybrid, a, s);
        case 2: return launch_shape<HP_PRISM, T, false>(hybrid, a, s);
        case 3: return launch_shape<HP_PRISM, T, true>(hybrid, a, s);
        case 4: return launch_shape<HP_PYR, T, false>(hybrid, a, s);
        case 5: return launch_shape<HP_PYR, T, true>(hybrid, a, s);
        case 6: return launch_shape<HP_TET, T, false>(hybrid, a, s);
        default: return launch_shape<HP_TET, T, true>(hybrid, a, s);
    }
}

}  // namespace

cudaError_t launch_elem_diag(const Block& b, const DeviceBlobs& blob, double lambda, double* diag, cudaStream_t s) {
    if (b.n_elem == 0) return cudaSuccess;
    const int NP = n_modes(b.shape, b.P), Q = b.Q;
    const BlobLayout L = blob_layout_c(b.shape, b.P, 8);
    const double* zt = reinterpret_cast<const double*>(blob.d64) + L.z;
    const double* wt = reinterpret_cast<const double*>(blob.d64) + L.w;
    int nt = 128;
    unsigned nb = (unsigned)((b.n_elem * NP + nt - 1) / nt);
    const int NQp = nqp(Q);
#define HP_DIAG(S)                                                                                               \
    if (b.curved)                                                                                                \
        elem_diag_kernel<S, false><<<nb, nt, 0, s>>>(b.n_elem, b.P, Q, NP, NQp, b.d_coeff_off, b.d_geom,         \
                                                     blob.A4_64, zt, wt, lambda, diag);                          \
    else                                                                                                         \
        elem_diag_kernel<S, true><<<nb, nt, 0, s>>>(b.n_elem, b.P, Q, NP, NQp, b.d_coeff_off, b.d_geom,          \
                                                    blob.A4_64, zt, wt, lambda, diag);
    switch (b.shape) {
        case HP_HEX: HP_DIAG(HP_HEX) break;
        case HP_PRISM: HP_DIAG(HP_PRISM) break;
        case HP_PYR: HP_DIAG(HP_PYR) break;
        default: HP_DIAG(HP_TET)
    }
#undef HP_DIAG
    return cudaGetLastError();
}

cudaError_t emat_launch_f64(bool hybrid, bool affine, const EMArgs<double>& a, cudaStream_t s) {
    return launch_any<double>(hybrid, affine, a, s);
}
cudaError_t emat_launch_f32(bool hybrid, bool affine, const EMArgs<float>& a, cudaStream_t s) {
    return launch_any<float>(hybrid, affine, a, s);
}

}  // namespace hp
