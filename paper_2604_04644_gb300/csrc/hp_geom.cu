// Geometric factors in FP64 (paper Sec. 2.1: chain rule grad_x = J^{-T}
// grad_xi; Sec. 2.3: grad_xi = T grad_eta on collapsed coordinates; Sec. 4:
// deformed elements load six metric terms and the Jacobian at every point).
//
// Curved element, per quadrature point l (eta_l, xi_l = xi(eta_l)):
//   y = X0 + E (xi + 1)/2, J = D Phi(y) E/2,  d xi / d x = J^{-1},
//   Gx[d][i] = d eta_d / d x_i = sum_a T[d][a] (J^{-1})[a][i],
//   w|J| = w_l det J,  G_dd' = w|J| sum_i Gx[d][i] Gx[d'][i];
// stored as [elem][7][NQp] (G11 G12 G13 G22 G23 G33 w|J|) and, for the
// derivative building blocks, [elem][9][NQp] (Gx row-major).
// Affine element: per element K = |J| J^{-1} J^{-T} (6), |J| and J^{-1} (9).
// Iso-parametric curved element: J from the degree-P expansion of the map
// (geom_iso_kernel), the factors as above.
#include <algorithm>

#include "hp_device.cuh"

namespace hp {
namespace {

__device__ void deform_jacobian(int kind, const double y[3], double Dphi[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Dphi[i][j] = (i == j) ? 1.0 : 0.0;
    if (kind == 2) {   // Phi_i = x_i + 0.1 x_j x_k
        Dphi[0][1] = 0.1 * y[2]; Dphi[0][2] = 0.1 * y[1];
        Dphi[1][2] = 0.1 * y[0]; Dphi[1][0] = 0.1 * y[2];
        Dphi[2][0] = 0.1 * y[1]; Dphi[2][1] = 0.1 * y[0];
        return;
    }
    if (kind != 1) return;
    double s[3], c[3];
    for (int i = 0; i < 3; ++i) sincospi(y[i], &s[i], &c[i]);
    const double a = 0.05 * 3.14159265358979323846;
    // Phi_1 = x1 + 0.05 s2 s3, Phi_2 = x2 + 0.05 s3 s1, Phi_3 = x3 + 0.05 s1 s2
    Dphi[0][1] = a * c[1] * s[2];
    Dphi[0][2] = a * s[1] * c[2];
    Dphi[1][2] = a * c[2] * s[0];
    Dphi[1][0] = a * s[2] * c[0];
    Dphi[2][0] = a * c[0] * s[1];
    Dphi[2][1] = a * s[0] * c[1];
}

__device__ double inv3(const double J[3][3], double Ji[3][3]) {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    double r = 1.0 / det;
    Ji[0][0] = c00 * r;
    Ji[1][0] = c01 * r;
    Ji[2][0] = c02 * r;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
    return det;
}

// The factors of point l of element e from J = d x / d xi there: G_dd',
// w|J| (wl = the point's reference weight) and, if asked, d eta / d x.
template <int SHAPE>
__device__ void store_factors(const double J[3][3], double e1, double e2, double e3, double wl, int64_t e, int l,
                              int NQp, int want_deriv, double* __restrict__ geom, double* __restrict__ dgeom,
                              unsigned int* err, int* bad_elem) {
    double Ji[3][3];
    const double det = inv3(J, Ji);
    if (!(det > 0.0)) {
        atomicOr(err, DERR_GEOM);
        atomicMin(bad_elem, (int)e);
        return;
    }
    double T[3][3];
    deta_dxi<SHAPE, double>(e1, e2, e3, T);
    double Gx[3][3];
    for (int d = 0; d < 3; ++d)
        for (int c = 0; c < 3; ++c) Gx[d][c] = T[d][0] * Ji[0][c] + T[d][1] * Ji[1][c] + T[d][2] * Ji[2][c];
    const double wJ = wl * det;
    auto dot = [&](int a, int b) { return wJ * (Gx[a][0] * Gx[b][0] + Gx[a][1] * Gx[b][1] + Gx[a][2] * Gx[b][2]); };
    double* g = geom + e * 7 * (int64_t)NQp + l;
    g[0 * NQp] = dot(0, 0);
    g[1 * NQp] = dot(0, 1);
    g[2 * NQp] = dot(0, 2);
    g[3 * NQp] = dot(1, 1);
    g[4 * NQp] = dot(1, 2);
    g[5 * NQp] = dot(2, 2);
    g[6 * NQp] = wJ;
    if (want_deriv) {
        double* h = dgeom + e * 9 * (int64_t)NQp + l;
        for (int d = 0; d < 3; ++d)
            for (int c = 0; c < 3; ++c) h[(3 * d + c) * NQp] = Gx[d][c];
    }
}

// x = Phi(A_e(xi)) at a reference point: A_e from the element frame, Phi the deformation
__device__ __forceinline__ void map_point(int kind, const double* F, const double xi[3], double o[3]) {
    double y[3];
    for (int r = 0; r < 3; ++r) {
        y[r] = F[r];
        for (int d = 0; d < 3; ++d) y[r] += F[3 + r * 3 + d] * 0.5 * (xi[d] + 1.0);
    }
    o[0] = y[0]; o[1] = y[1]; o[2] = y[2];
    if (kind == 1) {
        double sn[3], cs[3];
        for (int r = 0; r < 3; ++r) sincospi(y[r], &sn[r], &cs[r]);
        o[0] += 0.05 * sn[1] * sn[2];
        o[1] += 0.05 * sn[2] * sn[0];
        o[2] += 0.05 * sn[0] * sn[1];
    } else if (kind == 2) {
        o[0] += 0.1 * y[1] * y[2];
        o[1] += 0.1 * y[2] * y[0];
        o[2] += 0.1 * y[0] * y[1];
    }
}

// Iso-parametric geometry of a curved element: the map's values at the Q^3
// points projected onto the element's degree-P expansion (coefficients c = S x
// in functions orthonormal in the reference quadrature, S^T in RT [point][mode];
// projected values V c, VT [mode][point]), then d x / d eta_d by collocation
// differentiation of the projected values along each eta line (exact: the
// projection has degree <= P < Q in each eta) and d x / d xi = (d x / d eta)
// (d eta / d xi).  One CTA per element (grid stride); shared memory holds the
// element's 3 Q^3 values and 3 N_P coefficients.
template <int SHAPE>
__global__ void __launch_bounds__(256) geom_iso_kernel(int Q, int NP, int NQp, int64_t n_elem,
                                                       const double* __restrict__ frame, const double* __restrict__ z,
                                                       const double* __restrict__ w, const double* __restrict__ Dt,
                                                       int kind, const double* __restrict__ RT,
                                                       const double* __restrict__ VT, int want_deriv,
                                                       double* __restrict__ geom, double* __restrict__ dgeom,
                                                       unsigned int* err, int* bad_elem) {
    extern __shared__ __align__(16) double gsm[];
    const int NQ = Q * Q * Q, QQ = Q * Q;
    double* xq = gsm;              // [3][NQ]: the map's values, then the projected values
    double* xh = gsm + 3 * NQ;     // [3][NP]
    for (int64_t e = blockIdx.x; e < n_elem; e += gridDim.x) {
        const double* F = frame + e * 12;
        for (int l = threadIdx.x; l < NQ; l += blockDim.x) {
            const int i = l / QQ, j = (l / Q) % Q, k = l % Q;
            double xi[3], o[3];
            xi_from_eta<SHAPE>(z[i], z[Q + j], z[2 * Q + k], xi);
            map_point(kind, F, xi, o);
            for (int c = 0; c < 3; ++c) xq[c * NQ + l] = o[c];
        }
        __syncthreads();
        for (int m = threadIdx.x; m < NP; m += blockDim.x) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int l = 0; l < NQ; ++l) {
                const double r = RT[(int64_t)l * NP + m];
                a0 += r * xq[l];
                a1 += r * xq[NQ + l];
                a2 += r * xq[2 * NQ + l];
            }
            xh[m] = a0;
            xh[NP + m] = a1;
            xh[2 * NP + m] = a2;
        }
        __syncthreads();
        for (int l = threadIdx.x; l < NQ; l += blockDim.x) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int m = 0; m < NP; ++m) {
                const double v = VT[(int64_t)m * NQ + l];
                a0 += v * xh[m];
                a1 += v * xh[NP + m];
                a2 += v * xh[2 * NP + m];
            }
            xq[l] = a0;
            xq[NQ + l] = a1;
            xq[2 * NQ + l] = a2;
        }
        __syncthreads();
        for (int l = threadIdx.x; l < NQ; l += blockDim.x) {
            const int i = l / QQ, j = (l / Q) % Q, k = l % Q;
            double D[3][3];   // d x_c / d eta_d
            for (int c = 0; c < 3; ++c) {
                const double* u = xq + c * NQ;
                double d0 = 0.0, d1 = 0.0, d2 = 0.0;
                for (int mm = 0; mm < Q; ++mm) {
                    d0 += Dt[i * Q + mm] * u[mm * QQ + j * Q + k];
                    d1 += Dt[QQ + j * Q + mm] * u[i * QQ + mm * Q + k];
                    d2 += Dt[2 * QQ + k * Q + mm] * u[i * QQ + j * Q + mm];
                }
                D[c][0] = d0; D[c][1] = d1; D[c][2] = d2;
            }
            const double e1 = z[i], e2 = z[Q + j], e3 = z[2 * Q + k];
            double T[3][3], J[3][3];
            deta_dxi<SHAPE, double>(e1, e2, e3, T);
            for (int c = 0; c < 3; ++c)
                for (int a = 0; a < 3; ++a) J[c][a] = D[c][0] * T[0][a] + D[c][1] * T[1][a] + D[c][2] * T[2][a];
            store_factors<SHAPE>(J, e1, e2, e3, w[i] * w[Q + j] * w[2 * Q + k], e, l, NQp, want_deriv, geom, dgeom,
                                 err, bad_elem);
        }
        __syncthreads();
    }
}

// per-direction point counts q1, q2, q3 (Q each for the full rule) and the
// points / weights of each direction
struct Rule3 {
    int q1, q2, q3;
    const double *z1, *z2, *z3, *w1, *w2, *w3;
};

template <int SHAPE>
__global__ void geom_curved_kernel(Rule3 R, int NQp, int64_t n_elem, const double* __restrict__ frame, int kind,
                                   int want_deriv, double* __restrict__ geom, double* __restrict__ dgeom,
                                   unsigned int* err, int* bad_elem) {
    const int NQ = R.q1 * R.q2 * R.q3;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_elem * NQ) return;
    int64_t e = idx / NQ;
    int l = (int)(idx % NQ);
    int i = l / (R.q2 * R.q3), j = (l / R.q3) % R.q2, k = l % R.q3;
    double e1 = R.z1[i], e2 = R.z2[j], e3 = R.z3[k];
    double xi[3];
    xi_from_eta<SHAPE>(e1, e2, e3, xi);
    const double* F = frame + e * 12;
    double y[3], JA[3][3];
    for (int r = 0; r < 3; ++r) {
        y[r] = F[r];
        for (int d = 0; d < 3; ++d) {
            y[r] += F[3 + r * 3 + d] * 0.5 * (xi[d] + 1.0);
            JA[r][d] = 0.5 * F[3 + r * 3 + d];
        }
    }
    double Dp[3][3], J[3][3];
    deform_jacobian(kind, y, Dp);
    for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) J[r][d] = Dp[r][0] * JA[0][d] + Dp[r][1] * JA[1][d] + Dp[r][2] * JA[2][d];
    store_factors<SHAPE>(J, e1, e2, e3, R.w1[i] * R.w2[j] * R.w3[k], e, l, NQp, want_deriv, geom, dgeom, err,
                         bad_elem);
}

__global__ void geom_affine_kernel(int64_t n_elem, const double* __restrict__ frame, double* __restrict__ rec,
                                   unsigned int* err, int* bad_elem) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    const double* F = frame + e * 12;
    double J[3][3], Ji[3][3];
    for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) J[r][d] = 0.5 * F[3 + r * 3 + d];
    double det = inv3(J, Ji);
    if (!(det > 0.0)) {
        atomicOr(err, DERR_GEOM);
        atomicMin(bad_elem, (int)e);
        return;
    }
    double* o = rec + e * 16;
    auto K = [&](int a, int b) { return det * (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2]); };
    o[0] = K(0, 0); o[1] = K(0, 1); o[2] = K(0, 2); o[3] = K(1, 1); o[4] = K(1, 2); o[5] = K(2, 2);
    o[6] = det;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) o[7 + 3 * a + c] = Ji[a][c];
}

// Per-point factors of affine elements, expanded once from their records
// (K = |J| J^{-1} J^{-T}, |J|): G_dd' = wl (T K T^T)_dd' and wl |J|, the
// layout of the curved factors [elem][7][NQp].  The FP64 operators read
// these instead of rebuilding T K T^T at every point of every apply.
template <int SHAPE>
__global__ void affine_points_kernel(int Q, int NQp, int64_t n_elem, const double* __restrict__ rec,
                                     const double* __restrict__ z, const double* __restrict__ w,
                                     double* __restrict__ out) {
    const int NQ = Q * Q * Q;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_elem * NQ) return;
    const int64_t e = idx / NQ;
    const int l = (int)(idx % NQ);
    const int i = l / (Q * Q), j = (l / Q) % Q, k = l % Q;
    double T[3][3];
    deta_dxi<SHAPE, double>(z[i], z[Q + j], z[2 * Q + k], T);
    const double* r = rec + e * 16;
    const double K[3][3] = {{r[0], r[1], r[2]}, {r[1], r[3], r[4]}, {r[2], r[4], r[5]}};
    const double wl = w[i] * w[Q + j] * w[2 * Q + k];
    double M[3][3];
    for (int d = 0; d < 3; ++d)
        for (int b = 0; b < 3; ++b) M[d][b] = T[d][0] * K[0][b] + T[d][1] * K[1][b] + T[d][2] * K[2][b];
    auto g = [&](int d, int d2) { return wl * (M[d][0] * T[d2][0] + M[d][1] * T[d2][1] + M[d][2] * T[d2][2]); };
    double* o = out + e * 7 * (int64_t)NQp + l;
    o[0 * NQp] = g(0, 0);
    o[1 * NQp] = g(0, 1);
    o[2 * NQp] = g(0, 2);
    o[3 * NQp] = g(1, 1);
    o[4 * NQp] = g(1, 2);
    o[5 * NQp] = g(2, 2);
    o[6 * NQp] = wl * r[6];
}

template <int SHAPE>
__global__ void points_kernel(int Q, int64_t n_elem, const double* __restrict__ frame, const int64_t* __restrict__ phys_off,
                              const double* __restrict__ z, int kind, int curved, double* __restrict__ xyz, int64_t n_phys) {
    const int NQ = Q * Q * Q;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n_elem * NQ) return;
    int64_t e = idx / NQ;
    int l = (int)(idx % NQ);
    int i = l / (Q * Q), j = (l / Q) % Q, k = l % Q;
    double xi[3];
    xi_from_eta<SHAPE>(z[i], z[Q + j], z[2 * Q + k], xi);
    double o[3];
    map_point(curved ? kind : 0, frame + e * 12, xi, o);
    for (int r = 0; r < 3; ++r) xyz[r * n_phys + phys_off[e] + l] = o[r];
}

__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) dst[i] = (float)src[i];
}

}  // namespace

cudaError_t launch_geom(const Block& b, const DeviceBlobs& blob, int deformation, bool want_deriv,
                        unsigned int* d_err, int* d_bad_elem, cudaStream_t s) {
    if (b.n_elem == 0) return cudaSuccess;
    if (!b.curved) {
        int nt = 128;
        int64_t nb = (b.n_elem + nt - 1) / nt;
        geom_affine_kernel<<<(unsigned)nb, nt, 0, s>>>(b.n_elem, b.d_frame, b.d_geom, d_err, d_bad_elem);
        return cudaGetLastError();
    }
    const BlobLayout L = blob_layout_c(b.shape, b.P, 8);
    const double* vals = reinterpret_cast<const double*>(blob.d64);
    const double* z = vals + L.z;
    const double* w = vals + L.w;
    const int Q = b.Q;
    Rule3 R{Q, Q, Q, z, z + Q, z + 2 * Q, w, w + Q, w + 2 * Q};
    // every block here keeps per-point factors; the reduced rule's affine blocks
    // (curved = 1 for the layout, map_curved = 0) take the map without deformation
    const int kind = b.map_curved ? deformation : 0;
    if (b.nq != Q * Q * Q) {       // reduced rule: its own points
        if (!blob.rq_zw) return cudaErrorInvalidValue;
        const double* p = blob.rq_zw;
        R = Rule3{b.q[0], b.q[1], b.q[2], p, p + 2 * b.q[0], p + 2 * (b.q[0] + b.q[1]),
                  p + b.q[0], p + 2 * b.q[0] + b.q[1], p + 2 * (b.q[0] + b.q[1]) + b.q[2]};
    }
    const int NQ = R.q1 * R.q2 * R.q3;
    int nt = 128;
    int64_t total = b.n_elem * NQ;
    unsigned nb = (unsigned)((total + nt - 1) / nt);
    const int NQp = (NQ + 3) & ~3;
    switch (b.shape) {
        case HP_HEX:
            geom_curved_kernel<HP_HEX><<<nb, nt, 0, s>>>(R, NQp, b.n_elem, b.d_frame, kind, want_deriv, b.d_geom,
                                                         b.d_dgeom, d_err, d_bad_elem);
            break;
        case HP_PRISM:
            geom_curved_kernel<HP_PRISM><<<nb, nt, 0, s>>>(R, NQp, b.n_elem, b.d_frame, kind, want_deriv, b.d_geom,
                                                           b.d_dgeom, d_err, d_bad_elem);
            break;
        case HP_PYR:
            geom_curved_kernel<HP_PYR><<<nb, nt, 0, s>>>(R, NQp, b.n_elem, b.d_frame, kind, want_deriv, b.d_geom,
                                                         b.d_dgeom, d_err, d_bad_elem);
            break;
        default:
            geom_curved_kernel<HP_TET><<<nb, nt, 0, s>>>(R, NQp, b.n_elem, b.d_frame, kind, want_deriv, b.d_geom,
                                                         b.d_dgeom, d_err, d_bad_elem);
    }
    return cudaGetLastError();
}

cudaError_t launch_geom_iso(const Block& b, const DeviceBlobs& blob, int deformation, bool want_deriv,
                            unsigned int* d_err, int* d_bad_elem, cudaStream_t s) {
    if (b.n_elem == 0) return cudaSuccess;
    if (!blob.iso_RT || !blob.iso_VT) return cudaErrorInvalidValue;
    const BlobLayout L = blob_layout_c(b.shape, b.P, 8);
    const double* vals = reinterpret_cast<const double*>(blob.d64);
    const int NQ = b.Q * b.Q * b.Q, NP = n_modes(b.shape, b.P);
    const int smem = (3 * NQ + 3 * NP) * (int)sizeof(double);
    auto run = [&](auto kern) -> cudaError_t {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const int grid = (int)std::min<int64_t>(b.n_elem, (int64_t)sms * 8);
        kern<<<grid, 256, smem, s>>>(b.Q, NP, nqp(b.Q), b.n_elem, b.d_frame, vals + L.z, vals + L.w, vals + L.D,
                                     deformation, blob.iso_RT, blob.iso_VT, want_deriv ? 1 : 0, b.d_geom, b.d_dgeom,
                                     d_err, d_bad_elem);
        return cudaGetLastError();
    };
    switch (b.shape) {
        case HP_HEX: return run(geom_iso_kernel<HP_HEX>);
        case HP_PRISM: return run(geom_iso_kernel<HP_PRISM>);
        case HP_PYR: return run(geom_iso_kernel<HP_PYR>);
        default: return run(geom_iso_kernel<HP_TET>);
    }
}

cudaError_t launch_affine_points(const Block& b, const DeviceBlobs& blob, double* out, cudaStream_t s) {
    if (b.n_elem == 0) return cudaSuccess;
    const BlobLayout L = blob_layout_c(b.shape, b.P, 8);
    const double* vals = reinterpret_cast<const double*>(blob.d64);
    const int NQ = b.Q * b.Q * b.Q, nt = 128;
    const unsigned nb = (unsigned)((b.n_elem * NQ + nt - 1) / nt);
    const int NQp = nqp(b.Q);
    switch (b.shape) {
        case HP_HEX: affine_points_kernel<HP_HEX><<<nb, nt, 0, s>>>(b.Q, NQp, b.n_elem, b.d_geom, vals + L.z, vals + L.w, out); break;
        case HP_PRISM: affine_points_kernel<HP_PRISM><<<nb, nt, 0, s>>>(b.Q, NQp, b.n_elem, b.d_geom, vals + L.z, vals + L.w, out); break;
        case HP_PYR: affine_points_kernel<HP_PYR><<<nb, nt, 0, s>>>(b.Q, NQp, b.n_elem, b.d_geom, vals + L.z, vals + L.w, out); break;
        default: affine_points_kernel<HP_TET><<<nb, nt, 0, s>>>(b.Q, NQp, b.n_elem, b.d_geom, vals + L.z, vals + L.w, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_points(const Block& b, const DeviceBlobs& blob, int deformation, double* xyz,
                          int64_t n_phys_total, cudaStream_t s) {
    if (b.n_elem == 0) return cudaSuccess;
    const BlobLayout L = blob_layout_c(b.shape, b.P, 8);
    const double* z = reinterpret_cast<const double*>(blob.d64) + L.z;
    int NQ = b.Q * b.Q * b.Q, nt = 128;
    unsigned nb = (unsigned)((b.n_elem * NQ + nt - 1) / nt);
    switch (b.shape) {
        case HP_HEX: points_kernel<HP_HEX><<<nb, nt, 0, s>>>(b.Q, b.n_elem, b.d_frame, b.d_phys_off, z, deformation, b.curved, xyz, n_phys_total); break;
        case HP_PRISM: points_kernel<HP_PRISM><<<nb, nt, 0, s>>>(b.Q, b.n_elem, b.d_frame, b.d_phys_off, z, deformation, b.curved, xyz, n_phys_total); break;
        case HP_PYR: points_kernel<HP_PYR><<<nb, nt, 0, s>>>(b.Q, b.n_elem, b.d_frame, b.d_phys_off, z, deformation, b.curved, xyz, n_phys_total); break;
        default: points_kernel<HP_TET><<<nb, nt, 0, s>>>(b.Q, b.n_elem, b.d_frame, b.d_phys_off, z, deformation, b.curved, xyz, n_phys_total);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    to_f32_kernel<<<1024, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace hp
