// Two-dimensional formulation (paper Sec. 2.2): mass, Laplacian and
// Helmholtz operators on quadrilaterals and triangles, by the collocated
// algorithm (Eq. helm1 in two dimensions),
//   out = B^T { sum_d D_d^T [sum_d' G_dd' D_d'] + lambda W } B uhat,
// with B applied as two sum-factorised passes (eta_2, then eta_1) over the
// slot tensor of the modal coefficients, Lagrange collocation derivatives
// D_1, D_2 along the lines of the Q x Q points, and the pointwise metric
// G_dd' = w|J| sum_i (d eta_d / d x_i)(d eta_d' / d x_i) (3 unique entries)
// and w|J| computed once per mesh in FP64 (FP32 copy for the FP32 operator).
//
// Bases and points (the modified C0 basis of the paper's 3-D shapes, in two
// dimensions): the quadrilateral's modes are A_a(xi_1) A_b(xi_2) with
// A = (L, R, psi_1 .. psi_{P-1}); the triangle's, on eta_1 = 2 (1 + xi_1) /
// (1 - xi_2) - 1, eta_2 = xi_2, are A_a(eta_1) W_{w(a), b}(eta_2) with the
// family of weight w(a) of the first factor (family 0 = A for a = L, R); the
// collapsed vertex (1, R) occupies slots (L, R) and (R, R), whose sum is one
// coefficient.  A mode's slot is its key (a, b) in the shared mode order
// (quadrilateral: (a, b) by family index; triangle: (a, r) with r the
// warped-family index when a is a bubble).  Points: Gauss-Lobatto-Legendre
// (Q = P + 2) in eta_1 and in the quadrilateral's eta_2, Gauss-Radau-Jacobi
// (alpha = 1, weights halved for the Duffy factor) in the triangle's eta_2.
//
// Layout: modal vectors element-major in user order (N_P values each), point
// vectors Q^2 values each; metric factors [element][4][Q^2] (G11, G12, G22,
// w|J|) per block of equal (shape, P, curved).  The kernels stage the block's
// tables in shared memory and keep every intermediate of EPB elements there.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "hp_internal.h"

namespace hp {
namespace {

constexpr int kT2 = 256;   // threads per CTA

// Reference tables of one (shape, P) as values (FP64 or FP32): Ta[a][i] (the
// eta_1 factor of slot row a at eta_1 point i), Tb[row][j] (the eta_2 factor of
// slot (a, b), row = tbrow[a] + b, at eta_2 point j), D1[i][m], D2[j][m]; and
// int16 maps: slot2mode[a][b] (-1: no mode), tbrow[a], lenb[a] (valid b per
// row a), mode_slots[m][2] (second -1 unless the collapsed vertex mode).
struct Tab2 {
    int n, Q, NP, nrows;
    int oTa, oTb, oD1, oD2, nvals;
    int o_s2m, o_row, o_len, o_ms, nidx;
    std::vector<double> vals;
    std::vector<int16_t> idx;
};

Tab2 build_tab2(int shape, int P) {
    Tab2 t;
    const int n = P + 1, Q = P + 2;
    const RefTables& r = ref_tables(shape == 4 ? HP_HEX : HP_TET, P);   // GLL x GLL or GLL x GRJ(1)/2
    t.n = n; t.Q = Q;
    std::vector<int> lenb(n), fam(n);
    for (int a = 0; a < n; ++a) {
        fam[a] = (shape == 5 && a >= 2) ? a - 1 : 0;
        lenb[a] = fam[a] == 0 ? n : P - fam[a];
    }
    std::vector<int> tbrow(n);
    int rows = 0;
    for (int a = 0; a < n; ++a) { tbrow[a] = rows; rows += lenb[a]; }
    t.nrows = rows;
    t.oTa = 0;
    t.oTb = n * Q;
    t.oD1 = t.oTb + rows * Q;
    t.oD2 = t.oD1 + Q * Q;
    t.nvals = t.oD2 + Q * Q;
    t.vals.assign(t.nvals, 0.0);
    for (int a = 0; a < n; ++a)
        for (int i = 0; i < Q; ++i) t.vals[t.oTa + a * Q + i] = family_value(P, 0, a, r.z[0][i]);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < lenb[a]; ++b)
            for (int j = 0; j < Q; ++j) t.vals[t.oTb + (tbrow[a] + b) * Q + j] = family_value(P, fam[a], b, r.z[1][j]);
    for (int k = 0; k < Q * Q; ++k) {
        t.vals[t.oD1 + k] = r.D[0][k];
        t.vals[t.oD2 + k] = r.D[1][k];
    }
    // modes in the shared order: slot keys (a, b) sorted, b fastest
    std::vector<std::pair<int, int>> keys;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < lenb[a]; ++b) {
            if (shape == 5 && a == 1 && b == 1) continue;   // (R, R): part of the collapsed vertex (L, R) + (R, R)
            keys.push_back({a, b});
        }
    std::sort(keys.begin(), keys.end());
    t.NP = (int)keys.size();
    t.o_s2m = 0;
    t.o_row = n * n;
    t.o_len = t.o_row + n;
    t.o_ms = t.o_len + n;
    t.nidx = t.o_ms + 2 * t.NP;
    t.idx.assign(t.nidx, -1);
    for (int m = 0; m < t.NP; ++m) {
        const int a = keys[m].first, b = keys[m].second;
        t.idx[t.o_s2m + a * n + b] = (int16_t)m;
        t.idx[t.o_ms + 2 * m] = (int16_t)(a * n + b);
        if (shape == 5 && a == 0 && b == 1) {            // the collapsed vertex also takes slot (R, R)
            t.idx[t.o_s2m + 1 * n + 1] = (int16_t)m;
            t.idx[t.o_ms + 2 * m + 1] = (int16_t)(1 * n + 1);
        }
    }
    for (int a = 0; a < n; ++a) {
        t.idx[t.o_row + a] = (int16_t)tbrow[a];
        t.idx[t.o_len + a] = (int16_t)lenb[a];
    }
    return t;
}

template <typename T>
struct SF2Args {
    int op, n, Q, NP, epb;
    int64_t n_elem;
    T lambda;
    const int64_t* coeff_off;   // per block element
    const T* in;
    T* out;
    const T* geom;              // [e][4][Q^2]
    const T* tab;               // Tab2 values
    const int16_t* idx;         // Tab2 int16 maps
    int nvals, nidx, oTa, oTb, oD1, oD2, o_s2m, o_row, o_len, o_ms;
};

// One CTA per group of EPB elements (persistent over the groups).  Shared
// memory: the tables, then per element S (n x Q: slots, later the eta_1
// restriction), U, V1, V2 and O (Q^2 each).
template <typename T>
__global__ void __launch_bounds__(kT2) sf2d_kernel(const SF2Args<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tab = reinterpret_cast<T*>(smem_raw);
    int16_t* idx = reinterpret_cast<int16_t*>(tab + a.nvals);
    const int n = a.n, Q = a.Q, QQ = Q * Q, NP = a.NP, E = a.epb, tid = threadIdx.x;
    T* S = reinterpret_cast<T*>(smem_raw + ((size_t)a.nvals * sizeof(T) + (size_t)a.nidx * 2 + 15) / 16 * 16);
    T* U = S + (size_t)E * n * Q;
    T* V1 = U + (size_t)E * QQ;
    T* V2 = V1 + (size_t)E * QQ;
    T* O = V2 + (size_t)E * QQ;
    for (int k = tid; k < a.nvals; k += kT2) tab[k] = a.tab[k];
    for (int k = tid; k < a.nidx; k += kT2) idx[k] = a.idx[k];
    __syncthreads();
    const T* Ta = tab + a.oTa;
    const T* Tb = tab + a.oTb;
    const T* D1 = tab + a.oD1;
    const T* D2 = tab + a.oD2;
    const int16_t* s2m = idx + a.o_s2m;
    const int16_t* trow = idx + a.o_row;
    const int16_t* lenb = idx + a.o_len;
    const int16_t* ms = idx + a.o_ms;
    const bool lap = a.op != HP_MASS;
    const int64_t ngroups = (a.n_elem + E - 1) / E;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const int64_t e0 = g * E;
        const int ne = (int)min((int64_t)E, a.n_elem - e0);
        // gather the coefficients into the slot tensor S[e][a][b]
        for (int k = tid; k < E * n * n; k += kT2) {
            const int e = k / (n * n), s = k - e * n * n;
            const int m = s2m[s];
            S[(size_t)e * n * Q + s] = (e < ne && m >= 0) ? a.in[a.coeff_off[e0 + e] + m] : T(0);
        }
        __syncthreads();
        // eta_2 pass: F[a][j] = sum_b Tb[row(a) + b][j] S[a][b], into V1 as [a][j]
        for (int k = tid; k < E * n * Q; k += kT2) {
            const int e = k / (n * Q), r = k - e * n * Q, aa = r / Q, j = r - aa * Q;
            const T* s = S + (size_t)e * n * Q + aa * n;
            const T* tb = Tb + (size_t)trow[aa] * Q + j;
            T acc = T(0);
            for (int b = 0; b < lenb[aa]; ++b) acc += tb[b * Q] * s[b];
            V1[(size_t)e * QQ + r] = acc;
        }
        __syncthreads();
        // eta_1 pass: U[i][j] = sum_a Ta[a][i] F[a][j]
        for (int k = tid; k < E * QQ; k += kT2) {
            const int e = k / QQ, r = k - e * QQ, i = r / Q, j = r - i * Q;
            const T* f = V1 + (size_t)e * QQ + j;
            T acc = T(0);
            for (int aa = 0; aa < n; ++aa) acc += Ta[aa * Q + i] * f[aa * Q];
            U[(size_t)e * QQ + r] = acc;
        }
        __syncthreads();
        // collocation derivatives and the pointwise metric (w = G v, t = lambda w|J| u)
        for (int k = tid; k < E * QQ; k += kT2) {
            const int e = k / QQ, r = k - e * QQ, i = r / Q, j = r - i * Q;
            const T* u = U + (size_t)e * QQ;
            T* o = O + (size_t)e * QQ + r;
            if (e >= ne) { *o = T(0); V2[(size_t)e * QQ + r] = T(0); continue; }
            const T* gp = a.geom + (e0 + e) * 4 * (int64_t)QQ + r;
            const T wJ = gp[3 * QQ];
            if (!lap) { *o = wJ * u[r]; continue; }
            T v1 = T(0), v2 = T(0);
            for (int m = 0; m < Q; ++m) {
                v1 += D1[i * Q + m] * u[m * Q + j];
                v2 += D2[j * Q + m] * u[i * Q + m];
            }
            const T g11 = gp[0], g12 = gp[QQ], g22 = gp[2 * QQ];
            *o = (a.op == HP_HELMHOLTZ) ? a.lambda * wJ * u[r] : T(0);
            // V1 held F, read by the eta_1 pass before the barrier above; U is only read here
            V1[(size_t)e * QQ + r] = g11 * v1 + g12 * v2;
            V2[(size_t)e * QQ + r] = g12 * v1 + g22 * v2;
        }
        __syncthreads();
        // u' = t + D_1^T w_1 + D_2^T w_2
        if (lap)
            for (int k = tid; k < E * QQ; k += kT2) {
                const int e = k / QQ, r = k - e * QQ, i = r / Q, j = r - i * Q;
                const T* w1 = V1 + (size_t)e * QQ;
                const T* w2 = V2 + (size_t)e * QQ;
                T acc = O[(size_t)e * QQ + r];
                for (int m = 0; m < Q; ++m) acc += D1[m * Q + i] * w1[m * Q + j] + D2[m * Q + j] * w2[i * Q + m];
                U[(size_t)e * QQ + r] = acc;
            }
        __syncthreads();
        const T* up = lap ? U : O;
        // eta_1 restriction: Gr[a][j] = sum_i Ta[a][i] u'[i][j] (into S as [a][j])
        for (int k = tid; k < E * n * Q; k += kT2) {
            const int e = k / (n * Q), r = k - e * n * Q, aa = r / Q, j = r - aa * Q;
            const T* x = up + (size_t)e * QQ + j;
            T acc = T(0);
            for (int i = 0; i < Q; ++i) acc += Ta[aa * Q + i] * x[i * Q];
            S[(size_t)e * n * Q + r] = acc;
        }
        __syncthreads();
        // eta_2 restriction of every valid slot, then the scatter to modes
        for (int k = tid; k < E * n * n; k += kT2) {
            const int e = k / (n * n), s = k - e * n * n, aa = s / n, b = s - aa * n;
            T acc = T(0);
            if (b < lenb[aa]) {
                const T* x = S + (size_t)e * n * Q + aa * Q;
                const T* tb = Tb + (size_t)(trow[aa] + b) * Q;
                for (int j = 0; j < Q; ++j) acc += tb[j] * x[j];
            }
            V2[(size_t)e * QQ + s] = acc;       // n^2 <= Q^2
        }
        __syncthreads();
        for (int k = tid; k < E * NP; k += kT2) {
            const int e = k / NP, m = k - e * NP;
            if (e >= ne) continue;
            const T* rs = V2 + (size_t)e * QQ;
            T acc = rs[ms[2 * m]];
            if (ms[2 * m + 1] >= 0) acc += rs[ms[2 * m + 1]];
            a.out[a.coeff_off[e0 + e] + m] = acc;
        }
        __syncthreads();
    }
}

// Metric factors of one block, FP64, one thread per (element, point):
// x = Phi(A_e(xi)), J = d x / d xi (analytic: the affine frame E / 2 times
// d Phi / d y), d eta / d xi of the collapse (triangle), and
// G_dd' = w|J| sum_i (d eta_d / d x_i)(d eta_d' / d x_i), w|J|; FP32 copy.
// A non-positive |J| latches DERR_GEOM.
__global__ void geom2d_kernel(int shape, int Q, int curved, int deformation, int64_t ne, const double* __restrict__ frame,
                              const double* __restrict__ z1, const double* __restrict__ w1,
                              const double* __restrict__ z2, const double* __restrict__ w2, double* __restrict__ g64,
                              float* __restrict__ g32, unsigned int* err) {
    const int QQ = Q * Q;
    const int64_t total = ne * QQ;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / QQ;
        const int l = (int)(k - e * QQ), i = l / Q, j = l - i * Q;
        const double e1 = z1[i], e2 = z2[j];
        const double x1 = shape == 4 ? e1 : 0.5 * (1.0 + e1) * (1.0 - e2) - 1.0, x2 = e2;
        const double* f = frame + e * 6;
        const double y1 = f[0] + 0.5 * (x1 + 1.0) * f[2] + 0.5 * (x2 + 1.0) * f[4];
        const double y2 = f[1] + 0.5 * (x1 + 1.0) * f[3] + 0.5 * (x2 + 1.0) * f[5];
        double F[2][2] = {{1.0, 0.0}, {0.0, 1.0}};     // d Phi / d y
        if (curved && deformation == 1) {
            const double pi = 3.14159265358979323846;
            const double d1 = 0.05 * pi * cos(pi * y1) * sin(pi * y2), d2 = 0.05 * pi * sin(pi * y1) * cos(pi * y2);
            F[0][0] += d1; F[0][1] += d2; F[1][0] += d1; F[1][1] += d2;
        }
        double J[2][2];
        for (int r = 0; r < 2; ++r)
            for (int d = 0; d < 2; ++d) J[r][d] = 0.5 * (F[r][0] * f[2 + 2 * d] + F[r][1] * f[3 + 2 * d]);
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (!(det > 0.0)) {
            atomicOr(err, DERR_GEOM);
            continue;
        }
        const double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};   // d xi_d / d x_i
        double Tm[2][2] = {{1.0, 0.0}, {0.0, 1.0}};    // d eta_d / d xi_a
        if (shape == 5) { Tm[0][0] = 2.0 / (1.0 - x2); Tm[0][1] = (1.0 + e1) / (1.0 - e2); }
        double Gx[2][2];
        for (int d = 0; d < 2; ++d)
            for (int c = 0; c < 2; ++c) Gx[d][c] = Tm[d][0] * Ji[0][c] + Tm[d][1] * Ji[1][c];
        const double wJ = w1[i] * w2[j] * det;
        const double g[4] = {wJ * (Gx[0][0] * Gx[0][0] + Gx[0][1] * Gx[0][1]), wJ * (Gx[0][0] * Gx[1][0] + Gx[0][1] * Gx[1][1]),
                             wJ * (Gx[1][0] * Gx[1][0] + Gx[1][1] * Gx[1][1]), wJ};
        for (int c = 0; c < 4; ++c) {
            g64[(e * 4 + c) * QQ + l] = g[c];
            g32[(e * 4 + c) * QQ + l] = (float)g[c];
        }
    }
}

template <typename T>
cudaError_t sf2d_launch(const SF2Args<T>& a0, cudaStream_t s) {
    if (a0.n_elem <= 0) return cudaSuccess;
    SF2Args<T> a = a0;
    const int QQ = a.Q * a.Q;
    const size_t head = ((size_t)a.nvals * sizeof(T) + (size_t)a.nidx * 2 + 15) / 16 * 16;
    const size_t per = ((size_t)a.n * a.Q + 4 * (size_t)QQ) * sizeof(T);
    // elements per CTA: up to 32, within 64 KB of shared memory
    int epb = (int)std::max<size_t>(1, std::min<size_t>(32, (64 * 1024 - std::min<size_t>(head, 32 * 1024)) / per));
    a.epb = epb;
    const size_t smem = head + (size_t)epb * per;
    auto kern = sf2d_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int per_sm = std::max(1, std::min(2048 / kT2, (int)(228 * 1024 / (smem + 1024))));
    const int64_t groups = (a.n_elem + epb - 1) / epb;
    const int grid = (int)std::min<int64_t>(groups, (int64_t)sms * per_sm);
    kern<<<grid, kT2, smem, s>>>(a);
    return cudaGetLastError();
}

struct Block2 {
    int shape = 4, P = 1, Q = 3, curved = 0;
    std::vector<int64_t> elems;                 // user element ids, in order
    int64_t* d_coeff_off = nullptr;             // global coefficient offset per block element
    double* d_geom = nullptr;                   // [e][4][Q^2]
    float* d_geom32 = nullptr;
};

struct Tab2Dev {
    Tab2 t;
    double* d64 = nullptr;
    float* d32 = nullptr;
    int16_t* didx = nullptr;
};

}  // namespace
}  // namespace hp

struct hp_mesh2d_s {
    int device = 0;
    int64_t n_elem = 0;
    int deformation = 0;
    std::vector<int64_t> coeff_off, phys_off;   // user order, n_elem + 1
    std::vector<hp::Block2> blocks;
    std::map<int, hp::Tab2Dev> tabs;            // key shape * 16 + P
    unsigned int* d_err = nullptr;
};

using namespace hp;

namespace {

struct Guard2 {
    int prev = -1;
    explicit Guard2(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard2() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

template <typename T>
hp_status up2(T** dst, const T* src, size_t count) {
    *dst = nullptr;
    if (count == 0) return HP_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if (src) {
        e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    }
    return HP_OK;
}

int n_modes2(int shape, int P) { return shape == HP_QUAD ? (P + 1) * (P + 1) : (P + 1) * (P + 2) / 2; }

void free_mesh2d(hp_mesh2d m) {
    for (Block2& b : m->blocks) {
        cudaFree(b.d_coeff_off);
        cudaFree(b.d_geom);
        cudaFree(b.d_geom32);
    }
    for (auto& kv : m->tabs) {
        cudaFree(kv.second.d64);
        cudaFree(kv.second.d32);
        cudaFree(kv.second.didx);
    }
    cudaFree(m->d_err);
    delete m;
}

}  // namespace

extern "C" {

hp_status hp_mesh2d_create(const hp_mesh2d_desc* d, int device, hp_mesh2d* out) {
    if (!d || !out) { set_error("hp_mesh2d_create: null argument"); return HP_ERR_ARG; }
    *out = nullptr;
    if (d->n_elem < 1 || !d->shape || !d->P || !d->vert || !d->xy || d->n_vert < 1 || !d->curved) {
        set_error("hp_mesh2d_create: empty mesh or null array");
        return HP_ERR_ARG;
    }
    if (d->deformation != 0 && d->deformation != 1) { set_error("hp_mesh2d_create: deformation must be 0 or 1"); return HP_ERR_ARG; }
    for (int64_t e = 0; e < d->n_elem; ++e) {
        const int s = d->shape[e], P = d->P[e];
        if ((s != HP_QUAD && s != HP_TRI) || P < 1 || P > 10) {
            set_error("hp_mesh2d_create: bad shape or order in element " + std::to_string(e));
            return HP_ERR_ARG;
        }
        for (int v = 0; v < (s == HP_QUAD ? 4 : 3); ++v) {
            const int64_t id = d->vert[e * 4 + v];
            if (id < 0 || id >= d->n_vert) {
                set_error("hp_mesh2d_create: vertex id out of range in element " + std::to_string(e));
                return HP_ERR_ARG;
            }
        }
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("hp_mesh2d_create: no such CUDA device");
        return HP_ERR_CUDA;
    }
    Guard2 guard(device);
    auto m = new hp_mesh2d_s();
    m->device = device;
    m->n_elem = d->n_elem;
    m->deformation = d->deformation;
    m->coeff_off.assign(d->n_elem + 1, 0);
    m->phys_off.assign(d->n_elem + 1, 0);
    for (int64_t e = 0; e < d->n_elem; ++e) {
        m->coeff_off[e + 1] = m->coeff_off[e] + n_modes2(d->shape[e], d->P[e]);
        m->phys_off[e + 1] = m->phys_off[e] + (int64_t)(d->P[e] + 2) * (d->P[e] + 2);
    }
    // blocks of equal (shape, P, curved), in order of first appearance
    std::map<std::tuple<int, int, int>, size_t> index;
    for (int64_t e = 0; e < d->n_elem; ++e) {
        auto key = std::make_tuple((int)d->shape[e], (int)d->P[e], d->curved[e] ? 1 : 0);
        auto it = index.find(key);
        if (it == index.end()) {
            Block2 b;
            b.shape = d->shape[e]; b.P = d->P[e]; b.Q = b.P + 2; b.curved = d->curved[e] ? 1 : 0;
            it = index.emplace(key, m->blocks.size()).first;
            m->blocks.push_back(b);
        }
        m->blocks[it->second].elems.push_back(e);
    }
    hp_status st = up2<unsigned int>(&m->d_err, nullptr, 1);
    if (!st && cudaMemset(m->d_err, 0, sizeof(unsigned int)) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "cudaMemset");
    for (size_t bi = 0; bi < m->blocks.size() && !st; ++bi) {
        Block2& b = m->blocks[bi];
        const int key = b.shape * 16 + b.P;
        if (!m->tabs.count(key)) {
            Tab2Dev td;
            td.t = build_tab2(b.shape, b.P);
            std::vector<float> v32(td.t.vals.begin(), td.t.vals.end());
            st = up2(&td.d64, td.t.vals.data(), td.t.vals.size());
            if (!st) st = up2(&td.d32, v32.data(), v32.size());
            if (!st) st = up2(&td.didx, td.t.idx.data(), td.t.idx.size());
            m->tabs[key] = td;
            if (st) break;
        }
        const int64_t ne = (int64_t)b.elems.size();
        std::vector<int64_t> co(ne);
        std::vector<double> frame(ne * 6);
        const int v2 = b.shape == HP_QUAD ? 3 : 2;
        for (int64_t k = 0; k < ne; ++k) {
            const int64_t e = b.elems[k];
            co[k] = m->coeff_off[e];
            const double* X0 = d->xy + 2 * d->vert[e * 4];
            const double* X1 = d->xy + 2 * d->vert[e * 4 + 1];
            const double* X2 = d->xy + 2 * d->vert[e * 4 + v2];
            const double f[6] = {X0[0], X0[1], X1[0] - X0[0], X1[1] - X0[1], X2[0] - X0[0], X2[1] - X0[1]};
            for (int c = 0; c < 6; ++c) frame[k * 6 + c] = f[c];
        }
        double* d_frame = nullptr;
        double* d_rule = nullptr;
        st = up2(&b.d_coeff_off, co.data(), co.size());
        if (!st) st = up2(&d_frame, frame.data(), frame.size());
        if (!st) st = up2<double>(&b.d_geom, nullptr, (size_t)ne * 4 * b.Q * b.Q);
        if (!st) st = up2<float>(&b.d_geom32, nullptr, (size_t)ne * 4 * b.Q * b.Q);
        if (!st) {
            const RefTables& r = ref_tables(b.shape == HP_QUAD ? HP_HEX : HP_TET, b.P);
            std::vector<double> rule;
            for (int dd = 0; dd < 2; ++dd) {
                rule.insert(rule.end(), r.z[dd].begin(), r.z[dd].end());
                rule.insert(rule.end(), r.w[dd].begin(), r.w[dd].end());
            }
            st = up2(&d_rule, rule.data(), rule.size());
        }
        if (!st) {
            const int Q = b.Q;
            const int64_t total = ne * Q * Q;
            const int grid = (int)std::min<int64_t>((total + 255) / 256, 65535);
            geom2d_kernel<<<grid, 256>>>(b.shape, Q, b.curved, m->deformation, ne, d_frame, d_rule, d_rule + Q,
                                         d_rule + 2 * Q, d_rule + 3 * Q, b.d_geom, b.d_geom32, m->d_err);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) st = cuda_fail(e, "hp_mesh2d_create geometry");
        }
        cudaFree(d_frame);
        cudaFree(d_rule);
    }
    if (!st) {
        unsigned int err = 0;
        cudaError_t e = cudaMemcpy(&err, m->d_err, sizeof(err), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "hp_mesh2d_create");
        else if (err & DERR_GEOM) { set_error("hp_mesh2d_create: non-positive Jacobian"); st = HP_ERR_GEOM; }
    }
    if (st) { free_mesh2d(m); return st; }
    *out = m;
    return HP_OK;
}

hp_status hp_mesh2d_layout(hp_mesh2d m, int64_t* coeff_offset, int64_t* phys_offset) {
    if (!m) { set_error("hp_mesh2d_layout: null mesh"); return HP_ERR_ARG; }
    for (int64_t e = 0; e <= m->n_elem; ++e) {
        if (coeff_offset) coeff_offset[e] = m->coeff_off[e];
        if (phys_offset) phys_offset[e] = m->phys_off[e];
    }
    return HP_OK;
}

hp_status hp_op2d_apply(hp_mesh2d m, hp_opkind kind, hp_dtype dtype, double lambda, const void* in, void* out,
                        void* stream) {
    if (!m || !in || !out) { set_error("hp_op2d_apply: null argument"); return HP_ERR_ARG; }
    if (in == out) { set_error("hp_op2d_apply: in and out must not alias"); return HP_ERR_ARG; }
    if ((kind != HP_MASS && kind != HP_LAPLACIAN && kind != HP_HELMHOLTZ) || (dtype != HP_FP64 && dtype != HP_FP32)) {
        set_error("hp_op2d_apply: two-dimensional operators are mass, Laplacian and Helmholtz in HP_FP64 / HP_FP32");
        return HP_ERR_UNSUPPORTED;
    }
    Guard2 guard(m->device);
    for (const Block2& b : m->blocks) {
        const Tab2Dev& td = m->tabs.at(b.shape * 16 + b.P);
        const Tab2& t = td.t;
        cudaError_t e;
        auto fill = [&](auto& a) {
            a.op = kind; a.n = t.n; a.Q = t.Q; a.NP = t.NP; a.epb = 1;
            a.n_elem = (int64_t)b.elems.size();
            a.coeff_off = b.d_coeff_off;
            a.idx = td.didx;
            a.nvals = t.nvals; a.nidx = t.nidx;
            a.oTa = t.oTa; a.oTb = t.oTb; a.oD1 = t.oD1; a.oD2 = t.oD2;
            a.o_s2m = t.o_s2m; a.o_row = t.o_row; a.o_len = t.o_len; a.o_ms = t.o_ms;
        };
        if (dtype == HP_FP64) {
            SF2Args<double> a{};
            fill(a);
            a.lambda = lambda; a.in = static_cast<const double*>(in); a.out = static_cast<double*>(out);
            a.geom = b.d_geom; a.tab = td.d64;
            e = sf2d_launch(a, (cudaStream_t)stream);
        } else {
            SF2Args<float> a{};
            fill(a);
            a.lambda = (float)lambda; a.in = static_cast<const float*>(in); a.out = static_cast<float*>(out);
            a.geom = b.d_geom32; a.tab = td.d32;
            e = sf2d_launch(a, (cudaStream_t)stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "hp_op2d_apply launch");
    }
    return HP_OK;
}

hp_status hp_mesh2d_factors(hp_mesh2d m, double* host_out) {
    if (!m || !host_out) { set_error("hp_mesh2d_factors: null argument"); return HP_ERR_ARG; }
    Guard2 guard(m->device);
    for (const Block2& b : m->blocks) {
        const int64_t per = 4 * (int64_t)b.Q * b.Q;
        std::vector<double> g((size_t)per * b.elems.size());
        cudaError_t e = cudaMemcpy(g.data(), b.d_geom, g.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "hp_mesh2d_factors");
        for (size_t k = 0; k < b.elems.size(); ++k)
            std::copy(g.begin() + k * per, g.begin() + (k + 1) * per, host_out + 4 * m->phys_off[b.elems[k]]);
    }
    return HP_OK;
}

hp_status hp_mesh2d_sync(hp_mesh2d m, void* stream) {
    if (!m) { set_error("hp_mesh2d_sync: null mesh"); return HP_ERR_ARG; }
    Guard2 guard(m->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "hp_mesh2d_sync");
    return HP_OK;
}

void hp_mesh2d_destroy(hp_mesh2d m) {
    if (!m) return;
    Guard2 guard(m->device);
    free_mesh2d(m);
}

}  // extern "C"
