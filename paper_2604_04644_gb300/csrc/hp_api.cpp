// C ABI of libhp: mesh creation and validation, block grouping, geometric
// factors, operator creation and application (declarations in include/hp.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>

#include "hp_internal.h"
#include "hp_tc.cuh"

namespace hp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

hp_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HP_ERR_OOM : HP_ERR_CUDA;
}

int nqp(int Q) { return (Q * Q * Q + 3) & ~3; }

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

const int kNV[4] = {8, 6, 5, 4};
const int kAxis[4][3] = {{1, 3, 4}, {1, 3, 4}, {1, 3, 4}, {1, 2, 3}};
const double kRef[4][8][3] = {
    {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {1, 1, 1}, {-1, 1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}, {-1, 1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1}, {-1, -1, 1}},
    {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}}};

template <typename T>
hp_status upload(T** dst, const T* src, size_t count) {
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

void free_block(Block& b) {
    cudaFree(b.d_coeff_off);
    cudaFree(b.d_phys_off);
    cudaFree(b.d_frame);
    cudaFree(b.d_geom);
    cudaFree(b.d_dgeom);
    cudaFree(b.d_geom32);
    cudaFree(b.d_dgeom32);
    cudaFree(b.d_geom_tc);
    cudaFree(b.d_gscale_tc);
    cudaFree(b.d_geom_pts);
    b.d_geom_pts = nullptr;
    b.d_geom_tc = nullptr;
    b.d_gscale_tc = nullptr;
    b.d_coeff_off = b.d_phys_off = nullptr;
    b.d_frame = b.d_geom = b.d_dgeom = nullptr;
    b.d_geom32 = b.d_dgeom32 = nullptr;
}

int bnqp(const Block& b) { return (b.nq + 3) & ~3; }   // padded points per element of the block's rule
int64_t geom_count(const Block& b) { return b.curved ? b.n_elem * 7 * (int64_t)bnqp(b) : b.n_elem * 16; }
int64_t dgeom_count(const Block& b) { return b.curved ? b.n_elem * 9 * (int64_t)bnqp(b) : 0; }

hp_status check_device_error(hp_mesh m, unsigned int* d_err, int* d_bad, const char* what) {
    unsigned int herr = 0;
    cudaError_t e = cudaMemcpy(&herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (herr == 0) return HP_OK;
    cudaMemset(d_err, 0, sizeof(unsigned int));
    if (herr & DERR_GEOM) {
        int bad = -1;
        if (d_bad) cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
        set_error(std::string(what) + ": non-positive Jacobian at a quadrature point (block element " +
                  std::to_string(bad) + ")");
        return HP_ERR_GEOM;
    }
    if (herr & DERR_TIMEOUT) {
        set_error(std::string(what) + ": a bounded device wait gave up");
        return HP_ERR_TIMEOUT;
    }
    set_error(std::string(what) + ": device bounds check failed");
    return HP_ERR_DEVICE_BOUNDS;
}

hp_status ensure_dense(hp_mesh m);
hp_status ensure_iso(hp_mesh m);

hp_status compute_geom(hp_mesh m, bool want_deriv, cudaStream_t s) {
    if (m->geometry == 1) {
        hp_status sti = ensure_iso(m);
        if (sti) return sti;
    }
    int* d_bad = nullptr;
    hp_status st = upload<int>(&d_bad, nullptr, 1);
    if (st) return st;
    int big = 0x7fffffff;
    cudaMemcpy(d_bad, &big, sizeof(int), cudaMemcpyHostToDevice);
    for (Block& b : m->blocks) {
        if (!b.d_geom) {
            st = upload<double>(&b.d_geom, nullptr, geom_count(b));
            if (st) { cudaFree(d_bad); return st; }
        }
        if (want_deriv && b.curved && !b.d_dgeom) {
            st = upload<double>(&b.d_dgeom, nullptr, dgeom_count(b));
            if (st) { cudaFree(d_bad); return st; }
        }
        const DeviceBlobs& blob = m->blobs.at(b.shape * 16 + b.P);
        cudaError_t e = (b.curved && m->geometry == 1)
                            ? launch_geom_iso(b, blob, m->deformation, want_deriv, m->d_err, d_bad, s)
                            : launch_geom(b, blob, m->deformation, want_deriv && b.curved, m->d_err, d_bad, s);
        if (e != cudaSuccess) { cudaFree(d_bad); return cuda_fail(e, "geometry kernel"); }
        cudaError_t se = cudaStreamSynchronize(s);
        if (se != cudaSuccess) { cudaFree(d_bad); return cuda_fail(se, "geometry kernel"); }
        st = check_device_error(m, m->d_err, d_bad, "hp_geom_factors");
        if (st) {
            int bad = -1;
            cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
            if (bad >= 0 && bad < b.n_elem)
                set_error("hp_geom_factors: non-positive Jacobian in element " + std::to_string(b.elems[bad]));
            cudaFree(d_bad);
            return st;
        }
    }
    cudaFree(d_bad);
    m->geom_ready = true;
    if (want_deriv) m->dgeom_ready = true;
    m->geom32_ready = false;
    return HP_OK;
}

hp_status ensure_geom(hp_mesh m, bool deriv, bool f32, cudaStream_t s) {
    hp_status st = HP_OK;
    if (!m->geom_ready || (deriv && !m->dgeom_ready)) {
        st = compute_geom(m, deriv || m->dgeom_ready, s);
        if (st) return st;
    }
    if (f32 && !m->geom32_ready) {
        for (Block& b : m->blocks) {
            cudaFree(b.d_geom32);
            cudaFree(b.d_dgeom32);
            b.d_geom32 = b.d_dgeom32 = nullptr;
            st = upload<float>(&b.d_geom32, nullptr, geom_count(b));
            if (st) return st;
            cudaError_t e = launch_to_f32(b.d_geom, b.d_geom32, geom_count(b), s);
            if (e != cudaSuccess) return cuda_fail(e, "fp32 geometry");
            if (b.d_dgeom) {
                st = upload<float>(&b.d_dgeom32, nullptr, dgeom_count(b));
                if (st) return st;
                e = launch_to_f32(b.d_dgeom, b.d_dgeom32, dgeom_count(b), s);
                if (e != cudaSuccess) return cuda_fail(e, "fp32 geometry");
            }
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "fp32 geometry");
        m->geom32_ready = true;
    }
    return HP_OK;
}

// Affine blocks of FP64 collocated Laplacian / Helmholtz operators read
// per-point factors expanded from their records (like curved blocks): on
// GB300 the FP64 pipe is the limit and HBM has bandwidth to spare, so
// loading G costs less than rebuilding T K T^T at every point.
bool affine_expanded(const hp_op_s* op, const Block& b) {
    return !b.curved && b.d_geom_pts && op->dtype == HP_FP64 && op->collocated &&
           (op->kind == HP_LAPLACIAN || op->kind == HP_HELMHOLTZ);
}

hp_status ensure_affine_points(hp_mesh m, cudaStream_t s) {
    for (Block& b : m->blocks) {
        if (b.curved || b.d_geom_pts || b.n_elem == 0) continue;
        hp_status st = upload<double>(&b.d_geom_pts, nullptr, (size_t)b.n_elem * 7 * bnqp(b));
        if (st) return st;
        cudaError_t e = launch_affine_points(b, m->blobs.at(b.shape * 16 + b.P), b.d_geom_pts, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "affine point factors");
    }
    return HP_OK;
}

bool coeff_in(hp_opkind k) {
    return k == HP_MASS || k == HP_LAPLACIAN || k == HP_HELMHOLTZ || k == HP_BWDTRANS ||
           k == HP_ADVECTION_DIFFUSION_REACTION;
}
bool coeff_out(hp_opkind k) { return k != HP_BWDTRANS && k != HP_PHYSDERIV; }
// kinds that read d eta / d x at the points (and are sum-factorised only)
bool needs_deriv_geom(hp_opkind k) {
    return k == HP_PHYSDERIV || k == HP_IPRODUCT_WRT_DERIV_BASE || k == HP_ADVECTION_DIFFUSION_REACTION;
}

hp_status ensure_dense(hp_mesh m) {
    for (auto& kv : m->blobs) {
        DeviceBlobs& db = kv.second;
        if (db.A4_64) continue;
        int shape = kv.first / 16, P = kv.first % 16;
        const int NQ = n_points(shape, P, m->quadrature), NP = n_modes(shape, P);
        std::vector<double> A = m->quadrature ? dense_matrices_rq(shape, P) : dense_matrices(shape, P);
        std::vector<double> AT(A.size());
        for (int q = 0; q < 4; ++q)
            for (int l = 0; l < NQ; ++l)
                for (int mm = 0; mm < NP; ++mm) AT[((size_t)mm * 4 + q) * NQ + l] = A[((size_t)q * NQ + l) * NP + mm];
        std::vector<float> A32(A.begin(), A.end()), AT32(AT.begin(), AT.end());
        hp_status st;
        if ((st = upload(&db.A4_64, A.data(), A.size()))) return st;
        if ((st = upload(&db.A4T_64, AT.data(), AT.size()))) return st;
        if ((st = upload(&db.A4_32, A32.data(), A32.size()))) return st;
        if ((st = upload(&db.A4T_32, AT32.data(), AT32.size()))) return st;
    }
    return HP_OK;
}

// Projection tables of the iso-parametric geometry for every (shape, P) of the
// mesh's curved blocks.  The L2 projection on the reference element of point
// values x onto the element's expansion is W^{-1/2} Qo Qo^T W^{1/2} x, with
// W^{1/2} B = Qo R a Householder QR (B the modes at the points, W the
// reference weights) and Qo formed explicitly from the reflectors: the
// orthonormal columns keep it well conditioned, where the normal equations
// B^T W B (or R^{-1}) of the modal basis lose digits at high order.
// Stored (FP64): iso_RT [point][mode] = Qo W^{1/2} (coefficients c = S x of
// the projection in the orthonormal functions, S = RT^T) and iso_VT
// [mode][point] = (W^{-1/2} Qo)^T (their values at the points).
hp_status ensure_iso(hp_mesh m) {
    for (auto& kv : m->blobs) {
        DeviceBlobs& db = kv.second;
        const int shape = kv.first / 16, P = kv.first % 16;
        bool used = false;
        for (const Block& b : m->blocks) used |= b.curved && b.shape == shape && b.P == P;
        if (!used || db.iso_RT) continue;
        const RefTables& t = ref_tables(shape, P);
        const int Q = t.Q, NQ = Q * Q * Q, NP = n_modes(shape, P);
        std::vector<double> A4 = dense_matrices(shape, P);             // [4][NQ][NP], q = 0: B
        std::vector<double> sw(NQ);
        for (int i = 0; i < Q; ++i)
            for (int j = 0; j < Q; ++j)
                for (int k = 0; k < Q; ++k) sw[(i * Q + j) * Q + k] = std::sqrt(t.w[0][i] * t.w[1][j] * t.w[2][k]);
        // Householder QR of A = W^{1/2} B, column-major; reflector j in V[j][.] (rows >= j)
        std::vector<double> A((size_t)NP * NQ), V((size_t)NP * NQ, 0.0), vv(NP, 0.0);
        for (int l = 0; l < NQ; ++l)
            for (int c = 0; c < NP; ++c) A[(size_t)c * NQ + l] = sw[l] * A4[(size_t)l * NP + c];
        for (int j = 0; j < NP; ++j) {
            double* x = &A[(size_t)j * NQ];
            double* v = &V[(size_t)j * NQ];
            double nrm = 0.0;
            for (int r = j; r < NQ; ++r) nrm += x[r] * x[r];
            nrm = std::sqrt(nrm);
            if (!(nrm > 0.0)) { set_error("iso-parametric geometry: rank-deficient mode table"); return HP_ERR_GEOM; }
            const double alpha = x[j] > 0.0 ? -nrm : nrm;
            for (int r = j; r < NQ; ++r) v[r] = x[r];
            v[j] -= alpha;
            for (int r = j; r < NQ; ++r) vv[j] += v[r] * v[r];
            x[j] = alpha;
            for (int r = j + 1; r < NQ; ++r) x[r] = 0.0;
            for (int c = j + 1; c < NP; ++c) {
                double* y = &A[(size_t)c * NQ];
                double sdot = 0.0;
                for (int r = j; r < NQ; ++r) sdot += v[r] * y[r];
                const double f = 2.0 * sdot / vv[j];
                for (int r = j; r < NQ; ++r) y[r] -= f * v[r];
            }
        }
        // Qo = H_0 H_1 ... H_{NP-1} [I; 0], column-major (backward accumulation)
        std::vector<double> Qo((size_t)NP * NQ, 0.0);
        for (int c = 0; c < NP; ++c) Qo[(size_t)c * NQ + c] = 1.0;
        for (int j = NP - 1; j >= 0; --j) {
            const double* v = &V[(size_t)j * NQ];
            for (int c = j; c < NP; ++c) {
                double* y = &Qo[(size_t)c * NQ];
                double sdot = 0.0;
                for (int r = j; r < NQ; ++r) sdot += v[r] * y[r];
                const double f = 2.0 * sdot / vv[j];
                for (int r = j; r < NQ; ++r) y[r] -= f * v[r];
            }
        }
        std::vector<double> RT((size_t)NQ * NP), VT((size_t)NP * NQ);
        for (int l = 0; l < NQ; ++l)
            for (int c = 0; c < NP; ++c) {
                RT[(size_t)l * NP + c] = Qo[(size_t)c * NQ + l] * sw[l];
                VT[(size_t)c * NQ + l] = Qo[(size_t)c * NQ + l] / sw[l];
            }
        hp_status st;
        if ((st = upload(&db.iso_RT, RT.data(), RT.size()))) return st;
        if ((st = upload(&db.iso_VT, VT.data(), VT.size()))) return st;
    }
    return HP_OK;
}

// round to the TF32 grid (10-bit mantissa, nearest, ties away from zero)
float round_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0x1000u;
        u &= 0xffffe000u;
    }
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// round to bfloat16 (8 significant bits, nearest, ties to even); finite inputs
uint16_t round_bf16(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Reference tiles of the tensor-core elemental-matrix operator for operands of
// es bytes (4: TF32, 2: BF16), per chunk of tc_chunk_points() quadrature
// points: the forward operand (64 rows = 4 components x 16 points, K = modes)
// in K-slices of 128 bytes of modes (zero padded), 128-byte swizzled, then the
// backward tiles R_c[mode][point] (rows padded to NPpad; 16 points = 64-byte
// (TF32) or 32-byte (BF16) swizzled rows) of the 4 components: the K-major
// swizzled order the tensor core reads from shared memory.
hp_status ensure_tc(hp_mesh m, int es) {
    for (auto& kv : m->blobs) {
        DeviceBlobs& db = kv.second;
        const int shape = kv.first / 16, P = kv.first % 16;
        const int NQ = n_points(shape, P, m->quadrature), NP = n_modes(shape, P), NPT = tc_chunk_points();
        if (NP > (es == 2 ? kTcHybMaxModes : kTcHybMaxModesTF32)) continue;   // the hybrid's limit (>= the elemental matrix's)
        const int KR = 128 / es, vrow = NPT * es;
        const int KP = (NP + KR - 1) / KR * KR, NPpad = (NP + 15) & ~15, nch = (NQ + NPT - 1) / NPT;
        const int slice = 4 * NPT * 128;                       // 64 rows x 128 bytes
        const int fwd = (KP / KR) * slice, bwd = NPpad * vrow;
        const int64_t chunk = fwd + 4 * (int64_t)bwd;
        if ((es == 4 && db.tc_img) || (es == 2 && db.tc_img16)) continue;
        std::vector<double> A = m->quadrature ? dense_matrices_rq(shape, P) : dense_matrices(shape, P);
        std::vector<unsigned char> img((size_t)(chunk * nch), 0);
        auto put = [&](unsigned char* dst, double x) {
            if (es == 4) {
                const float v = round_tf32((float)x);
                std::memcpy(dst, &v, 4);
            } else {
                const uint16_t v = round_bf16((float)x);
                std::memcpy(dst, &v, 2);
            }
        };
        for (int k = 0; k < nch; ++k) {
            unsigned char* F = img.data() + (size_t)k * chunk;
            for (int c = 0; c < 4; ++c) {
                unsigned char* R = img.data() + (size_t)k * chunk + fwd + (size_t)c * bwd;
                for (int r = 0; r < NPT; ++r) {
                    const int l = k * NPT + r;
                    if (l >= NQ) continue;
                    for (int mm = 0; mm < NP; ++mm) {
                        const double x = A[((size_t)c * NQ + l) * NP + mm];
                        const int row = c * NPT + r, kk = mm % KR;
                        put(F + (size_t)(mm / KR) * slice + row * 128 + ((((kk * es) >> 4) ^ (row & 7)) << 4) + ((kk * es) & 15), x);
                        const uint32_t rv = es == 4 ? tc::sw64_offset(mm, r)
                                                    : mm * 32 + ((((r * 2) >> 4) ^ ((mm >> 2) & 1)) << 4) + ((r * 2) & 15);
                        put(R + rv, x);
                    }
                }
            }
        }
        hp_status st0 = upload(es == 4 ? &db.tc_img : &db.tc_img16, img.data(), img.size());
        if (st0) return st0;
        if (es == 4) {
            db.tc_KP = KP; db.tc_fwd = fwd; db.tc_bwd = bwd; db.tc_chunk = chunk;
        } else {
            db.tc_KP16 = KP; db.tc_fwd16 = fwd; db.tc_bwd16 = bwd; db.tc_chunk16 = chunk;
        }
        db.tc_NPpad = NPpad; db.tc_nch = nch;
    }
    // FP16 metric factors (scaled per element) at every point in the tile-major
    // order the epilogue reads: from the curved factors or the affine records
    // (only the blocks this operand type's elemental matrix takes, whose
    // images, and so their chunk count, were built above)
    for (Block& b : m->blocks) {
        if (b.d_geom_tc || n_modes(b.shape, b.P) > (es == 2 ? kTcMaxModes16 : kTcMaxModes)) continue;
        const DeviceBlobs& db = m->blobs.at(b.shape * 16 + b.P);
        if (db.tc_nch <= 0) {   // unreachable: the image loop above set it
            set_error("tensor-core geometry layout: no reference image for the block");
            return HP_ERR_UNSUPPORTED;
        }
        hp_status st = upload<uint16_t>(&b.d_geom_tc, nullptr, (size_t)tc_geom_halves(b.n_elem, db.tc_nch));
        if (!st) st = upload<float>(&b.d_gscale_tc, nullptr, (size_t)((b.n_elem + 127) / 128 * 128 * 2));
        if (st) return st;
        const BlobLayout L = blob_layout_c(b.shape, b.P, 8);
        const double* v64 = static_cast<const double*>(db.d64);
        cudaError_t e = tc_geom_layout16(b.shape, b.curved != 0, b.d_geom, bnqp(b), b.nq, v64 + L.z, v64 + L.w, b.Q,
                                         b.d_geom_tc, b.d_gscale_tc, b.n_elem, db.tc_nch, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core geometry layout");
    }
    return HP_OK;
}

// the tensor-core elemental matrix: 256 modes (TF32), 320 (BF16, streamed backward tiles)
bool tc_fits(const Block& b, hp_dtype dt) { return n_modes(b.shape, b.P) <= (dt == HP_BF16 ? kTcMaxModes16 : kTcMaxModes); }
bool tc_hyb_fits(const Block& b, hp_dtype dt) {
    return n_modes(b.shape, b.P) <= (dt == HP_BF16 ? kTcHybMaxModes : kTcHybMaxModesTF32);
}
bool tc_strategy_fits(const Block& b, hp_dtype dt, int k) {
    return (k == HP_STRAT_ELEMAT && tc_fits(b, dt)) || (k == HP_STRAT_HYBRID && tc_hyb_fits(b, dt));
}
bool mat_fits(const Block& b) { return n_modes(b.shape, b.P) <= kMatMaxModes; }

// strategy k (HP_STRAT_SUMFAC / ELEMAT / HYBRID / MATRIX) is built for block i
// of op: derivative building blocks are sum-factorised only; a TF32 / BF16
// operator has FP32 sum factorisation, the tensor-core elemental matrix
// (N_P <= 256) and the tensor-core hybrid (N_P <= 512 BF16, 352 TF32); stored
// matrices are mass, Laplacian or Helmholtz in FP64 / FP32 (N_P <= 256)
bool strategy_available(const hp_op_s* op, size_t i, int k) {
    if (op->mesh->quadrature)   // the reduced rule: elemental matrices only (tensor cores up to 256 modes)
        return k == HP_STRAT_ELEMAT &&
               (!(op->dtype == HP_TF32 || op->dtype == HP_BF16) || tc_fits(op->mesh->blocks[i], op->dtype));
    if (k == HP_STRAT_SUMFAC) return true;
    if (needs_deriv_geom(op->kind)) return false;
    if (op->dtype == HP_TF32 || op->dtype == HP_BF16) return tc_strategy_fits(op->mesh->blocks[i], op->dtype, k);
    if (k == HP_STRAT_MATRIX)
        return (op->kind == HP_MASS || op->kind == HP_LAPLACIAN || op->kind == HP_HELMHOLTZ) &&
               mat_fits(op->mesh->blocks[i]);
    return k == HP_STRAT_ELEMAT || k == HP_STRAT_HYBRID;
}

// flops of the elemental-matrix (hybrid = false) or hybrid strategy per element
double elem_flops_dense(int shape, int P, hp_opkind k, bool hybrid, int nq = 0) {
    const int Q = P + 2;
    const double NQ = nq > 0 ? (double)nq : (double)Q * Q * Q, NP = n_modes(shape, P);
    const double deriv = 3.0 * 2.0 * Q * NQ;
    const double mv = 2.0 * NQ * NP;
    switch (k) {
        case HP_BWDTRANS: return mv;
        case HP_IPRODUCT_WRT_BASE: return mv + NQ;
        case HP_MASS: return 2 * mv + NQ;
        case HP_LAPLACIAN: return hybrid ? 2 * mv + 2 * deriv + 15 * NQ : 8 * mv + 15 * NQ;
        default: return hybrid ? 2 * mv + 2 * deriv + 18 * NQ : 8 * mv + 18 * NQ;
    }
}

// flops of the sum-factorised collocated algorithm per element (FMA = 2)
double elem_flops(int shape, int P, hp_opkind k) {
    const RefTables& t = ref_tables(shape, P);
    const int n = t.n, Q = t.Q;
    const double NQ = (double)Q * Q * Q;
    auto fam_len = [&](int s) { return s == 0 ? n : (s >= P ? 0 : P - s); };
    double c3 = 0, c2 = 0;
    for (int a = 0; a < n; ++a) {
        int blen = shape == HP_TET ? fam_len(t.famb[a]) : n;
        c2 += blen;
        for (int b = 0; b < blen; ++b) c3 += fam_len(t.famc[a * n + b]);
    }
    double bwd = 2.0 * (c3 * Q + c2 * Q * Q + n * NQ);
    double deriv = 3.0 * 2.0 * Q * NQ;
    switch (k) {
        case HP_BWDTRANS: return bwd;
        case HP_IPRODUCT_WRT_BASE: return bwd + NQ;
        case HP_MASS: return 2 * bwd + NQ;
        case HP_LAPLACIAN: return 2 * bwd + 2 * deriv + 15 * NQ;
        case HP_HELMHOLTZ: return 2 * bwd + 2 * deriv + 18 * NQ;
        case HP_ADVECTION_DIFFUSION_REACTION: return 2 * bwd + 2 * deriv + 40 * NQ;   // + velocity in eta, c . v
        case HP_PHYSDERIV: return deriv + 15 * NQ;
        default: return bwd + deriv + 18 * NQ;
    }
}

// floating-point operations the sum-factorisation kernel issues per element
// (FMA = 2): the compact eta3/eta2 passes over the valid index sets; in FP64
// the even-odd eta1 pass (u, and du/deta1 for the derivative operators, from
// the parity-form table), collocated derivatives along eta2 and eta3 only,
// the paired transposed pass with its even-odd sweeps and the eta1
// restriction of (y, w1); in FP32 the line passes of the plain algorithm
double elem_flops_exec(int shape, int P, hp_opkind k, bool fp64) {
    const int n = P + 1, Q = P + 2, Qh = (Q + 1) / 2;
    const double NQ = (double)Q * Q * Q, QQ = (double)Q * Q;
    const double npr = npairs_c(shape, P), nvl = nvalid_c(shape, P);
    const double b3 = 2.0 * Q * nvl, b2 = 2.0 * QQ * npr;
    const double r3 = b3, r2 = 2.0 * Q * Q * npr;
    if (!fp64 || k == HP_PHYSDERIV || k == HP_IPRODUCT_WRT_DERIV_BASE) return elem_flops(shape, P, k);
    const double u1 = Qh * QQ * (2.0 * n + 2.0);                 // eta1 pass, u only
    const double v1 = Qh * QQ * (2.0 * (n - 1) + 2.0);           // du/deta1 in the same pass
    const double r1_plain = 2.0 * Q * n * QQ;
    switch (k) {
        case HP_BWDTRANS: return b3 + b2 + u1;
        case HP_IPRODUCT_WRT_BASE: return NQ + r1_plain + r2 + r3;
        case HP_MASS: return b3 + b2 + u1 + NQ + r1_plain + r2 + r3;
        default: {
            const double d = 4.0 * Q * NQ;                           // eta2, eta3 derivatives
            const double dt = Qh * QQ * (8.0 * Q + 4.0);              // paired transposed pass + sweeps
            const double r1 = 4.0 * Qh * n * QQ;                      // eta1 restriction of (y, w1)
            const double metric = (k == HP_HELMHOLTZ ? 18.0 : k == HP_ADVECTION_DIFFUSION_REACTION ? 40.0 : 15.0) * NQ;
            return b3 + b2 + u1 + v1 + d + metric + dt + r1 + r2 + r3;
        }
    }
}

}  // namespace

double elem_flops_helmholtz(int shape, int P) { return elem_flops(shape, P, HP_HELMHOLTZ); }

namespace {

template <typename T>
void fill_const_tables(const Block& b, SFArgs<T>& a) {
    const RefTables& t = ref_tables(b.shape, b.P);
    for (int d = 0; d < 3; ++d)
        for (size_t i = 0; i < t.D[d].size(); ++i) a.cD[d][i] = (T)t.D[d][i];
    for (size_t i = 0; i < t.Tp.size(); ++i) a.cTa[i] = (T)t.Tp[i];
}

// the FP64 sum-factorised operator `kind` over block b (tile 0)
cudaError_t launch_sf64(hp_mesh m, const Block& b, int kind, double lambda, const double* in, double* out,
                        unsigned int* err, cudaStream_t s) {
    const DeviceBlobs& blob = m->blobs.at(b.shape * 16 + b.P);
    SFArgs<double> a{};
    a.op = kind;
    a.n_elem = b.n_elem;
    a.lambda = lambda;
    a.coeff_off = b.d_coeff_off;
    a.phys_off = b.d_phys_off;
    a.in = in;
    a.out = out;
    a.n_phys_total = m->phys_off.back();
    a.geom = b.d_geom;
    a.dgeom = b.d_dgeom;
    a.blob = static_cast<const unsigned char*>(blob.d64);
    a.blob_bytes = blob.bytes64;
    a.err = err;
    fill_const_tables(b, a);
    return sf_launch_f64(b.shape, b.P, !b.curved, 0, a, s);
}

// Stored matrices of matrix-based block bi, built (or rebuilt when lambda
// changed, Helmholtz) column by column: column n of every H^e of the block is
// the FP64 sum-factorised operator applied to the block's n-th unit
// coefficient vectors.  Synchronises s when it builds.
cudaError_t ensure_matrix(hp_op op, size_t bi, double lambda, cudaStream_t s) {
    if (op->mat.size() != op->strat.size()) {
        op->mat.assign(op->strat.size(), nullptr);
        op->mat_lambda.assign(op->strat.size(), 0.0);
    }
    if (op->mat[bi] && (op->kind != HP_HELMHOLTZ || op->mat_lambda[bi] == lambda)) return cudaSuccess;
    // a captured graph reads the stored matrices in place: rebuilding them for
    // another lambda makes it stale (hp_op_apply_graph captures afresh)
    if (op->mat[bi] && op->graph) {
        cudaGraphExecDestroy(op->graph);
        op->graph = nullptr;
    }
    // the matrices are overwritten in place: applies or graph replays already
    // queued on other streams may still read them, so every earlier piece of
    // work on the device completes first
    if (op->mat[bi]) {
        cudaError_t se = cudaDeviceSynchronize();
        if (se != cudaSuccess) return se;
    }
    hp_mesh m = op->mesh;
    const Block& b = m->blocks[bi];
    const int NP = n_modes(b.shape, b.P);
    const bool f64 = op->dtype == HP_FP64;
    const int64_t ne = b.n_elem;
    cudaError_t e = cudaSuccess;
    if (!op->mat[bi]) {
        e = cudaMalloc(&op->mat[bi], (size_t)ne * NP * NP * (f64 ? 8 : 4));
        if (e != cudaSuccess) {
            cudaGetLastError();   // an allocation failure is reported here, not by the next launch
            op->mat[bi] = nullptr;
            return e;
        }
    }
    const int64_t ncoef = m->coeff_off.back();
    double* x = nullptr;
    double* y = nullptr;
    e = cudaMalloc(&x, sizeof(double) * ncoef);
    if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(double) * ncoef);
    if (e == cudaErrorMemoryAllocation) cudaGetLastError();
    for (int col = 0; col < NP && e == cudaSuccess; ++col) {
        e = mat_unit(x, b.d_coeff_off, ne, NP, col, s);
        if (e == cudaSuccess) e = launch_sf64(m, b, op->kind, lambda, x, y, op->d_err, s);
        if (e == cudaSuccess) e = mat_collect(y, b.d_coeff_off, ne, NP, col, op->mat[bi], f64, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(x);
    cudaFree(y);
    if (e != cudaSuccess) {
        cudaFree(op->mat[bi]);
        op->mat[bi] = nullptr;
        return e;
    }
    op->mat_lambda[bi] = lambda;
    return cudaSuccess;
}

// descriptors of every block of an FP64 sum-factorised op for the work-list kernel
std::vector<SFDesc> worklist_descs(hp_op op, double lambda, const void* in, void* out) {
    hp_mesh m = op->mesh;
    std::vector<SFDesc> d(m->blocks.size());
    for (size_t i = 0; i < m->blocks.size(); ++i) {
        const Block& b = m->blocks[i];
        const DeviceBlobs& blob = m->blobs.at(b.shape * 16 + b.P);
        SFDesc& a = d[i];
        a.op = op->kind;
        a.n_elem = b.n_elem;
        a.lambda = lambda;
        for (int k = 0; k < 3; ++k) a.adv[k] = op->adv[k];
        a.coeff_off = b.d_coeff_off;
        a.phys_off = b.d_phys_off;
        a.in = static_cast<const double*>(in);
        a.out = static_cast<double*>(out);
        a.n_phys_total = m->phys_off.back();
        a.geom = affine_expanded(op, b) ? b.d_geom_pts : b.d_geom;
        a.dgeom = b.d_dgeom;
        a.blob = static_cast<const unsigned char*>(blob.d64);
        a.blob_bytes = blob.bytes64;
        a.err = op->d_err;
    }
    return d;
}

// one persistent launch over all blocks; the descriptors are copied from
// pageable host memory (the copy has consumed the host buffer when it returns)
cudaError_t launch_worklist(hp_op op, double lambda, const void* in, void* out, cudaStream_t s) {
    std::vector<SFDesc> d = worklist_descs(op, lambda, in, out);
    cudaError_t e = cudaMemcpyAsync(op->d_desc, d.data(), sizeof(SFDesc) * d.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return sf_worklist_launch(static_cast<const SFDesc*>(op->d_desc), static_cast<const WorkItem*>(op->d_items),
                              op->n_items, op->d_next, op->wl_smem, op->wl_grid, op->d_err, s);
}

cudaError_t launch_block(hp_op op, size_t bi, int tile, double lambda, const void* in, void* out, cudaStream_t s) {
    hp_mesh m = op->mesh;
    const Block& b = m->blocks[bi];
    if (op->strat[bi] == HP_STRAT_MATRIX) {
        cudaError_t e = ensure_matrix(op, bi, lambda, s);
        if (e != cudaSuccess) return e;
        return mat_apply(op->mat[bi], b.d_coeff_off, b.n_elem, n_modes(b.shape, b.P), in, out, op->dtype == HP_FP64, s);
    }
    const DeviceBlobs& blob = m->blobs.at(b.shape * 16 + b.P);
    const int64_t nphys = m->phys_off.back();
    if ((op->dtype == HP_TF32 || op->dtype == HP_BF16) && op->strat[bi] == HP_STRAT_ELEMAT) {
        const bool bf = op->dtype == HP_BF16;
        TCArgs a{};
        a.op = op->kind; a.Q = b.Q; a.NQ = b.nq; a.NQp = bnqp(b); a.NP = n_modes(b.shape, b.P);
        a.KP = bf ? blob.tc_KP16 : blob.tc_KP; a.NPpad = blob.tc_NPpad; a.nch = blob.tc_nch;
        a.es = bf ? 2 : 4;
        a.c0 = op->kind == HP_LAPLACIAN ? 1 : 0;
        a.c1 = op->kind == HP_MASS ? 1 : 4;
        a.n_elem = b.n_elem; a.lambda = (float)lambda; a.coeff_off = b.d_coeff_off;
        a.in = static_cast<const float*>(in); a.out = static_cast<float*>(out);
        a.geom16 = b.d_geom_tc;
        a.gscale = b.d_gscale_tc;
        a.img = bf ? blob.tc_img16 : blob.tc_img;
        a.chunk_bytes = bf ? blob.tc_chunk16 : blob.tc_chunk;
        a.fwd_bytes = bf ? blob.tc_fwd16 : blob.tc_fwd;
        a.bwd_bytes = bf ? blob.tc_bwd16 : blob.tc_bwd;
        // BF16: one stage per chunk (its whole forward operand, read again by the
        // backward MMAs; past 256 modes the lean variant where it fits); TF32,
        // and BF16 in mode parts: forward slices and backward tiles separately
        a.variant = tc_variant(a.KP, a.NPpad, a.fwd_bytes, a.es);
        a.stage_bytes = (bf && a.variant != 1) ? a.fwd_bytes
                                              : (std::max(4 * tc_chunk_points() * 128, a.bwd_bytes) + 1023) & ~1023;
        a.err = op->d_err;
        // split for the graph's share: BF16 always; TF32 up to 16 point chunks
        // (measured on the 16^3 mesh: TF32 at P = 5..7 ran 9-13 % slower
        // unsplit, where its longer chunks keep more CTAs busy when split)
        a.slot_share = (bi < op->tc_share.size()) ? op->tc_share[bi] : 0.0;
        a.part_out = nullptr;
        if (op->deterministic) {   // split tiles: partial outputs in a scratch of the op, summed in part order
            const int ns = tc_emat_nsplit(a);
            if (ns < 1) return cudaErrorInvalidValue;
            const int64_t need = ns > 1 ? (int64_t)ns * b.n_elem * a.NP : 0;
            if (op->part_buf.size() != op->strat.size()) {
                op->part_buf.assign(op->strat.size(), nullptr);
                op->part_cap.assign(op->strat.size(), 0);
            }
            if (need > op->part_cap[bi]) {
                cudaFree(op->part_buf[bi]);
                op->part_buf[bi] = nullptr;
                op->part_cap[bi] = 0;
                cudaError_t e = cudaMalloc(&op->part_buf[bi], sizeof(float) * (size_t)need);
                if (e != cudaSuccess) { cudaGetLastError(); op->part_buf[bi] = nullptr; return e; }
                op->part_cap[bi] = need;
            }
            a.part_out = need > 0 ? op->part_buf[bi] : nullptr;
        }
        return tc_emat_launch(a, s);
    }
    if ((op->dtype == HP_TF32 || op->dtype == HP_BF16) && op->strat[bi] == HP_STRAT_HYBRID) {
        // u = B uhat (tensor cores) -> u' = point-space core (FP32 CUDA cores) -> out = B^T u' (tensor cores)
        if (!op->hyb_u) {
            const size_t n = sizeof(float) * (size_t)std::max<int64_t>(nphys, 1);
            cudaError_t e = cudaMalloc(&op->hyb_u, n);
            if (e == cudaSuccess) e = cudaMalloc(&op->hyb_v, n);
            if (e != cudaSuccess) {
                cudaGetLastError();
                cudaFree(op->hyb_u);
                op->hyb_u = op->hyb_v = nullptr;
                return e;
            }
        }
        const bool bf = op->dtype == HP_BF16;
        HybArgs h{};
        h.NQ = b.nq; h.NP = n_modes(b.shape, b.P);
        h.KP = bf ? blob.tc_KP16 : blob.tc_KP; h.NPpad = blob.tc_NPpad; h.nch = blob.tc_nch; h.es = bf ? 2 : 4;
        h.n_elem = b.n_elem; h.coeff_off = b.d_coeff_off; h.phys_off = b.d_phys_off;
        h.img = bf ? blob.tc_img16 : blob.tc_img;
        h.chunk_bytes = bf ? blob.tc_chunk16 : blob.tc_chunk;
        h.fwd_bytes = bf ? blob.tc_fwd16 : blob.tc_fwd;
        h.bwd_bytes = bf ? blob.tc_bwd16 : blob.tc_bwd;
        h.err = op->d_err;
        h.in = static_cast<const float*>(in); h.out = op->hyb_u;
        cudaError_t e = tc_hyb_launch(h, 0, s);
        if (e != cudaSuccess) return e;
        SFArgs<float> c{};
        c.op = op->kind; c.n_elem = b.n_elem; c.lambda = (float)lambda;
        c.coeff_off = b.d_coeff_off; c.phys_off = b.d_phys_off;
        c.in = op->hyb_u; c.out = op->hyb_v; c.n_phys_total = nphys;
        c.geom = b.d_geom32; c.dgeom = b.d_dgeom32;
        c.blob = static_cast<const unsigned char*>(blob.d32); c.blob_bytes = blob.bytes32;
        c.err = op->d_err;
        c.point_io = 1;
        fill_const_tables(b, c);
        e = sf_launch_f32(b.shape, b.P, !b.curved, tile, c, s);
        if (e != cudaSuccess) return e;
        h.in = op->hyb_v; h.out = static_cast<float*>(out);
        return tc_hyb_launch(h, 1, s);
    }
    if (op->strat[bi] != HP_STRAT_SUMFAC) {
        const bool hybrid = op->strat[bi] == HP_STRAT_HYBRID;
        if (op->dtype == HP_FP64) {
            EMArgs<double> a{};
            a.op = op->kind; a.shape = b.shape; a.P = b.P; a.Q = b.Q; a.NQ = b.nq;
            a.NP = n_modes(b.shape, b.P); a.NQp = bnqp(b); a.n_elem = b.n_elem; a.lambda = lambda;
            a.coeff_off = b.d_coeff_off; a.phys_off = b.d_phys_off;
            a.in = static_cast<const double*>(in); a.out = static_cast<double*>(out);
            a.geom = b.d_geom; a.A4 = blob.A4_64; a.A4T = blob.A4T_64;
            a.blob = static_cast<const unsigned char*>(blob.d64); a.err = op->d_err;
            return emat_launch_f64(hybrid, !b.curved, a, s);
        }
        EMArgs<float> a{};
        a.op = op->kind; a.shape = b.shape; a.P = b.P; a.Q = b.Q; a.NQ = b.nq;
        a.NP = n_modes(b.shape, b.P); a.NQp = bnqp(b); a.n_elem = b.n_elem; a.lambda = (float)lambda;
        a.coeff_off = b.d_coeff_off; a.phys_off = b.d_phys_off;
        a.in = static_cast<const float*>(in); a.out = static_cast<float*>(out);
        a.geom = b.d_geom32; a.A4 = blob.A4_32; a.A4T = blob.A4T_32;
        a.blob = static_cast<const unsigned char*>(blob.d32); a.err = op->d_err;
        return emat_launch_f32(hybrid, !b.curved, a, s);
    }
    if (op->dtype == HP_FP64) {
        SFArgs<double> a{};
        a.op = op->kind;
        a.n_elem = b.n_elem;
        a.lambda = lambda;
        a.coeff_off = b.d_coeff_off;
        a.phys_off = b.d_phys_off;
        a.in = static_cast<const double*>(in);
        a.out = static_cast<double*>(out);
        a.n_phys_total = nphys;
        const bool expanded = affine_expanded(op, b);
        a.geom = expanded ? b.d_geom_pts : b.d_geom;
        a.dgeom = b.d_dgeom;
        a.blob = static_cast<const unsigned char*>(blob.d64);
        a.blob_bytes = blob.bytes64;
        a.err = op->d_err;
        for (int i = 0; i < 3; ++i) a.adv[i] = op->adv[i];
        fill_const_tables(b, a);
        if (!op->collocated && (op->kind == HP_LAPLACIAN || op->kind == HP_HELMHOLTZ))
            return sf_nc_launch(b.shape, b.P, !b.curved, a, blob.d_nc64, s);
        return sf_launch_f64(b.shape, b.P, !b.curved && !expanded, tile, a, s);
    }
    SFArgs<float> a{};
    a.op = op->kind;
    a.n_elem = b.n_elem;
    a.lambda = (float)lambda;
    a.coeff_off = b.d_coeff_off;
    a.phys_off = b.d_phys_off;
    a.in = static_cast<const float*>(in);
    a.out = static_cast<float*>(out);
    a.n_phys_total = nphys;
    a.geom = b.d_geom32;
    a.dgeom = b.d_dgeom32;
    a.blob = static_cast<const unsigned char*>(blob.d32);
    a.blob_bytes = blob.bytes32;
    a.err = op->d_err;
    for (int i = 0; i < 3; ++i) a.adv[i] = (float)op->adv[i];
    fill_const_tables(b, a);
    return sf_launch_f32(b.shape, b.P, !b.curved, tile, a, s);
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" {

const char* hp_status_str(hp_status s) {
    switch (s) {
        case HP_OK: return "HP_OK";
        case HP_ERR_ARG: return "HP_ERR_ARG";
        case HP_ERR_OOM: return "HP_ERR_OOM";
        case HP_ERR_CUDA: return "HP_ERR_CUDA";
        case HP_ERR_GEOM: return "HP_ERR_GEOM";
        case HP_ERR_UNSUPPORTED: return "HP_ERR_UNSUPPORTED";
        case HP_ERR_TIMEOUT: return "HP_ERR_TIMEOUT";
        case HP_ERR_DEVICE_BOUNDS: return "HP_ERR_DEVICE_BOUNDS";
        case HP_ERR_NOT_CONVERGED: return "HP_ERR_NOT_CONVERGED";
    }
    return "HP_ERR_UNKNOWN";
}

const char* hp_last_error(void) { return g_last_error.c_str(); }

hp_status hp_mesh_create(const hp_mesh_desc* d, int device, hp_mesh* out) {
    if (!d || !out) { set_error("hp_mesh_create: null argument"); return HP_ERR_ARG; }
    *out = nullptr;
    if (d->n_elem < 1 || !d->shape || !d->P || !d->Q || !d->vert || !d->xyz || d->n_vert < 1 || !d->curved) {
        set_error("hp_mesh_create: bad descriptor (null array or empty mesh)");
        return HP_ERR_ARG;
    }
    if (d->deformation < 0 || d->deformation > 2) { set_error("hp_mesh_create: unknown deformation"); return HP_ERR_ARG; }
    if (d->geometry < 0 || d->geometry > 1) { set_error("hp_mesh_create: geometry must be 0 or 1"); return HP_ERR_ARG; }
    if (d->quadrature < 0 || d->quadrature > 1) { set_error("hp_mesh_create: quadrature must be 0 or 1"); return HP_ERR_ARG; }
    if (d->quadrature == 1 && d->geometry == 1) {
        set_error("hp_mesh_create: the iso-parametric geometry is built on the full quadrature rule");
        return HP_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("hp_mesh_create: no such CUDA device");
        return HP_ERR_ARG;
    }
    DeviceGuard guard(device);
    auto m = new hp_mesh_s();
    m->device = device;
    m->n_elem = d->n_elem;
    m->deformation = d->deformation;
    m->geometry = d->geometry;
    m->quadrature = d->quadrature;
    m->shape.assign(d->shape, d->shape + d->n_elem);
    m->P.assign(d->P, d->P + d->n_elem);
    m->Q.assign(d->Q, d->Q + d->n_elem);
    m->curved.assign(d->curved, d->curved + d->n_elem);
    m->vert.assign(d->vert, d->vert + 8 * d->n_elem);
    m->coeff_off.assign(d->n_elem + 1, 0);
    m->phys_off.assign(d->n_elem + 1, 0);
    std::vector<double> frames(12 * d->n_elem);
    for (int64_t e = 0; e < d->n_elem; ++e) {
        int s = d->shape[e], P = d->P[e], Q = d->Q[e];
        if (s > 3) { set_error("hp_mesh_create: bad shape in element " + std::to_string(e)); delete m; return HP_ERR_ARG; }
        if (P < 1 || P > PMAX) {
            set_error("hp_mesh_create: order out of range 1..10 in element " + std::to_string(e));
            delete m;
            return P < 1 ? HP_ERR_ARG : HP_ERR_UNSUPPORTED;
        }
        if (Q != P + 2) {
            set_error("hp_mesh_create: only Q = P + 2 is built (element " + std::to_string(e) + ")");
            delete m;
            return HP_ERR_UNSUPPORTED;
        }
        double X[8][3];
        double scale = 0.0;
        for (int v = 0; v < kNV[s]; ++v) {
            int64_t id = d->vert[e * 8 + v];
            if (id < 0 || id >= d->n_vert) {
                set_error("hp_mesh_create: vertex id out of range in element " + std::to_string(e));
                delete m;
                return HP_ERR_ARG;
            }
            for (int c = 0; c < 3; ++c) X[v][c] = d->xyz[3 * id + c];
        }
        double* F = &frames[12 * e];
        for (int c = 0; c < 3; ++c) F[c] = X[0][c];
        for (int r = 0; r < 3; ++r)
            for (int ax = 0; ax < 3; ++ax) {
                F[3 + r * 3 + ax] = X[kAxis[s][ax]][r] - X[0][r];
                scale = std::max(scale, std::fabs(F[3 + r * 3 + ax]));
            }
        const double* E = F + 3;
        double det = E[0] * (E[4] * E[8] - E[5] * E[7]) - E[1] * (E[3] * E[8] - E[5] * E[6]) +
                     E[2] * (E[3] * E[7] - E[4] * E[6]);
        if (!(det > 1e-300) || !(scale > 0)) {
            set_error("hp_mesh_create: element " + std::to_string(e) + " has non-positive volume");
            delete m;
            return HP_ERR_GEOM;
        }
        for (int v = 0; v < kNV[s]; ++v)
            for (int r = 0; r < 3; ++r) {
                double y = X[0][r];
                for (int ax = 0; ax < 3; ++ax) y += E[r * 3 + ax] * 0.5 * (kRef[s][v][ax] + 1.0);
                if (std::fabs(y - X[v][r]) > 1e-10 * scale) {
                    set_error("hp_mesh_create: vertices of element " + std::to_string(e) +
                              " are not an affine image of the reference element");
                    delete m;
                    return HP_ERR_GEOM;
                }
            }
        m->coeff_off[e + 1] = m->coeff_off[e] + n_modes(s, P);
        m->phys_off[e + 1] = m->phys_off[e] + (int64_t)n_points(s, P, m->quadrature);
    }
    // blocks of equal (shape, P, curved), in order of first appearance
    std::map<std::tuple<int, int, int>, int> key2blk;
    for (int64_t e = 0; e < d->n_elem; ++e) {
        auto key = std::make_tuple((int)d->shape[e], (int)d->P[e], d->curved[e] ? 1 : 0);
        auto it = key2blk.find(key);
        if (it == key2blk.end()) {
            Block b{};
            b.shape = d->shape[e];
            b.P = d->P[e];
            b.Q = d->Q[e];
            b.curved = d->curved[e] ? 1 : 0;
            b.map_curved = b.curved;
            b.n_elem = 0;
            {
                std::vector<double> zz[3], ww[3];
                rule_points(b.shape, b.P, m->quadrature, zz, ww);
                for (int dd = 0; dd < 3; ++dd) b.q[dd] = (int)zz[dd].size();
                b.nq = b.q[0] * b.q[1] * b.q[2];
            }
            if (m->quadrature) b.curved = 1;     // the reduced rule keeps per-point factors for every block
            m->blocks.push_back(b);
            it = key2blk.emplace(key, (int)m->blocks.size() - 1).first;
        }
        m->blocks[it->second].elems.push_back(e);
    }
    hp_status st = HP_OK;
    for (Block& b : m->blocks) {
        b.n_elem = (int64_t)b.elems.size();
        std::vector<int64_t> co(b.n_elem), po(b.n_elem);
        std::vector<double> fr(12 * b.n_elem);
        for (int64_t i = 0; i < b.n_elem; ++i) {
            int64_t e = b.elems[i];
            co[i] = m->coeff_off[e];
            po[i] = m->phys_off[e];
            std::memcpy(&fr[12 * i], &frames[12 * e], 12 * sizeof(double));
            b.coeff_total += m->coeff_off[e + 1] - m->coeff_off[e];
            b.phys_total += m->phys_off[e + 1] - m->phys_off[e];
        }
        if ((st = upload(&b.d_coeff_off, co.data(), co.size()))) break;
        if ((st = upload(&b.d_phys_off, po.data(), po.size()))) break;
        if ((st = upload(&b.d_frame, fr.data(), fr.size()))) break;
        int key = b.shape * 16 + b.P;
        if (!m->blobs.count(key)) {
            const RefTables& t = ref_tables(b.shape, b.P);
            DeviceBlobs db;
            std::vector<unsigned char> b64 = make_blob(t, 8), b32 = make_blob(t, 4);
            unsigned char *p64 = nullptr, *p32 = nullptr;
            if ((st = upload(&p64, b64.data(), b64.size()))) break;
            if ((st = upload(&p32, b32.data(), b32.size()))) { cudaFree(p64); break; }
            db.d64 = p64;
            db.d32 = p32;
            db.bytes64 = (int)b64.size();
            db.bytes32 = (int)b32.size();
            std::vector<double> dtab(t.Tbd);
            dtab.insert(dtab.end(), t.Tcd.begin(), t.Tcd.end());
            if ((st = upload(&db.d_nc64, dtab.data(), dtab.size()))) { cudaFree(p64); cudaFree(p32); break; }
            if (m->quadrature) {
                std::vector<double> zz[3], ww[3], zw;
                rule_points(b.shape, b.P, 1, zz, ww);
                for (int dd = 0; dd < 3; ++dd) {
                    zw.insert(zw.end(), zz[dd].begin(), zz[dd].end());
                    zw.insert(zw.end(), ww[dd].begin(), ww[dd].end());
                }
                if ((st = upload(&db.rq_zw, zw.data(), zw.size()))) { cudaFree(p64); cudaFree(p32); cudaFree(db.d_nc64); break; }
            }
            m->blobs[key] = db;
        }
    }
    if (!st) st = upload<unsigned int>(&m->d_err, nullptr, 1);
    if (!st) {
        cudaError_t e = cudaMemset(m->d_err, 0, sizeof(unsigned int));
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemset");
    }
    if (st) {
        hp_mesh_destroy(m);
        return st;
    }
    *out = m;
    return HP_OK;
}

hp_status hp_mesh_layout(hp_mesh m, int64_t* coeff_offset, int64_t* phys_offset, int64_t* n_coeff,
                         int64_t* n_phys) {
    if (!m) { set_error("hp_mesh_layout: null mesh"); return HP_ERR_ARG; }
    if (coeff_offset) std::memcpy(coeff_offset, m->coeff_off.data(), m->coeff_off.size() * sizeof(int64_t));
    if (phys_offset) std::memcpy(phys_offset, m->phys_off.data(), m->phys_off.size() * sizeof(int64_t));
    if (n_coeff) *n_coeff = m->coeff_off.back();
    if (n_phys) *n_phys = m->phys_off.back();
    return HP_OK;
}

hp_status hp_geom_factors(hp_mesh m, void* stream) {
    if (!m) { set_error("hp_geom_factors: null mesh"); return HP_ERR_ARG; }
    DeviceGuard guard(m->device);
    if (m->geom_ready) return HP_OK;
    return compute_geom(m, false, (cudaStream_t)stream);
}

hp_status hp_geom_copy(hp_mesh m, double* out7, double* out9) {
    if (!m || !out7) { set_error("hp_geom_copy: null argument"); return HP_ERR_ARG; }
    DeviceGuard guard(m->device);
    hp_status st = ensure_geom(m, out9 != nullptr, false, 0);
    if (st) return st;
    for (const Block& b : m->blocks) {
        const int Q = b.Q, NQ = b.nq, NQp = bnqp(b);
        std::vector<double> g(geom_count(b)), h(dgeom_count(b));
        cudaError_t e = cudaMemcpy(g.data(), b.d_geom, g.size() * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "hp_geom_copy");
        if (out9 && b.curved) {
            e = cudaMemcpy(h.data(), b.d_dgeom, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(e, "hp_geom_copy");
        }
        const RefTables& t = ref_tables(b.shape, b.P);
        for (int64_t i = 0; i < b.n_elem; ++i) {
            int64_t e0 = b.elems[i];
            double* o7 = out7 + m->phys_off[e0] * 7;
            double* o9 = out9 ? out9 + m->phys_off[e0] * 9 : nullptr;
            if (b.curved) {
                for (int f = 0; f < 7; ++f)
                    for (int l = 0; l < NQ; ++l) o7[f * NQ + l] = g[(i * 7 + f) * NQp + l];
                if (o9)
                    for (int f = 0; f < 9; ++f)
                        for (int l = 0; l < NQ; ++l) o9[f * NQ + l] = h[(i * 9 + f) * NQp + l];
                continue;
            }
            // affine: expand the per-element record to the points
            const double* rec = &g[i * 16];
            for (int l = 0; l < NQ; ++l) {
                int ii = l / (Q * Q), jj = (l / Q) % Q, kk = l % Q;
                double e1 = t.z[0][ii], e2 = t.z[1][jj], e3 = t.z[2][kk];
                double T[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
                if (b.shape == HP_PRISM) { T[0][0] = 2 / (1 - e3); T[0][2] = (1 + e1) / (1 - e3); }
                if (b.shape == HP_PYR) {
                    T[0][0] = 2 / (1 - e3); T[0][2] = (1 + e1) / (1 - e3);
                    T[1][1] = 2 / (1 - e3); T[1][2] = (1 + e2) / (1 - e3);
                }
                if (b.shape == HP_TET) {
                    double r23 = 2 / ((1 - e2) * (1 - e3));
                    T[0][0] = 2 * r23; T[0][1] = (1 + e1) * r23; T[0][2] = (1 + e1) * r23;
                    T[1][1] = 2 / (1 - e3); T[1][2] = (1 + e2) / (1 - e3);
                }
                double Gx[3][3];
                for (int dd = 0; dd < 3; ++dd)
                    for (int c = 0; c < 3; ++c)
                        Gx[dd][c] = T[dd][0] * rec[7 + c] + T[dd][1] * rec[10 + c] + T[dd][2] * rec[13 + c];
                double wJ = t.w[0][ii] * t.w[1][jj] * t.w[2][kk] * rec[6];
                auto G = [&](int a, int bb) { return wJ * (Gx[a][0] * Gx[bb][0] + Gx[a][1] * Gx[bb][1] + Gx[a][2] * Gx[bb][2]); };
                o7[0 * NQ + l] = G(0, 0); o7[1 * NQ + l] = G(0, 1); o7[2 * NQ + l] = G(0, 2);
                o7[3 * NQ + l] = G(1, 1); o7[4 * NQ + l] = G(1, 2); o7[5 * NQ + l] = G(2, 2);
                o7[6 * NQ + l] = wJ;
                if (o9)
                    for (int dd = 0; dd < 3; ++dd)
                        for (int c = 0; c < 3; ++c) o9[(3 * dd + c) * NQ + l] = Gx[dd][c];
            }
        }
    }
    return HP_OK;
}

hp_status hp_op_create(hp_mesh m, hp_opkind kind, hp_strategy strategy, hp_dtype dtype, hp_op* out) {
    if (!m || !out) { set_error("hp_op_create: null argument"); return HP_ERR_ARG; }
    *out = nullptr;
    if ((int)kind < 0 || kind > HP_ADVECTION_DIFFUSION_REACTION) { set_error("hp_op_create: bad kind"); return HP_ERR_ARG; }
    if ((int)strategy < 0 || strategy > HP_STRAT_MATRIX) { set_error("hp_op_create: bad strategy"); return HP_ERR_ARG; }
    if ((int)dtype < 0 || dtype > HP_BF16) { set_error("hp_op_create: bad dtype"); return HP_ERR_ARG; }
    const bool tcore = dtype == HP_TF32 || dtype == HP_BF16;
    if (strategy == HP_STRAT_AUTO) strategy = (tcore || m->quadrature) ? HP_STRAT_ELEMAT : HP_STRAT_SUMFAC;
    if (m->quadrature) {
        bool ok = strategy == HP_STRAT_ELEMAT && (kind == HP_MASS || kind == HP_LAPLACIAN || kind == HP_HELMHOLTZ);
        if (ok && tcore)
            for (const Block& b : m->blocks) ok = ok && tc_fits(b, dtype);
        if (!ok) {
            set_error("hp_op_create: a reduced-rule mesh has the elemental-matrix mass, Laplacian and Helmholtz "
                      "operators (tensor cores: blocks of at most 256 modes)");
            return HP_ERR_UNSUPPORTED;
        }
    }
    if (tcore && ((strategy != HP_STRAT_ELEMAT && strategy != HP_STRAT_HYBRID) ||
                  (kind != HP_MASS && kind != HP_LAPLACIAN && kind != HP_HELMHOLTZ))) {
        set_error("hp_op_create: HP_TF32 / HP_BF16 are the tensor-core elemental-matrix and hybrid forms of mass, "
                  "Laplacian and Helmholtz");
        return HP_ERR_UNSUPPORTED;
    }
    if (strategy != HP_STRAT_SUMFAC && needs_deriv_geom(kind)) {
        set_error("hp_op_create: derivative building blocks and the advection-diffusion-reaction operator exist only "
                  "with HP_STRAT_SUMFAC");
        return HP_ERR_UNSUPPORTED;
    }
    if (strategy == HP_STRAT_MATRIX && kind != HP_MASS && kind != HP_LAPLACIAN && kind != HP_HELMHOLTZ) {
        set_error("hp_op_create: HP_STRAT_MATRIX stores mass, Laplacian or Helmholtz matrices");
        return HP_ERR_UNSUPPORTED;
    }
    DeviceGuard guard(m->device);
    hp_status st = ensure_geom(m, needs_deriv_geom(kind), dtype != HP_FP64, 0);
    if (st) return st;
    if (dtype == HP_FP64 && (kind == HP_LAPLACIAN || kind == HP_HELMHOLTZ) && (st = ensure_affine_points(m, 0))) return st;
    if (tcore) {
        if ((st = ensure_tc(m, dtype == HP_BF16 ? 2 : 4))) return st;
    } else if ((strategy == HP_STRAT_ELEMAT || strategy == HP_STRAT_HYBRID) && (st = ensure_dense(m))) {
        return st;
    }
    auto op = new hp_op_s();
    op->mesh = m;
    op->kind = kind;
    op->strategy = strategy;
    op->dtype = dtype;
    // every block starts on the 20 KB tile: block by block on GB300 it ran FP64
    // and FP32 sum factorisation as fast as the 56 KB one or faster (more CTAs;
    // P = 1..6 on the 16^3 mixed mesh, FP32 up to 26 % faster), the same from
    // P = 7 in FP64 (one element a CTA either way); hp_op_tune times all three
    op->tile.assign(m->blocks.size(), kDefaultTile);
    op->strat.assign(m->blocks.size(), (int)strategy);
    if (tcore)   // blocks beyond the form's tensor-memory / shared-memory budget run FP32 sum factorisation
        for (size_t i = 0; i < m->blocks.size(); ++i) {
            const Block& b = m->blocks[i];
            if (!tc_strategy_fits(b, dtype, strategy)) op->strat[i] = HP_STRAT_SUMFAC;
            // BF16 elemental matrices past 320 modes (output in parts of a tile
            // that each repeat the forward) are built but start on FP32 sum
            // factorisation, measured faster on them (hex P6 / P7, prism P8:
            // 1.4-1.7x alone; the 16^3 mesh's graph at P6 16.8 vs 25.3 GDOF/s);
            // hp_op_strategies and the schedulers can move them.  A
            // reduced-rule mesh has no sum factorisation: its blocks stay.
            if (strategy == HP_STRAT_ELEMAT && !m->quadrature && n_modes(b.shape, b.P) > kTcDefaultMaxModes16)
                op->strat[i] = HP_STRAT_SUMFAC;
        }
    if (strategy == HP_STRAT_MATRIX)   // blocks beyond the stored-matrix size run sum factorisation
        for (size_t i = 0; i < m->blocks.size(); ++i)
            if (!mat_fits(m->blocks[i])) op->strat[i] = HP_STRAT_SUMFAC;
    op->mat.assign(m->blocks.size(), nullptr);
    op->mat_lambda.assign(m->blocks.size(), 0.0);
    st = upload<unsigned int>(&op->d_err, nullptr, 1);
    if (!st) cudaMemset(op->d_err, 0, sizeof(unsigned int));
    if (st) { delete op; return st; }
    *out = op;
    return HP_OK;
}

hp_status hp_op_apply(hp_op op, double lambda, const void* in, void* out, void* stream) {
    if (!op || !in || !out) { set_error("hp_op_apply: null argument"); return HP_ERR_ARG; }
    if (in == out) { set_error("hp_op_apply: in and out must not alias"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    if (op->batching == 1) {
        cudaError_t e = launch_worklist(op, lambda, in, out, (cudaStream_t)stream);
        return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_op_apply work-list launch");
    }
    for (size_t i = 0; i < op->mesh->blocks.size(); ++i) {
        cudaError_t e = launch_block(op, i, op->tile[i], lambda, in, out, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "hp_op_apply launch");
    }
    return HP_OK;
}

hp_status hp_op_set_batching(hp_op op, int mode) {
    if (!op || (mode != 0 && mode != 1)) { set_error("hp_op_set_batching: bad argument"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    if (mode == 0) { op->batching = 0; return HP_OK; }
    const hp_mesh m = op->mesh;
    if (op->dtype != HP_FP64 || !op->collocated) {
        set_error("hp_op_set_batching: the work-list launch is for FP64 collocated sum factorisation");
        return HP_ERR_UNSUPPORTED;
    }
    for (size_t i = 0; i < m->blocks.size(); ++i)
        if (op->strat[i] != HP_STRAT_SUMFAC || m->blocks[i].P > kWorklistMaxP) {
            set_error("hp_op_set_batching: every block must be sum-factorised with P <= 8");
            return HP_ERR_UNSUPPORTED;
        }
    int smem = 0;
    for (const Block& b : m->blocks) smem = std::max(smem, sf_worklist_smem(b.shape, b.P));
    int grid = 0;
    cudaError_t e = sf_worklist_grid(smem, &grid);
    if (e != cudaSuccess) return cuda_fail(e, "hp_op_set_batching");
    // work items: each block's element groups cut into chunks of about a
    // quarter of a CTA's fair share of the total cost (FP64 operations), the
    // chunks ordered by decreasing cost so that the last items are small
    std::vector<WorkItem> items;
    std::vector<double> cost;
    double total = 0.0;
    std::vector<double> gcost(m->blocks.size());
    std::vector<int64_t> ng(m->blocks.size());
    for (size_t i = 0; i < m->blocks.size(); ++i) {
        const Block& b = m->blocks[i];
        const int epb = sf_worklist_epb(b.P);
        ng[i] = (b.n_elem + epb - 1) / epb;
        gcost[i] = epb * elem_flops_exec(b.shape, b.P, op->kind, true);
        total += gcost[i] * ng[i];
    }
    const double target = total / (4.0 * grid);
    for (size_t i = 0; i < m->blocks.size(); ++i) {
        const Block& b = m->blocks[i];
        const int64_t per = std::max<int64_t>(1, (int64_t)(target / std::max(gcost[i], 1.0)));
        for (int64_t g = 0; g < ng[i]; g += per) {
            WorkItem w;
            w.block = (int32_t)i;
            w.key = b.shape * 32 + b.P * 2 + ((b.curved || affine_expanded(op, b)) ? 0 : 1);
            w.g0 = g;
            w.g1 = std::min(ng[i], g + per);
            items.push_back(w);
            cost.push_back(gcost[i] * (double)(w.g1 - w.g0));
        }
    }
    std::vector<size_t> ord(items.size());
    for (size_t k = 0; k < ord.size(); ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<WorkItem> sorted(items.size());
    for (size_t k = 0; k < ord.size(); ++k) sorted[k] = items[ord[k]];
    cudaFree(op->d_items);
    cudaFree(op->d_desc);
    cudaFree(op->d_desc_graph);
    cudaFree(op->d_next);
    op->d_items = op->d_desc = op->d_desc_graph = nullptr;
    op->d_next = nullptr;
    hp_status st;
    WorkItem* di = nullptr;
    SFDesc *dd = nullptr, *dg = nullptr;
    if ((st = upload(&di, sorted.data(), sorted.size())) || (st = upload<SFDesc>(&dd, nullptr, m->blocks.size())) ||
        (st = upload<SFDesc>(&dg, nullptr, m->blocks.size())) || (st = upload<int>(&op->d_next, nullptr, 1))) {
        cudaFree(di);
        cudaFree(dd);
        cudaFree(dg);
        return st;
    }
    op->d_items = di;
    op->d_desc = dd;
    op->d_desc_graph = dg;
    op->n_items = (int)sorted.size();
    op->wl_smem = smem;
    op->wl_grid = grid;
    op->batching = 1;
    return HP_OK;
}

hp_status hp_op_tune(hp_op op, double lambda, const void* in, void* out, void* stream) {
    if (!op || !in || !out) { set_error("hp_op_tune: null argument"); return HP_ERR_ARG; }
    if (in == out) { set_error("hp_op_tune: in and out must not alias"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const bool f64 = op->dtype == HP_FP64;
    for (size_t i = 0; i < op->mesh->blocks.size(); ++i) {
        const Block& blk = op->mesh->blocks[i];
        if (op->strat[i] != HP_STRAT_SUMFAC) continue;
        float best = 1e30f;
        int best_t = 0;
        std::vector<int> seen;
        for (int t = 0; t < kTiles; ++t) {
            int epb = sf_epb_host(blk.P, t, f64);
            if (std::find(seen.begin(), seen.end(), epb) != seen.end()) continue;
            seen.push_back(epb);
            float tot = 0.f;
            for (int r = 0; r < 5; ++r) {
                cudaEventRecord(a, s);
                cudaError_t e = launch_block(op, i, t, lambda, in, out, s);
                cudaEventRecord(b, s);
                if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(e, "hp_op_tune"); }
                cudaError_t se = cudaEventSynchronize(b);
                if (se != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(se, "hp_op_tune"); }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (r >= 1) tot += ms;     // first launch warms up
            }
            if (tot < best) { best = tot; best_t = t; }
        }
        op->tile[i] = best_t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    return check_device_error(op->mesh, op->d_err, nullptr, "hp_op_tune");
}

hp_status hp_op_tiles(hp_op op, int* tiles, int64_t n_blocks, int set) {
    if (!op || !tiles || n_blocks != (int64_t)op->tile.size()) { set_error("hp_op_tiles: bad argument"); return HP_ERR_ARG; }
    for (int64_t i = 0; i < n_blocks; ++i) {
        if (set) {
            if (tiles[i] < 0 || tiles[i] >= kTiles) { set_error("hp_op_tiles: bad tile"); return HP_ERR_ARG; }
            op->tile[i] = tiles[i];
        } else {
            tiles[i] = op->tile[i];
        }
    }
    if (set && op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    return HP_OK;
}

hp_status hp_op_set_collocated(hp_op op, int collocated) {
    if (!op || (collocated != 0 && collocated != 1)) { set_error("hp_op_set_collocated: bad argument"); return HP_ERR_ARG; }
    if (!collocated && op->dtype != HP_FP64) {
        set_error("hp_op_set_collocated: the non-collocated form is FP64 only");
        return HP_ERR_UNSUPPORTED;
    }
    if (op->collocated != collocated && op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    op->collocated = collocated;
    if (!collocated) op->batching = 0;   // the work-list launch runs the collocated form
    return HP_OK;
}

hp_status hp_op_set_advection(hp_op op, const double* velocity) {
    if (!op || !velocity) { set_error("hp_op_set_advection: null argument"); return HP_ERR_ARG; }
    if (op->kind != HP_ADVECTION_DIFFUSION_REACTION) {
        set_error("hp_op_set_advection: the operator is not HP_ADVECTION_DIFFUSION_REACTION");
        return HP_ERR_ARG;
    }
    for (int i = 0; i < 3; ++i) op->adv[i] = velocity[i];
    if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    return HP_OK;
}

hp_status hp_op_set_deterministic(hp_op op, int deterministic) {
    if (!op || (deterministic != 0 && deterministic != 1)) {
        set_error("hp_op_set_deterministic: bad argument");
        return HP_ERR_ARG;
    }
    if (op->deterministic != deterministic && op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    op->deterministic = deterministic;
    return HP_OK;
}

hp_status hp_op_apply_graph(hp_op op, double lambda, const void* in, void* out, void* stream) {
    if (!op || !in || !out) { set_error("hp_op_apply_graph: null argument"); return HP_ERR_ARG; }
    if (in == out) { set_error("hp_op_apply_graph: in and out must not alias"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (op->batching == 1 && (!op->graph || op->g_in != in || op->g_out != out || op->g_lambda != lambda)) {
        // one persistent launch: the graph holds the counter reset and the kernel;
        // its descriptors are uploaded once, before the capture
        if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
        cudaError_t e = launch_worklist(op, lambda, in, out, s);   // warm-up (kernel attributes)
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        std::vector<SFDesc> d = worklist_descs(op, lambda, in, out);
        if (e == cudaSuccess) e = cudaMemcpy(op->d_desc_graph, d.data(), sizeof(SFDesc) * d.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "hp_op_apply_graph work-list warm-up");
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = sf_worklist_launch(static_cast<const SFDesc*>(op->d_desc_graph), static_cast<const WorkItem*>(op->d_items),
                                   op->n_items, op->d_next, op->wl_smem, op->wl_grid, op->d_err, cap);
            cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&op->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) { op->graph = nullptr; return cuda_fail(e, "hp_op_apply_graph work-list capture"); }
        op->g_in = in;
        op->g_out = out;
        op->g_lambda = lambda;
    }
    if (!op->graph || op->g_in != in || op->g_out != out || op->g_lambda != lambda) {
        if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
        const size_t nb = op->mesh->blocks.size();
        // the tensor-core blocks run concurrently in the graph: each splits its
        // tiles for its share of the GPU (the warm-up launches below size the
        // deterministic scratch with the same split)
        struct ResetShare {
            hp_op o;
            ~ResetShare() { o->tc_share.clear(); }
        } reset_share{op};
        op->tc_share.assign(nb, 0.0);
        if (op->dtype == HP_TF32 || op->dtype == HP_BF16) {
            // work of a block: tiles x point chunks x (K_P + N_P), the forward and
            // backward MMA widths; BF16 always, TF32 up to 16 chunks (measured on
            // the 16^3 mesh: TF32 at P = 5..7 ran 9-13 % slower unsplit)
            const bool bf = op->dtype == HP_BF16;
            double total = 0.0;
            for (size_t i = 0; i < nb; ++i) {
                const Block& b = op->mesh->blocks[i];
                if (op->strat[i] != HP_STRAT_ELEMAT) continue;
                const DeviceBlobs& blob = op->mesh->blobs.at(b.shape * 16 + b.P);
                if (!bf && blob.tc_nch > 16) continue;
                op->tc_share[i] = (double)((b.n_elem + 127) / 128) * blob.tc_nch *
                                  ((bf ? blob.tc_KP16 : blob.tc_KP) + blob.tc_NPpad);
                total += op->tc_share[i];
            }
            for (double& w : op->tc_share) w = total > 0.0 ? w / total : 0.0;
        }
        // first launches set kernel attributes outside the capture
        for (size_t i = 0; i < nb; ++i) {
            cudaError_t e = launch_block(op, i, op->tile[i], lambda, in, out, s);
            if (e != cudaSuccess) return cuda_fail(e, "hp_op_apply_graph warm-up");
        }
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "hp_op_apply_graph warm-up");
        const size_t np = std::min<size_t>(nb, 16);
        while (op->pool.size() < np) {
            cudaStream_t t;
            e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
            op->pool.push_back(t);
        }
        cudaStream_t cap;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        std::vector<cudaEvent_t> evs(nb + 1);
        for (auto& ev : evs) cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaEventRecord(evs[nb], cap);
            for (size_t i = 0; i < nb && e == cudaSuccess; ++i) {
                cudaStream_t si = op->pool[i % np];
                cudaStreamWaitEvent(si, evs[nb], 0);
                e = launch_block(op, i, op->tile[i], lambda, in, out, si);
                cudaEventRecord(evs[i], si);
                cudaStreamWaitEvent(cap, evs[i], 0);
            }
            cudaError_t e2 = cudaStreamEndCapture(cap, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&op->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        for (auto& ev : evs) cudaEventDestroy(ev);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) { op->graph = nullptr; return cuda_fail(e, "hp_op_apply_graph capture"); }
        op->g_in = in;
        op->g_out = out;
        op->g_lambda = lambda;
    }
    cudaError_t e = cudaGraphLaunch(op->graph, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return HP_OK;
}

hp_status hp_mesh_points(hp_mesh m, double* xyz, void* stream) {
    if (!m || !xyz) { set_error("hp_mesh_points: null argument"); return HP_ERR_ARG; }
    if (m->quadrature) { set_error("hp_mesh_points: the points of the full rule only"); return HP_ERR_UNSUPPORTED; }
    DeviceGuard guard(m->device);
    for (const Block& b : m->blocks) {
        cudaError_t e = launch_points(b, m->blobs.at(b.shape * 16 + b.P), m->deformation, xyz, m->phys_off.back(),
                                      (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "hp_mesh_points");
    }
    return HP_OK;
}

hp_status hp_op_strategies(hp_op op, int* strat, int64_t n_blocks, int set) {
    if (!op || !strat || n_blocks != (int64_t)op->strat.size()) { set_error("hp_op_strategies: bad argument"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    if (!set) {
        for (int64_t i = 0; i < n_blocks; ++i) strat[i] = op->strat[i];
        return HP_OK;
    }
    bool dense = false;
    for (int64_t i = 0; i < n_blocks; ++i) {
        if (strat[i] < HP_STRAT_SUMFAC || strat[i] > HP_STRAT_MATRIX || strat[i] == HP_STRAT_AUTO) {
            set_error("hp_op_strategies: bad strategy");
            return HP_ERR_ARG;
        }
        if (op->mesh->quadrature && !strategy_available(op, (size_t)i, strat[i])) {
            set_error("hp_op_strategies: a reduced-rule mesh runs elemental matrices only");
            return HP_ERR_UNSUPPORTED;
        }
        if (strat[i] == HP_STRAT_MATRIX &&
            ((op->kind != HP_MASS && op->kind != HP_LAPLACIAN && op->kind != HP_HELMHOLTZ) ||
             op->dtype == HP_TF32 || op->dtype == HP_BF16 || !mat_fits(op->mesh->blocks[i]))) {
            set_error("hp_op_strategies: HP_STRAT_MATRIX is for FP64 / FP32 mass, Laplacian or Helmholtz blocks of at most 256 modes");
            return HP_ERR_UNSUPPORTED;
        }
        if (strat[i] != HP_STRAT_SUMFAC && needs_deriv_geom(op->kind)) {
            set_error("hp_op_strategies: derivative building blocks exist only with HP_STRAT_SUMFAC");
            return HP_ERR_UNSUPPORTED;
        }
        if ((op->dtype == HP_TF32 || op->dtype == HP_BF16) && strat[i] != HP_STRAT_SUMFAC &&
            !tc_strategy_fits(op->mesh->blocks[i], op->dtype, strat[i])) {
            set_error("hp_op_strategies: HP_TF32 / HP_BF16 blocks are tensor-core elemental-matrix (N_P <= 256), "
                      "tensor-core hybrid (N_P <= 512 BF16, 352 TF32) or FP32 sum factorisation");
            return HP_ERR_UNSUPPORTED;
        }
        dense |= (strat[i] == HP_STRAT_ELEMAT || strat[i] == HP_STRAT_HYBRID) && op->dtype != HP_TF32 &&
                 op->dtype != HP_BF16;
    }
    if (dense) {
        hp_status st = ensure_dense(op->mesh);
        if (st) return st;
    }
    for (int64_t i = 0; i < n_blocks; ++i)
        if (strat[i] != HP_STRAT_SUMFAC) op->batching = 0;   // the work-list launch is sum factorisation only
    for (int64_t i = 0; i < n_blocks; ++i) {
        op->strat[i] = strat[i];
        if (strat[i] != HP_STRAT_MATRIX && i < (int64_t)op->mat.size() && op->mat[i]) {   // release its matrices
            cudaFree(op->mat[i]);
            op->mat[i] = nullptr;
        }
    }
    if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    return HP_OK;
}

hp_status hp_op_block_features(hp_op op, float* features, int64_t n_blocks) {
    if (!op || !features || n_blocks != (int64_t)op->strat.size()) { set_error("hp_op_block_features: bad argument"); return HP_ERR_ARG; }
    for (int64_t i = 0; i < n_blocks; ++i) {
        const Block& b = op->mesh->blocks[i];
        float* f = features + 5 * i;
        f[0] = b.shape / 3.0f;
        f[1] = b.P / 10.0f;
        f[2] = b.curved ? 1.0f : 0.0f;
        f[3] = (float)(std::log10((double)b.n_elem) / 6.0);
        f[4] = (op->dtype == HP_FP64 ? 0 : op->dtype) / 2.0f;
    }
    return HP_OK;
}

static bool matrix_room(hp_op op, size_t i);

hp_status hp_op_schedule_mlp(hp_op op, hp_mlp mlp, int graph_launch, void* stream) {
    if (!op || !mlp) { set_error("hp_op_schedule_mlp: null argument"); return HP_ERR_ARG; }
    if (graph_launch != 0 && graph_launch != 1) { set_error("hp_op_schedule_mlp: graph_launch must be 0 or 1"); return HP_ERR_ARG; }
    int n_in = 0, n_out = 0;
    hp_mlp_info(mlp, &n_in, nullptr, &n_out, nullptr);
    if ((n_in != 5 && n_in != 6) || (n_out != 3 && n_out != 4)) {
        set_error("hp_op_schedule_mlp: the network must map 5 or 6 features to 3 or 4 log-times");
        return HP_ERR_ARG;
    }
    DeviceGuard guard(op->mesh->device);
    const int64_t nb = (int64_t)op->strat.size();
    std::vector<float> f5(5 * nb), f((size_t)n_in * nb), y((size_t)n_out * nb);
    hp_op_block_features(op, f5.data(), nb);
    for (int64_t i = 0; i < nb; ++i) {
        for (int j = 0; j < 5; ++j) f[(size_t)n_in * i + j] = f5[5 * i + j];
        if (n_in == 6) f[(size_t)n_in * i + 5] = (float)graph_launch;
    }
    float *dx = nullptr, *dy = nullptr;
    hp_status st = upload(&dx, f.data(), f.size());
    if (!st) st = upload<float>(&dy, nullptr, y.size());
    if (!st) st = hp_mlp_forward(mlp, dx, nb, dy, stream);
    if (!st) {
        cudaError_t e = cudaMemcpyAsync(y.data(), dy, sizeof(float) * y.size(), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "hp_op_schedule_mlp");
    }
    cudaFree(dx);
    cudaFree(dy);
    if (st) return st;
    std::vector<int> choice(nb);
    for (int64_t i = 0; i < nb; ++i) {
        int best = 0;
        for (int k = 1; k < n_out; ++k) {
            const int strat = k == 3 ? HP_STRAT_MATRIX : k;
            if (strategy_available(op, (size_t)i, strat) && y[(size_t)n_out * i + k] < y[(size_t)n_out * i + best])
                best = k;
        }
        choice[i] = best == 3 ? HP_STRAT_MATRIX : best;
    }
    return hp_op_strategies(op, choice.data(), nb, 1);
}

hp_status hp_op_schedule(hp_op op, hp_mlp mlp, void* stream) { return hp_op_schedule_mlp(op, mlp, 0, stream); }

hp_status hp_op_schedule_exhaustive(hp_op op, double lambda, const void* in, void* out, float* times_ms,
                                    void* stream) {
    if (!op || !in || !out) { set_error("hp_op_schedule_exhaustive: null argument"); return HP_ERR_ARG; }
    if (in == out) { set_error("hp_op_schedule_exhaustive: in and out must not alias"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    op->batching = 0;
    const int64_t nb = (int64_t)op->strat.size();
    if (!needs_deriv_geom(op->kind) && op->dtype != HP_TF32 && op->dtype != HP_BF16) {
        hp_status st = ensure_dense(op->mesh);
        if (st) return st;
    }
    if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<int> saved = op->strat;
    std::vector<int> choice(nb, 0);
    // candidates in the order of the output columns: sum factorisation,
    // elemental matrix, hybrid, stored matrices (where they fit in memory)
    const int cand[4] = {HP_STRAT_SUMFAC, HP_STRAT_ELEMAT, HP_STRAT_HYBRID, HP_STRAT_MATRIX};
    for (int64_t i = 0; i < nb; ++i) {
        float best = 1e30f;
        for (int k = 0; k < 4; ++k) {
            float tot = 1e30f;
            const int sk = cand[k];
            if (strategy_available(op, (size_t)i, sk) && (sk != HP_STRAT_MATRIX || matrix_room(op, (size_t)i))) {
                op->strat[i] = sk;
                tot = 0.f;
                // the first launch warms up (and builds stored matrices), two are timed
                for (int r = 0; r < 3; ++r) {
                    cudaEventRecord(a, s);
                    cudaError_t e = launch_block(op, i, op->tile[i], lambda, in, out, s);
                    cudaEventRecord(b, s);
                    if (e == cudaSuccess) e = cudaEventSynchronize(b);
                    if (e != cudaSuccess) {
                        op->strat = saved;
                        cudaEventDestroy(a);
                        cudaEventDestroy(b);
                        return cuda_fail(e, "hp_op_schedule_exhaustive");
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, a, b);
                    if (r) tot += 0.5f * ms;
                }
                if (tot < best) { best = tot; choice[i] = sk; }
            }
            if (times_ms) times_ms[4 * i + k] = tot;
        }
        op->strat[i] = saved[i];
        if (choice[i] != HP_STRAT_MATRIX && saved[i] != HP_STRAT_MATRIX && i < (int64_t)op->mat.size() && op->mat[i]) {
            cudaFree(op->mat[i]);   // built for a trial that was not kept
            op->mat[i] = nullptr;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    hp_status st = check_device_error(op->mesh, op->d_err, nullptr, "hp_op_schedule_exhaustive");
    if (st) return st;
    return hp_op_strategies(op, choice.data(), nb, 1);
}

// the stored matrices of block i (and the build's two FP64 coefficient
// vectors) fit in half of the device's free memory
static bool matrix_room(hp_op op, size_t i) {
    if (i < op->mat.size() && op->mat[i]) return true;
    const Block& b = op->mesh->blocks[i];
    const double NP = n_modes(b.shape, b.P);
    const double need = (double)b.n_elem * NP * NP * (op->dtype == HP_FP64 ? 8.0 : 4.0) +
                        16.0 * (double)op->mesh->coeff_off.back();
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); return false; }
    return need < 0.5 * (double)free_b;
}

hp_status hp_op_schedule_graph(hp_op op, double lambda, const void* in, void* out, int reps, int passes, float* ms,
                               void* stream) {
    if (!op || !in || !out || in == out) { set_error("hp_op_schedule_graph: null or aliasing arrays"); return HP_ERR_ARG; }
    if (reps < 1 || reps > 64 || passes < 1 || passes > 8) { set_error("hp_op_schedule_graph: reps or passes out of range"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    op->batching = 0;   // the search times per-block graphs
    if (!needs_deriv_geom(op->kind) && op->dtype != HP_TF32 && op->dtype != HP_BF16) {
        hp_status st = ensure_dense(op->mesh);
        if (st) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    // median graph time of the current strategies (the graph is rebuilt first)
    auto time_graph = [&](float& t) -> hp_status {
        if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }
        hp_status st = hp_op_apply_graph(op, lambda, in, out, stream);
        if (st) return st;
        std::vector<float> v;
        for (int r = 0; r < reps; ++r) {
            cudaEventRecord(a, s);
            st = hp_op_apply_graph(op, lambda, in, out, stream);
            cudaEventRecord(b, s);
            cudaError_t e = cudaEventSynchronize(b);
            if (st) return st;
            if (e != cudaSuccess) return cuda_fail(e, "hp_op_schedule_graph");
            float x = 0.f;
            cudaEventElapsedTime(&x, a, b);
            v.push_back(x);
        }
        std::sort(v.begin(), v.end());
        t = v[v.size() / 2];
        return HP_OK;
    };
    float best = 0.f;
    hp_status st = time_graph(best);
    for (int pass = 0; pass < passes && !st; ++pass) {
        bool changed = false;
        for (size_t i = 0; i < op->strat.size() && !st; ++i) {
            const int cur = op->strat[i];
            for (int k : {HP_STRAT_SUMFAC, HP_STRAT_ELEMAT, HP_STRAT_HYBRID, HP_STRAT_MATRIX}) {
                if (st) break;
                if (k == op->strat[i] || !strategy_available(op, i, k)) continue;
                if (k == HP_STRAT_MATRIX && !matrix_room(op, i)) continue;
                const int prev = op->strat[i];
                op->strat[i] = k;
                float t = 0.f;
                st = time_graph(t);
                if (!st && t < 0.99f * best) best = t;
                else op->strat[i] = prev;
            }
            changed = changed || op->strat[i] != cur;
        }
        if (!changed) break;
    }
    if (op->graph) { cudaGraphExecDestroy(op->graph); op->graph = nullptr; }   // built for a trial
    for (size_t i = 0; i < op->mat.size(); ++i)   // matrices of trials that were not kept
        if (op->strat[i] != HP_STRAT_MATRIX && op->mat[i]) { cudaFree(op->mat[i]); op->mat[i] = nullptr; }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st) return st;
    if (ms) *ms = best;
    return check_device_error(op->mesh, op->d_err, nullptr, "hp_op_schedule_graph");
}

hp_status hp_op_sync(hp_op op, void* stream) {
    if (!op) { set_error("hp_op_sync: null op"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "hp_op_sync");
    return check_device_error(op->mesh, op->d_err, nullptr, "hp_op_sync");
}

hp_status hp_op_apply_block(hp_op op, int64_t block, double lambda, const void* in, void* out, void* stream) {
    if (!op || !in || !out) { set_error("hp_op_apply_block: null argument"); return HP_ERR_ARG; }
    if (in == out) { set_error("hp_op_apply_block: in and out must not alias"); return HP_ERR_ARG; }
    if (block < 0 || block >= (int64_t)op->mesh->blocks.size()) { set_error("hp_op_apply_block: bad block"); return HP_ERR_ARG; }
    DeviceGuard guard(op->mesh->device);
    cudaError_t e = launch_block(op, (size_t)block, op->tile[block], lambda, in, out, (cudaStream_t)stream);
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_op_apply_block launch");
}

hp_status hp_op_block_work(hp_op op, int64_t block, int64_t* n_elem, int64_t* out_dofs, double* flops,
                           double* exec_flops, double* bytes) {
    if (!op || block < -1 || block >= (int64_t)op->mesh->blocks.size()) {
        set_error("hp_op_block_work: bad argument");
        return HP_ERR_ARG;
    }
    const hp_mesh m = op->mesh;
    const double vs = op->dtype == HP_FP64 ? 8.0 : 4.0;
    int64_t dofs = 0, ne_tot = 0;
    double fl = 0, fx = 0, by = 0;
    for (const Block& b : m->blocks) {
        size_t bi = &b - &m->blocks[0];
        if (block >= 0 && (int64_t)bi != block) continue;
        const double NQ = (double)b.nq;
        const double np = (double)n_modes(b.shape, b.P);
        const double ne = (double)b.n_elem;
        ne_tot += b.n_elem;
        const int st = op->strat[bi];
        const double fd = st == HP_STRAT_SUMFAC ? elem_flops(b.shape, b.P, op->kind)
                        : st == HP_STRAT_MATRIX ? 2.0 * np * np
                                                : elem_flops_dense(b.shape, b.P, op->kind, st == HP_STRAT_HYBRID, b.nq);
        fl += ne * fd;
        fx += ne * (st == HP_STRAT_SUMFAC ? elem_flops_exec(b.shape, b.P, op->kind, op->dtype == HP_FP64) : fd);
        double in_v = coeff_in(op->kind) ? np : (op->kind == HP_IPRODUCT_WRT_DERIV_BASE ? 3 * NQ : NQ);
        double out_v = coeff_out(op->kind) ? np : (op->kind == HP_PHYSDERIV ? 3 * NQ : NQ);
        dofs += (int64_t)(ne * (coeff_out(op->kind) ? np : out_v));
        double geo = 0;
        switch (op->kind) {
            case HP_LAPLACIAN:
            case HP_HELMHOLTZ: geo = (b.curved || (st == HP_STRAT_SUMFAC && affine_expanded(op, b))) ? 7 * NQ : 7; break;
            case HP_MASS:
            case HP_IPRODUCT_WRT_BASE: geo = b.curved ? NQ : 1; break;
            case HP_PHYSDERIV: geo = b.curved ? 9 * NQ : 9; break;
            case HP_IPRODUCT_WRT_DERIV_BASE: geo = b.curved ? 10 * NQ : 10; break;
            case HP_ADVECTION_DIFFUSION_REACTION: geo = b.curved ? 16 * NQ : 16; break;
            default: geo = 0;
        }
        if (st == HP_STRAT_MATRIX) geo = np * np;   // the stored matrix takes the place of the factors
        double geo_bytes = geo * vs;
        if ((op->dtype == HP_TF32 || op->dtype == HP_BF16) && st == HP_STRAT_ELEMAT)
            // tensor-core form: FP16 factors at every point (affine ones expanded),
            // w|J| only for mass, and the element's two FP32 scales
            geo_bytes = (op->kind == HP_MASS ? 1.0 : 7.0) * NQ * 2.0 + 8.0;
        if ((op->dtype == HP_TF32 || op->dtype == HP_BF16) && st == HP_STRAT_HYBRID)
            // tensor-core hybrid: FP32 factors, and the point vectors u and u'
            // between its three kernels, each written once and read once
            geo_bytes += 16.0 * NQ;
        by += ne * ((in_v + out_v) * vs + geo_bytes + 8.0);
    }
    if (n_elem) *n_elem = ne_tot;
    if (out_dofs) *out_dofs = dofs;
    if (flops) *flops = fl;
    if (exec_flops) *exec_flops = fx;
    if (bytes) *bytes = by;
    return HP_OK;
}

hp_status hp_op_work(hp_op op, int64_t* out_dofs, double* flops, double* bytes) {
    if (!op) { set_error("hp_op_work: null op"); return HP_ERR_ARG; }
    return hp_op_block_work(op, -1, nullptr, out_dofs, flops, nullptr, bytes);
}

void hp_op_destroy(hp_op op) {
    if (!op) return;
    DeviceGuard guard(op->mesh->device);
    if (op->graph) cudaGraphExecDestroy(op->graph);
    for (cudaStream_t t : op->pool) cudaStreamDestroy(t);
    for (void* p : op->mat) cudaFree(p);
    for (float* p : op->part_buf) cudaFree(p);
    cudaFree(op->hyb_u);
    cudaFree(op->hyb_v);
    cudaFree(op->d_desc);
    cudaFree(op->d_desc_graph);
    cudaFree(op->d_items);
    cudaFree(op->d_next);
    cudaFree(op->d_err);
    delete op;
}

void hp_mesh_destroy(hp_mesh m) {
    if (!m) return;
    {
        DeviceGuard guard(m->device);
        for (Block& b : m->blocks) free_block(b);
        for (auto& kv : m->blobs) {
            cudaFree(kv.second.d64);
            cudaFree(kv.second.rq_zw);
            cudaFree(kv.second.d32);
            cudaFree(kv.second.d_nc64);
            cudaFree(kv.second.iso_RT);
            cudaFree(kv.second.iso_VT);
            cudaFree(kv.second.A4_64);
            cudaFree(kv.second.A4T_64);
            cudaFree(kv.second.A4_32);
            cudaFree(kv.second.A4T_32);
            cudaFree(kv.second.tc_img);
            cudaFree(kv.second.tc_img16);
        }
        cudaFree(m->d_err);
    }
    delete m;
}

}  // extern "C"

namespace hp {
#define HP_DECL(S, D, T) cudaError_t sf_launch_##S##_##D(int P, bool affine, int tile, const SFArgs<T>& a, cudaStream_t s);
HP_DECL(hex, f64, double) HP_DECL(prism, f64, double) HP_DECL(pyr, f64, double) HP_DECL(tet, f64, double)
HP_DECL(hex, f32, float) HP_DECL(prism, f32, float) HP_DECL(pyr, f32, float) HP_DECL(tet, f32, float)
#undef HP_DECL

cudaError_t sf_launch_f64(int shape, int P, bool affine, int tile, const SFArgs<double>& a, cudaStream_t s) {
    switch (shape) {
        case HP_HEX: return sf_launch_hex_f64(P, affine, tile, a, s);
        case HP_PRISM: return sf_launch_prism_f64(P, affine, tile, a, s);
        case HP_PYR: return sf_launch_pyr_f64(P, affine, tile, a, s);
        default: return sf_launch_tet_f64(P, affine, tile, a, s);
    }
}
cudaError_t sf_launch_f32(int shape, int P, bool affine, int tile, const SFArgs<float>& a, cudaStream_t s) {
    switch (shape) {
        case HP_HEX: return sf_launch_hex_f32(P, affine, tile, a, s);
        case HP_PRISM: return sf_launch_prism_f32(P, affine, tile, a, s);
        case HP_PYR: return sf_launch_pyr_f32(P, affine, tile, a, s);
        default: return sf_launch_tet_f32(P, affine, tile, a, s);
    }
}
}  // namespace hp
