// Assembled Helmholtz solve (paper Sec. 2.1: (grad u, grad v) + lambda (u, v)
// = (f, v) with homogeneous Dirichlet conditions; the element operators are
// the collocated sum-factorised kernels).
//
// Global <-> local: u_local = sign * u_global[gid] (gather), assembly
// y_global[g] = sum over the local copies of g of sign * y_local, done as a
// CSR transpose of the gather map in a fixed order (deterministic), with
// Dirichlet rows zeroed.  Jacobi-preconditioned CG in FP64, or iterative
// refinement with an FP64 residual around Jacobi-PCG solves in FP32 (the
// element operator then runs in FP32 sum factorisation or on the TF32 / BF16
// tensor cores instead of on the slow FP64 pipe).  Where every index fits 32
// bits the CG loop runs on 4-byte signed maps with fused kernels and one host
// round trip per iteration (pcg_fused).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hp_internal.h"

struct hp_c0_s {
    hp_mesh mesh = nullptr;
    int64_t n_local = 0, n_global = 0, n_boundary = 0;
    std::vector<int64_t> gid;
    std::vector<int8_t> sign;
    std::vector<uint8_t> bnd;
    int64_t* d_gid = nullptr;
    int8_t* d_sign = nullptr;
    int64_t* d_rowptr = nullptr;
    int64_t* d_col = nullptr;
    int8_t* d_csign = nullptr;
    uint8_t* d_bnd = nullptr;
    // solver state (created on first solve)
    hp_op op64 = nullptr, op32 = nullptr;
    int op32_mode = 0;                 // 1: FP32 sum factorisation, 2 / 3: TF32 / BF16 tensor-core elemental matrices
    int op64_sched = 0, op32_sched = 0;   // strategies chosen by the graph-aware schedule
    double diag_lambda = -1.0;
    double* d_diag = nullptr;          // assembled Jacobi diagonal (global)
    double* d_loc64[2] = {nullptr, nullptr};
    float* d_loc32[2] = {nullptr, nullptr};
    double* d_g64[6] = {};             // global FP64 work vectors
    float* d_g32[6] = {};              // global FP32 work vectors
    double* d_red = nullptr;           // reduction scratch: partial sums, then the scalars (kScal*)
    int red_blocks = 0;                // CTAs of the reducing kernels (a fixed grid: deterministic sums)
    double* h_scal = nullptr;          // pinned host copy of the scalars read each iteration
    // compact maps (local DOFs below 2^31): the index with its sign folded in
    // (i >= 0: +g[i], i < 0: -g[~i]); 4 bytes per entry instead of 9
    int32_t* d_gs32 = nullptr;         // gather: local -> signed global
    int32_t* d_rowptr32 = nullptr;     // assembly CSR (global rows over local copies)
    int32_t* d_cs32 = nullptr;
    double* d_dinv64 = nullptr;        // 1 / diag, 0 on Dirichlet rows
    float* d_dinv32 = nullptr;
};

namespace hp {
namespace {

constexpr int kRedBlocks = 1024;

template <typename T>
__global__ void gather_kernel(int64_t n, const int64_t* __restrict__ gid, const int8_t* __restrict__ sign,
                              const T* __restrict__ g, T* __restrict__ l) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) l[i] = sign[i] > 0 ? g[gid[i]] : -g[gid[i]];
}

template <typename T>
__global__ void assemble_kernel(int64_t n, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ col,
                                const int8_t* __restrict__ csign, const uint8_t* __restrict__ bnd, int mask,
                                const T* __restrict__ l, T* __restrict__ g) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; r < n; r += stride) {
        T acc = T(0);
        if (!(mask && bnd[r]))
            for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) acc += csign[k] > 0 ? l[col[k]] : -l[col[k]];
        g[r] = acc;
    }
}

// diagonal of A^T H A: each local copy contributes sign^2 = 1 times its element diagonal
__global__ void assemble_diag_kernel(int64_t n, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ col,
                                     const double* __restrict__ l, double* __restrict__ g) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; r < n; r += stride) {
        double acc = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) acc += l[col[k]];
        g[r] = acc;
    }
}

// Compact-map forms of the gather and the masked assembly (4-byte signed
// indices); each thread takes kVU entries per step with their loads issued
// first, which keeps enough bytes in flight for HBM.
constexpr int kVU = 4;

template <typename T>
__device__ __forceinline__ T signed_at(const T* __restrict__ v, int32_t i) {
    return i >= 0 ? v[i] : -v[~i];
}

template <typename T>
__global__ void gather32_kernel(int64_t n, const int32_t* __restrict__ gs, const T* __restrict__ g, T* __restrict__ l) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kVU * stride) {
        T v[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int64_t i = i0 + u * stride;
            v[u] = i < n ? signed_at(g, gs[i]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) l[i] = v[u];
        }
    }
}

// one row of the assembly: sum over the local copies of global DOF r
template <typename T>
__device__ __forceinline__ T assemble_row(int64_t r, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cs,
                                          const T* __restrict__ l) {
    T acc = T(0);
    for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) acc += signed_at(l, cs[k]);
    return acc;
}

template <typename T>
__global__ void assemble32_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cs,
                                  const uint8_t* __restrict__ bnd, int mask, const T* __restrict__ l, T* __restrict__ g) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride)
        g[r] = (mask && bnd[r]) ? T(0) : assemble_row(r, rowptr, cs, l);
}

// block sum of per-thread values into part[blockIdx.x] (fixed order)
__device__ __forceinline__ void block_sum(double acc, double* __restrict__ part) {
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// scalars kept on the device between the CG kernels
enum { kScalPQ = 0, kScalAlpha = 1, kScalRZ = 2, kScalRR = 3, kScalBeta = 4, kNumScal = 5 };

// q = masked assembly of l, with the partial sums of p.q (one per CTA)
template <typename T>
__global__ void assemble_dot_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cs,
                                    const uint8_t* __restrict__ bnd, const T* __restrict__ l, const T* __restrict__ p,
                                    T* __restrict__ q, double* __restrict__ part) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += stride) {
        const T v = bnd[r] ? T(0) : assemble_row(r, rowptr, cs, l);
        q[r] = v;
        acc += (double)p[r] * (double)v;
    }
    block_sum(acc, part);
}

// pq = sum of the partials (in order), alpha = rz / pq
__global__ void reduce_alpha_kernel(int nparts, const double* __restrict__ part, double* __restrict__ scal) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scal[kScalPQ] = sh[0];
        scal[kScalAlpha] = scal[kScalRZ] / sh[0];
    }
}

// x += alpha p, r -= alpha q, z = r / diag (0 on Dirichlet rows), with the
// partial sums of r.r and r.z (part[2 * CTA], part[2 * CTA + 1])
template <typename T>
__global__ void cg_update_kernel(int64_t n, const double* __restrict__ scal, const T* __restrict__ p,
                                 const T* __restrict__ q, const T* __restrict__ dinv, T* __restrict__ x,
                                 T* __restrict__ r, T* __restrict__ z, double* __restrict__ part) {
    const T alpha = (T)scal[kScalAlpha];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double rr = 0.0, rz = 0.0;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kVU * stride) {
        T pv[kVU], qv[kVU], xv[kVU], rv[kVU], dv[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int64_t i = i0 + u * stride;
            const bool in = i < n;
            pv[u] = in ? p[i] : T(0); qv[u] = in ? q[i] : T(0); xv[u] = in ? x[i] : T(0);
            rv[u] = in ? r[i] : T(0); dv[u] = in ? dinv[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= n) continue;
            const T rn = rv[u] - alpha * qv[u], zn = rn * dv[u];
            x[i] = xv[u] + alpha * pv[u];
            r[i] = rn;
            z[i] = zn;
            rr += (double)rn * (double)rn;
            rz += (double)rn * (double)zn;
        }
    }
    __shared__ double sh[2][256];
    sh[0][threadIdx.x] = rr;
    sh[1][threadIdx.x] = rz;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh[0][0];
        part[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// rr, rz' = sums of the partials (in order); beta = rz' / rz; rz = rz'
__global__ void reduce_beta_kernel(int nparts, const double* __restrict__ part, double* __restrict__ scal) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) { a += part[2 * i]; b += part[2 * i + 1]; }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scal[kScalRR] = sh[0][0];
        scal[kScalBeta] = sh[1][0] / scal[kScalRZ];
        scal[kScalRZ] = sh[1][0];
    }
}

// p = z + beta p (beta on the device)
template <typename T>
__global__ void xpby_dev_kernel(int64_t n, const double* __restrict__ scal, const T* __restrict__ z, T* __restrict__ p) {
    const T beta = (T)scal[kScalBeta];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += kVU * stride) {
        T zv[kVU], pv[kVU];
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int64_t i = i0 + u * stride;
            zv[u] = i < n ? z[i] : T(0);
            pv[u] = i < n ? p[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) p[i] = zv[u] + beta * pv[u];
        }
    }
}

// z = r * dinv
template <typename T>
__global__ void jacobi_dinv_kernel(int64_t n, const T* __restrict__ r, const T* __restrict__ dinv, T* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = r[i] * dinv[i];
}

// dinv = 1 / diag, 0 on Dirichlet rows
template <typename T>
__global__ void dinv_kernel(int64_t n, const double* __restrict__ diag, const uint8_t* __restrict__ bnd, T* __restrict__ dinv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dinv[i] = bnd[i] ? T(0) : (T)(1.0 / diag[i]);
}

// deterministic dot product in two stages: fixed per-block partial sums, then
// one block sums the partials in order
template <typename T>
__global__ void dot_partial_kernel(int64_t n, const T* __restrict__ a, const T* __restrict__ b, double* __restrict__ part) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(int nparts, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// y = y + a x
template <typename T>
__global__ void axpy_kernel(int64_t n, T a, const T* __restrict__ x, T* __restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * x[i];
}

// p = z + beta p
template <typename T>
__global__ void xpby_kernel(int64_t n, const T* __restrict__ z, T beta, T* __restrict__ p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

// z = r / diag (0 on Dirichlet DOFs)
template <typename T>
__global__ void jacobi_kernel(int64_t n, const T* __restrict__ r, const double* __restrict__ diag,
                              const uint8_t* __restrict__ bnd, T* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = bnd[i] ? T(0) : (T)((double)r[i] / diag[i]);
}

// r = b - q (Dirichlet rows zero)
__global__ void residual_kernel(int64_t n, const double* __restrict__ b, const double* __restrict__ q,
                                const uint8_t* __restrict__ bnd, double* __restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = bnd[i] ? 0.0 : b[i] - q[i];
}

__global__ void to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

__global__ void add_f32_to_f64(int64_t n, const float* __restrict__ d, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)d[i];
}

__global__ void fill_zero_bnd(int64_t n, const uint8_t* __restrict__ bnd, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (bnd[i]) x[i] = 0.0;
}

unsigned blocks_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

// d_red: partial sums (two per CTA of the reducing grid, at least kRedBlocks + 1
// for dot), then the kNumScal scalars
int64_t scal_offset(hp_c0 c) { return 2 * (int64_t)std::max(c->red_blocks, kRedBlocks + 1); }

template <typename T>
hp_status dot(hp_c0 c, const T* a, const T* b, int64_t n, double* host, cudaStream_t s) {
    dot_partial_kernel<T><<<kRedBlocks, 256, 0, s>>>(n, a, b, c->d_red);
    dot_final_kernel<<<1, 256, 0, s>>>(kRedBlocks, c->d_red, c->d_red + kRedBlocks);
    cudaError_t e = cudaMemcpyAsync(host, c->d_red + kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_solve dot");
}

// gather (local = sign * global[gid]) and assembly with the compact maps when
// they exist, else the 8-byte ones
template <typename T>
void launch_gather(hp_c0 c, const T* g, T* l, cudaStream_t s) {
    if (c->d_gs32) gather32_kernel<T><<<blocks_for(c->n_local), 256, 0, s>>>(c->n_local, c->d_gs32, g, l);
    else gather_kernel<T><<<blocks_for(c->n_local), 256, 0, s>>>(c->n_local, c->d_gid, c->d_sign, g, l);
}
template <typename T>
void launch_assemble(hp_c0 c, const T* l, T* g, int mask, cudaStream_t s) {
    if (c->d_cs32)
        assemble32_kernel<T><<<blocks_for(c->n_global), 256, 0, s>>>(c->n_global, c->d_rowptr32, c->d_cs32, c->d_bnd,
                                                                    mask, l, g);
    else
        assemble_kernel<T><<<blocks_for(c->n_global), 256, 0, s>>>(c->n_global, c->d_rowptr, c->d_col, c->d_csign,
                                                                  c->d_bnd, mask, l, g);
}

// q = mask(A^T H_e A p): gather, element Helmholtz, assembly
template <typename T>
hp_status apply_global(hp_c0 c, hp_op op, double lambda, const T* p, T* q, T* l0, T* l1, cudaStream_t s) {
    launch_gather<T>(c, p, l0, s);
    hp_status st = hp_op_apply(op, lambda, l0, l1, s);
    if (st) return st;
    launch_assemble<T>(c, l1, q, 1, s);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_solve apply");
}

template <typename T>
hp_status alloc(T** p, int64_t n) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * std::max<int64_t>(n, 1));
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_solve workspace");
}

hp_status prepare(hp_c0 c, double lambda, int mixed, int schedule, cudaStream_t s) {
    hp_status st;
    if (!schedule && c->op64_sched) {   // back to the default strategies
        hp_op_destroy(c->op64);
        c->op64 = nullptr;
        c->op64_sched = 0;
    }
    if (!c->op64 && (st = hp_op_create(c->mesh, HP_HELMHOLTZ, HP_STRAT_SUMFAC, HP_FP64, &c->op64))) return st;
    if (mixed && c->op32 && (c->op32_mode != mixed || (!schedule && c->op32_sched))) {
        hp_op_destroy(c->op32);
        c->op32 = nullptr;
        c->op32_sched = 0;
    }
    if (mixed && !c->op32) {
        st = mixed == 3 ? hp_op_create(c->mesh, HP_HELMHOLTZ, HP_STRAT_ELEMAT, HP_BF16, &c->op32)
           : mixed == 2 ? hp_op_create(c->mesh, HP_HELMHOLTZ, HP_STRAT_ELEMAT, HP_TF32, &c->op32)
                        : hp_op_create(c->mesh, HP_HELMHOLTZ, HP_STRAT_SUMFAC, HP_FP32, &c->op32);
        if (st) return st;
        // split tensor-core tiles summed in a fixed order: the solve is reproducible
        if ((st = hp_op_set_deterministic(c->op32, 1))) return st;
        c->op32_mode = mixed;
    }
    if (!c->d_red) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c->red_blocks = std::max(1, sms) * 8;          // eight 256-thread CTAs per SM
        if ((st = alloc(&c->d_red, scal_offset(c) + kNumScal))) return st;
        cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&c->h_scal), sizeof(double) * kNumScal);
        if (e != cudaSuccess) return cuda_fail(e, "hp_solve pinned scalars");
    }
    for (int i = 0; i < 2; ++i)
        if (!c->d_loc64[i] && (st = alloc(&c->d_loc64[i], c->n_local))) return st;
    for (int i = 0; i < 6; ++i)
        if (!c->d_g64[i] && (st = alloc(&c->d_g64[i], c->n_global))) return st;
    if (mixed) {
        for (int i = 0; i < 2; ++i)
            if (!c->d_loc32[i] && (st = alloc(&c->d_loc32[i], c->n_local))) return st;
        for (int i = 0; i < 6; ++i)
            if (!c->d_g32[i] && (st = alloc(&c->d_g32[i], c->n_global))) return st;
    }
    if (c->diag_lambda != lambda) {
        if (!c->d_diag && (st = alloc(&c->d_diag, c->n_global))) return st;
        // element diagonals need the dense reference matrices
        hp_op tmp = nullptr;
        if ((st = hp_op_create(c->mesh, HP_MASS, HP_STRAT_ELEMAT, HP_FP64, &tmp))) return st;
        hp_op_destroy(tmp);
        for (const Block& b : c->mesh->blocks) {
            cudaError_t e = launch_elem_diag(b, c->mesh->blobs.at(b.shape * 16 + b.P), lambda, c->d_loc64[0], s);
            if (e != cudaSuccess) return cuda_fail(e, "element diagonal");
        }
        assemble_diag_kernel<<<blocks_for(c->n_global), 256, 0, s>>>(c->n_global, c->d_rowptr, c->d_col,
                                                                    c->d_loc64[0], c->d_diag);
        if (!c->d_dinv64 && (st = alloc(&c->d_dinv64, c->n_global))) return st;
        if (!c->d_dinv32 && (st = alloc(&c->d_dinv32, c->n_global))) return st;
        dinv_kernel<double><<<blocks_for(c->n_global), 256, 0, s>>>(c->n_global, c->d_diag, c->d_bnd, c->d_dinv64);
        dinv_kernel<float><<<blocks_for(c->n_global), 256, 0, s>>>(c->n_global, c->d_diag, c->d_bnd, c->d_dinv32);
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "element diagonal");
        c->diag_lambda = lambda;
    }
    // graph-aware strategy choice, timed on the local work vectors (zeroed)
    if (schedule && !c->op64_sched) {
        cudaError_t e = cudaMemsetAsync(c->d_loc64[0], 0, sizeof(double) * c->n_local, s);
        if (e != cudaSuccess) return cuda_fail(e, "hp_solve schedule");
        if ((st = hp_op_schedule_graph(c->op64, lambda, c->d_loc64[0], c->d_loc64[1], 5, 1, nullptr, s))) return st;
        c->op64_sched = 1;
    }
    if (schedule && mixed && !c->op32_sched) {
        cudaError_t e = cudaMemsetAsync(c->d_loc32[0], 0, sizeof(float) * c->n_local, s);
        if (e != cudaSuccess) return cuda_fail(e, "hp_solve schedule");
        if ((st = hp_op_schedule_graph(c->op32, lambda, c->d_loc32[0], c->d_loc32[1], 5, 1, nullptr, s))) return st;
        c->op32_sched = 1;
    }
    return HP_OK;
}

// Jacobi-PCG on A x = b in precision T; x holds the initial guess; returns the
// iteration count and the final relative residual (||r|| / ||b||, FP64 dots).
template <typename T>
hp_status pcg(hp_c0 c, hp_op op, double lambda, const T* b, T* x, T* r, T* z, T* p, T* q, T* l0, T* l1,
              double tol, int max_iter, bool x_is_zero, int* iters, double* relres, cudaStream_t s) {
    const int64_t n = c->n_global;
    hp_status st;
    double bb = 0, rz = 0, rr = 0;
    if ((st = dot(c, b, b, n, &bb, s))) return st;
    const double bnorm = std::sqrt(bb);
    if (x_is_zero) {
        cudaMemcpyAsync(r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
    } else {
        if ((st = apply_global(c, op, lambda, x, q, l0, l1, s))) return st;
        cudaMemcpyAsync(r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
        axpy_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, T(-1), q, r);
    }
    if ((st = dot(c, r, r, n, &rr, s))) return st;
    *iters = 0;
    *relres = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
    if (bnorm == 0 || *relres <= tol) return HP_OK;
    jacobi_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, r, c->d_diag, c->d_bnd, z);
    cudaMemcpyAsync(p, z, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
    if ((st = dot(c, r, z, n, &rz, s))) return st;
    for (int it = 1; it <= max_iter; ++it) {
        if ((st = apply_global(c, op, lambda, p, q, l0, l1, s))) return st;
        double pq = 0;
        if ((st = dot(c, p, q, n, &pq, s))) return st;
        if (!(pq > 0)) {
            set_error("hp_solve: CG breakdown (p^T A p = " + std::to_string(pq) + " at iteration " +
                      std::to_string(it) + ", r.z = " + std::to_string(rz) + ", ||b|| = " + std::to_string(bnorm) + ")");
            return HP_ERR_NOT_CONVERGED;
        }
        const double alpha = rz / pq;
        axpy_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, (T)alpha, p, x);
        axpy_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, (T)(-alpha), q, r);
        if ((st = dot(c, r, r, n, &rr, s))) return st;
        *iters = it;
        *relres = std::sqrt(rr) / bnorm;
        if (!std::isfinite(*relres)) {
            set_error("hp_solve: residual is not finite");
            return HP_ERR_NOT_CONVERGED;
        }
        if (*relres <= tol) return HP_OK;
        jacobi_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, r, c->d_diag, c->d_bnd, z);
        double rz_new = 0;
        if ((st = dot(c, r, z, n, &rz_new, s))) return st;
        const double beta = rz_new / rz;
        rz = rz_new;
        xpby_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, z, (T)beta, p);
    }
    set_error("hp_solve: CG did not reach the tolerance in the iteration limit");
    return HP_ERR_NOT_CONVERGED;
}

template <typename T>
const T* dinv_of(hp_c0 c);
template <>
const double* dinv_of<double>(hp_c0 c) { return c->d_dinv64; }
template <>
const float* dinv_of<float>(hp_c0 c) { return c->d_dinv32; }

// The same Jacobi-PCG with the compact maps and fused kernels: per iteration
// gather, element operator, assembly with the p.q partial sums, alpha on the
// device, one update pass (x, r, z with the r.r and r.z partial sums), beta on
// the device, one copy of the scalars to the host (the only synchronisation:
// convergence and breakdown checks), p = z + beta p.  Same arithmetic as pcg
// (FP64 dot products, sums in a fixed order).
template <typename T>
hp_status pcg_fused(hp_c0 c, hp_op op, double lambda, const T* b, T* x, T* r, T* z, T* p, T* q, T* l0, T* l1,
                    double tol, int max_iter, bool x_is_zero, int* iters, double* relres, cudaStream_t s) {
    const int64_t n = c->n_global;
    const T* dinv = dinv_of<T>(c);
    double* part = c->d_red;
    double* scal = c->d_red + scal_offset(c);
    const int G = c->red_blocks;
    hp_status st;
    double bb = 0, rz = 0, rr = 0;
    if ((st = dot(c, b, b, n, &bb, s))) return st;
    const double bnorm = std::sqrt(bb);
    if (x_is_zero) {
        cudaMemcpyAsync(r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
    } else {
        if ((st = apply_global(c, op, lambda, x, q, l0, l1, s))) return st;
        cudaMemcpyAsync(r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
        axpy_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, T(-1), q, r);
    }
    if ((st = dot(c, r, r, n, &rr, s))) return st;
    *iters = 0;
    *relres = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
    if (bnorm == 0 || *relres <= tol) return HP_OK;
    jacobi_dinv_kernel<T><<<blocks_for(n), 256, 0, s>>>(n, r, dinv, z);
    cudaMemcpyAsync(p, z, sizeof(T) * n, cudaMemcpyDeviceToDevice, s);
    if ((st = dot(c, r, z, n, &rz, s))) return st;       // synchronises: h_scal is free
    c->h_scal[kScalRZ] = rz;
    cudaMemcpyAsync(scal + kScalRZ, c->h_scal + kScalRZ, sizeof(double), cudaMemcpyHostToDevice, s);
    for (int it = 1; it <= max_iter; ++it) {
        launch_gather<T>(c, p, l0, s);
        if ((st = hp_op_apply(op, lambda, l0, l1, s))) return st;
        assemble_dot_kernel<T><<<G, 256, 0, s>>>(n, c->d_rowptr32, c->d_cs32, c->d_bnd, l1, p, q, part);
        reduce_alpha_kernel<<<1, 256, 0, s>>>(G, part, scal);
        cg_update_kernel<T><<<G, 256, 0, s>>>(n, scal, p, q, dinv, x, r, z, part);
        const double rz_old = c->h_scal[kScalRZ];
        reduce_beta_kernel<<<1, 256, 0, s>>>(G, part, scal);
        cudaError_t e = cudaMemcpyAsync(c->h_scal, scal, sizeof(double) * kNumScal, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "hp_solve iteration");
        const double pq = c->h_scal[kScalPQ];
        rr = c->h_scal[kScalRR];
        if (!(pq > 0)) {
            set_error("hp_solve: CG breakdown (p^T A p = " + std::to_string(pq) + " at iteration " +
                      std::to_string(it) + ", r.z = " + std::to_string(rz_old) + ", ||b|| = " + std::to_string(bnorm) + ")");
            return HP_ERR_NOT_CONVERGED;
        }
        *iters = it;
        *relres = std::sqrt(rr) / bnorm;
        if (!std::isfinite(*relres)) {
            set_error("hp_solve: residual is not finite");
            return HP_ERR_NOT_CONVERGED;
        }
        if (*relres <= tol) return HP_OK;
        xpby_dev_kernel<T><<<G, 256, 0, s>>>(n, scal, z, p);
    }
    set_error("hp_solve: CG did not reach the tolerance in the iteration limit");
    return HP_ERR_NOT_CONVERGED;
}

// the fused loop where the compact maps exist, else the plain one
template <typename T>
hp_status pcg_run(hp_c0 c, hp_op op, double lambda, const T* b, T* x, T* r, T* z, T* p, T* q, T* l0, T* l1,
                  double tol, int max_iter, bool x_is_zero, int* iters, double* relres, cudaStream_t s) {
    if (c->d_cs32)
        return pcg_fused<T>(c, op, lambda, b, x, r, z, p, q, l0, l1, tol, max_iter, x_is_zero, iters, relres, s);
    return pcg<T>(c, op, lambda, b, x, r, z, p, q, l0, l1, tol, max_iter, x_is_zero, iters, relres, s);
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" {

hp_status hp_c0_create(hp_mesh mesh, hp_c0* out) {
    if (!mesh || !out) { set_error("hp_c0_create: null argument"); return HP_ERR_ARG; }
    *out = nullptr;
    if (mesh->quadrature) {
        set_error("hp_c0_create: the C0 space and its solves use the sum-factorised operators of the full rule");
        return HP_ERR_UNSUPPORTED;
    }
    cudaSetDevice(mesh->device);
    auto c = new hp_c0_s();
    c->mesh = mesh;
    c->n_local = mesh->coeff_off.back();
    hp_status st = build_c0(mesh, mesh->vert, c->gid, c->sign, c->bnd, c->n_global);
    if (st) { delete c; return st; }
    for (uint8_t b : c->bnd) c->n_boundary += b;
    // CSR transpose of the gather map: local copies of each global DOF in local order
    std::vector<int64_t> rowptr(c->n_global + 1, 0), col(c->n_local);
    std::vector<int8_t> csign(c->n_local);
    for (int64_t i = 0; i < c->n_local; ++i) rowptr[c->gid[i] + 1] += 1;
    for (int64_t g = 0; g < c->n_global; ++g) rowptr[g + 1] += rowptr[g];
    std::vector<int64_t> fill(rowptr.begin(), rowptr.end() - 1);
    for (int64_t i = 0; i < c->n_local; ++i) {
        int64_t k = fill[c->gid[i]]++;
        col[k] = i;
        csign[k] = c->sign[i];
    }
    auto up = [&](auto** dst, const auto* src, int64_t n) -> hp_status {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), sizeof(**dst) * std::max<int64_t>(n, 1));
        if (e == cudaSuccess) e = cudaMemcpy(*dst, src, sizeof(**dst) * n, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_c0_create upload");
    };
    if ((st = up(&c->d_gid, c->gid.data(), c->n_local)) || (st = up(&c->d_sign, c->sign.data(), c->n_local)) ||
        (st = up(&c->d_rowptr, rowptr.data(), c->n_global + 1)) || (st = up(&c->d_col, col.data(), c->n_local)) ||
        (st = up(&c->d_csign, csign.data(), c->n_local)) || (st = up(&c->d_bnd, c->bnd.data(), c->n_global))) {
        hp_c0_destroy(c);
        return st;
    }
    // compact maps for the solver's gather and assembly: the sign folded into a
    // 4-byte index (i for +, ~i for -), where every index fits
    if (c->n_local < ((int64_t)1 << 31) && c->n_global < ((int64_t)1 << 31)) {
        std::vector<int32_t> gs(c->n_local), rp(c->n_global + 1), cs(c->n_local);
        for (int64_t i = 0; i < c->n_local; ++i) gs[i] = c->sign[i] > 0 ? (int32_t)c->gid[i] : ~(int32_t)c->gid[i];
        for (int64_t g = 0; g <= c->n_global; ++g) rp[g] = (int32_t)rowptr[g];
        for (int64_t k = 0; k < c->n_local; ++k) cs[k] = csign[k] > 0 ? (int32_t)col[k] : ~(int32_t)col[k];
        if ((st = up(&c->d_gs32, gs.data(), c->n_local)) || (st = up(&c->d_rowptr32, rp.data(), c->n_global + 1)) ||
            (st = up(&c->d_cs32, cs.data(), c->n_local))) {
            hp_c0_destroy(c);
            return st;
        }
    }
    *out = c;
    return HP_OK;
}

hp_status hp_c0_map_host(const hp_mesh_desc* d, int64_t* gid, int8_t* sign, uint8_t* boundary, int64_t* n_global) {
    if (!d || !gid || !sign || !boundary || !n_global || d->n_elem < 1 || !d->shape || !d->P || !d->vert) {
        set_error("hp_c0_map_host: null argument");
        return HP_ERR_ARG;
    }
    hp_mesh_s m;
    m.n_elem = d->n_elem;
    m.shape.assign(d->shape, d->shape + d->n_elem);
    m.P.assign(d->P, d->P + d->n_elem);
    m.vert.assign(d->vert, d->vert + 8 * d->n_elem);
    m.coeff_off.assign(d->n_elem + 1, 0);
    for (int64_t e = 0; e < d->n_elem; ++e) {
        if (d->shape[e] > 3 || d->P[e] < 1 || d->P[e] > PMAX) { set_error("hp_c0_map_host: bad shape or order"); return HP_ERR_ARG; }
        m.coeff_off[e + 1] = m.coeff_off[e] + n_modes(d->shape[e], d->P[e]);
    }
    std::vector<int64_t> g;
    std::vector<int8_t> sg;
    std::vector<uint8_t> b;
    int64_t ng = 0;
    hp_status st = build_c0(&m, m.vert, g, sg, b, ng);
    if (st) return st;
    std::copy(g.begin(), g.end(), gid);
    std::copy(sg.begin(), sg.end(), sign);
    std::copy(b.begin(), b.end(), boundary);
    *n_global = ng;
    return HP_OK;
}

hp_status hp_c0_info(hp_c0 c, int64_t* n_global, int64_t* n_boundary) {
    if (!c) { set_error("hp_c0_info: null"); return HP_ERR_ARG; }
    if (n_global) *n_global = c->n_global;
    if (n_boundary) *n_boundary = c->n_boundary;
    return HP_OK;
}

hp_status hp_c0_maps(hp_c0 c, int64_t* gid, int8_t* sign, uint8_t* boundary) {
    if (!c) { set_error("hp_c0_maps: null"); return HP_ERR_ARG; }
    if (gid) std::copy(c->gid.begin(), c->gid.end(), gid);
    if (sign) std::copy(c->sign.begin(), c->sign.end(), sign);
    if (boundary) std::copy(c->bnd.begin(), c->bnd.end(), boundary);
    return HP_OK;
}

hp_status hp_c0_gather(hp_c0 c, const double* global, double* local, void* stream) {
    if (!c || !global || !local) { set_error("hp_c0_gather: null argument"); return HP_ERR_ARG; }
    launch_gather<double>(c, global, local, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_c0_gather");
}

hp_status hp_c0_assemble(hp_c0 c, const double* local, double* global, int mask_boundary, void* stream) {
    if (!c || !global || !local) { set_error("hp_c0_assemble: null argument"); return HP_ERR_ARG; }
    launch_assemble<double>(c, local, global, mask_boundary ? 1 : 0, (cudaStream_t)stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_c0_assemble");
}

hp_status hp_c0_diagonal(hp_c0 c, double lambda, double* diag, int local, void* stream) {
    if (!c || !diag) { set_error("hp_c0_diagonal: null argument"); return HP_ERR_ARG; }
    cudaSetDevice(c->mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    hp_status st = prepare(c, lambda, 0, c->op64_sched, s);   // keeps the operators' strategies
    if (st) return st;
    cudaError_t e;
    if (local) {
        for (const Block& b : c->mesh->blocks) {
            e = launch_elem_diag(b, c->mesh->blobs.at(b.shape * 16 + b.P), lambda, diag, s);
            if (e != cudaSuccess) return cuda_fail(e, "hp_c0_diagonal");
        }
        return HP_OK;
    }
    e = cudaMemcpyAsync(diag, c->d_diag, sizeof(double) * c->n_global, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_c0_diagonal");
}

hp_status hp_solve(hp_c0 c, double lambda, const double* rhs, double* x, const hp_solve_opts* opts,
                   hp_solve_stats* stats, void* stream) {
    if (!c || !rhs || !x || !opts) { set_error("hp_solve: null argument"); return HP_ERR_ARG; }
    if (!(opts->tol > 0) || opts->max_iter < 1 || opts->mixed < 0 || opts->mixed > 3 || opts->schedule < 0 ||
        opts->schedule > 1 ||
        (opts->mixed && (!(opts->inner_tol > 0) || opts->inner_max_iter < 1 || opts->max_refinements < 1))) {
        set_error("hp_solve: bad options");
        return HP_ERR_ARG;
    }
    cudaSetDevice(c->mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    hp_status st = prepare(c, lambda, opts->mixed, opts->schedule, s);
    if (st) return st;
    const int64_t n = c->n_global;
    hp_solve_stats S{};
    fill_zero_bnd<<<blocks_for(n), 256, 0, s>>>(n, c->d_bnd, x);
    double* b = c->d_g64[0];
    cudaMemcpyAsync(b, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    fill_zero_bnd<<<blocks_for(n), 256, 0, s>>>(n, c->d_bnd, b);
    if (!opts->mixed) {
        int it = 0;
        double rel = 0;
        st = pcg_run<double>(c, c->op64, lambda, b, x, c->d_g64[1], c->d_g64[2], c->d_g64[3], c->d_g64[4],
                         c->d_loc64[0], c->d_loc64[1], opts->tol, opts->max_iter, false, &it, &rel, s);
        S.iterations = it;
        S.rel_residual = rel;
    } else {
        // iterative refinement: FP64 residual, FP32 Jacobi-PCG correction
        double bb = 0;
        if ((st = dot(c, b, b, n, &bb, s))) return st;
        const double bnorm = std::sqrt(bb);
        double* r = c->d_g64[1];
        double* q = c->d_g64[2];
        float* r32 = c->d_g32[0];
        float* d32 = c->d_g32[1];
        for (int k = 0; k < opts->max_refinements; ++k) {
            if ((st = apply_global<double>(c, c->op64, lambda, x, q, c->d_loc64[0], c->d_loc64[1], s))) return st;
            residual_kernel<<<blocks_for(n), 256, 0, s>>>(n, b, q, c->d_bnd, r);
            double rr = 0;
            if ((st = dot(c, r, r, n, &rr, s))) return st;
            S.rel_residual = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
            S.refinements = k;
            if (S.rel_residual <= opts->tol) break;
            to_f32<<<blocks_for(n), 256, 0, s>>>(n, r, r32);
            cudaMemsetAsync(d32, 0, sizeof(float) * n, s);
            int it = 0;
            double rel = 0;
            st = pcg_run<float>(c, c->op32, lambda, r32, d32, c->d_g32[2], c->d_g32[3], c->d_g32[4], c->d_g32[5],
                            c->d_loc32[0], c->d_loc32[1], opts->inner_tol, opts->inner_max_iter, true, &it, &rel, s);
            S.inner_iterations += it;
            if (st && st != HP_ERR_NOT_CONVERGED) return st;
            add_f32_to_f64<<<blocks_for(n), 256, 0, s>>>(n, d32, x);
            S.refinements = k + 1;
        }
        if (S.rel_residual > opts->tol) {
            // one last residual after the final correction
            if ((st = apply_global<double>(c, c->op64, lambda, x, q, c->d_loc64[0], c->d_loc64[1], s))) return st;
            residual_kernel<<<blocks_for(n), 256, 0, s>>>(n, b, q, c->d_bnd, r);
            double rr = 0;
            if ((st = dot(c, r, r, n, &rr, s))) return st;
            S.rel_residual = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
        }
        S.iterations = S.inner_iterations;
        st = S.rel_residual <= opts->tol ? HP_OK : HP_ERR_NOT_CONVERGED;
        if (st) set_error("hp_solve: refinement did not reach the tolerance");
    }
    if (stats) *stats = S;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "hp_solve");
    return st;
}

void hp_c0_destroy(hp_c0 c) {
    if (!c) return;
    cudaSetDevice(c->mesh->device);
    cudaFree(c->d_gid); cudaFree(c->d_sign); cudaFree(c->d_rowptr); cudaFree(c->d_col); cudaFree(c->d_csign);
    cudaFree(c->d_bnd); cudaFree(c->d_diag); cudaFree(c->d_red);
    cudaFree(c->d_gs32); cudaFree(c->d_rowptr32); cudaFree(c->d_cs32); cudaFree(c->d_dinv64); cudaFree(c->d_dinv32);
    if (c->h_scal) cudaFreeHost(c->h_scal);
    for (auto* p : c->d_loc64) cudaFree(p);
    for (auto* p : c->d_loc32) cudaFree(p);
    for (auto* p : c->d_g64) cudaFree(p);
    for (auto* p : c->d_g32) cudaFree(p);
    if (c->op64) hp_op_destroy(c->op64);
    if (c->op32) hp_op_destroy(c->op32);
    delete c;
}

}  // extern "C"
