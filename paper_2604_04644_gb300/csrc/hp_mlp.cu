// Cost-model network: a small MLP (n_in -> H -> H -> n_out, ReLU, FP32) with
// its own forward, backward and Adam kernels.  Not in the paper: it predicts
// the log run time of each implementation strategy of an element block so the
// library can pick one per block (the paper picks by a fixed rule, Sec. 4).
//
// Parameters live in one flat device array, in this order:
//   W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H], b3 [n_out].
// Loss: mean squared error over batch and outputs,
//   L = 1/(B n_out) sum_s sum_o (y_so - t_so)^2.
// Gradients are reduced over samples deterministically (per-sample rows, then
// a fixed-order column sum), so training is bitwise reproducible.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hp_internal.h"

struct hp_mlp_s {
    int device = 0, n_in = 0, H = 0, n_out = 0;
    int64_t n_params = 0;
    float* d_params = nullptr;
    float* d_m = nullptr;      // Adam first moment
    float* d_v = nullptr;      // Adam second moment
    float* d_grad = nullptr;
    float* d_rows = nullptr;   // per-sample gradient rows (capacity cap_rows samples)
    float* d_act = nullptr;    // activations for backward: z1, z2 per sample
    float* d_y = nullptr;      // outputs per sample
    float* d_loss_rows = nullptr;
    int64_t cap = 0;
    int64_t step = 0;
};

namespace hp {
namespace {

struct Off {
    int64_t W1, b1, W2, b2, W3, b3, n;
};
Off offsets(int n_in, int H, int n_out) {
    Off o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)H * n_in;
    o.W2 = o.b1 + H;
    o.b2 = o.W2 + (int64_t)H * H;
    o.W3 = o.b2 + H;
    o.b3 = o.W3 + (int64_t)n_out * H;
    o.n = o.b3 + n_out;
    return o;
}

constexpr int kMaxH = 256;
constexpr int kMaxIn = 16;
constexpr int kMaxOut = 8;

// one CTA (H threads) per sample: forward pass, keeping z1, z2 for backward
__global__ void mlp_forward_kernel(const float* __restrict__ p, int n_in, int H, int n_out, Off o,
                                   const float* __restrict__ x, int64_t B, float* __restrict__ y,
                                   float* __restrict__ act) {
    __shared__ float xs[kMaxIn], a1[kMaxH], a2[kMaxH];
    const int64_t s = blockIdx.x;
    if (s >= B) return;
    const int h = threadIdx.x;
    if (h < n_in) xs[h] = x[s * n_in + h];
    __syncthreads();
    float z1 = p[o.b1 + h];
    for (int i = 0; i < n_in; ++i) z1 += p[o.W1 + (int64_t)h * n_in + i] * xs[i];
    a1[h] = z1 > 0.f ? z1 : 0.f;
    __syncthreads();
    float z2 = p[o.b2 + h];
    for (int i = 0; i < H; ++i) z2 += p[o.W2 + (int64_t)h * H + i] * a1[i];
    a2[h] = z2 > 0.f ? z2 : 0.f;
    if (act) {
        act[s * 2 * H + h] = z1;
        act[s * 2 * H + H + h] = z2;
    }
    __syncthreads();
    if (h < n_out) {
        float z3 = p[o.b3 + h];
        for (int i = 0; i < H; ++i) z3 += p[o.W3 + (int64_t)h * H + i] * a2[i];
        y[s * n_out + h] = z3;
    }
}

// one CTA per sample: this sample's gradient row and squared error
__global__ void mlp_backward_kernel(const float* __restrict__ p, int n_in, int H, int n_out, Off o,
                                    const float* __restrict__ x, const float* __restrict__ t, int64_t B,
                                    const float* __restrict__ y, const float* __restrict__ act,
                                    float* __restrict__ rows, float* __restrict__ loss_rows) {
    __shared__ float xs[kMaxIn], a1[kMaxH], a2[kMaxH], d2[kMaxH], d3[kMaxOut];
    const int64_t s = blockIdx.x;
    if (s >= B) return;
    const int h = threadIdx.x;
    const float inv = 1.0f / (float)(B * n_out);
    float* row = rows + s * o.n;
    if (h < n_in) xs[h] = x[s * n_in + h];
    const float z1 = act[s * 2 * H + h], z2 = act[s * 2 * H + H + h];
    a1[h] = z1 > 0.f ? z1 : 0.f;
    a2[h] = z2 > 0.f ? z2 : 0.f;
    if (h < n_out) {
        float e = y[s * n_out + h] - t[s * n_out + h];
        d3[h] = 2.f * e * inv;
        if (h == 0) {
            float se = 0.f;
            for (int q = 0; q < n_out; ++q) {
                float eq = y[s * n_out + q] - t[s * n_out + q];
                se += eq * eq;
            }
            loss_rows[s] = se * inv;
        }
    }
    __syncthreads();
    // layer 3
    for (int q = 0; q < n_out; ++q) row[o.W3 + (int64_t)q * H + h] = d3[q] * a2[h];
    if (h < n_out) row[o.b3 + h] = d3[h];
    float g2 = 0.f;
    for (int q = 0; q < n_out; ++q) g2 += p[o.W3 + (int64_t)q * H + h] * d3[q];
    d2[h] = z2 > 0.f ? g2 : 0.f;
    __syncthreads();
    // layer 2: dW2[h][i] = d2[h] a1[i]
    for (int i = 0; i < H; ++i) row[o.W2 + (int64_t)h * H + i] = d2[h] * a1[i];
    row[o.b2 + h] = d2[h];
    float g1 = 0.f;
    for (int k = 0; k < H; ++k) g1 += p[o.W2 + (int64_t)k * H + h] * d2[k];
    const float d1 = z1 > 0.f ? g1 : 0.f;
    for (int i = 0; i < n_in; ++i) row[o.W1 + (int64_t)h * n_in + i] = d1 * xs[i];
    row[o.b1 + h] = d1;
}

// grad[j] = sum_s rows[s][j] in sample order (deterministic)
__global__ void column_sum_kernel(const float* __restrict__ rows, int64_t B, int64_t n, float* __restrict__ out) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    float acc = 0.f;
    for (int64_t s = 0; s < B; ++s) acc += rows[s * n + j];
    out[j] = acc;
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    float gj = g[j];
    float mj = b1 * m[j] + (1.f - b1) * gj;
    float vj = b2 * v[j] + (1.f - b2) * gj * gj;
    m[j] = mj;
    v[j] = vj;
    p[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

hp_status ensure_cap(hp_mlp m, int64_t B) {
    if (B <= m->cap) return HP_OK;
    cudaFree(m->d_rows);
    cudaFree(m->d_act);
    cudaFree(m->d_y);
    cudaFree(m->d_loss_rows);
    m->d_rows = m->d_act = m->d_y = m->d_loss_rows = nullptr;
    cudaError_t e = cudaMalloc(&m->d_rows, sizeof(float) * B * m->n_params);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_act, sizeof(float) * B * 2 * m->H);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_y, sizeof(float) * B * m->n_out);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_loss_rows, sizeof(float) * B);
    if (e != cudaSuccess) return cuda_fail(e, "hp_mlp workspace");
    m->cap = B;
    return HP_OK;
}

hp_status grad_impl(hp_mlp m, const float* x, const float* t, int64_t B, float* grad, float* loss, cudaStream_t s) {
    hp_status st = ensure_cap(m, B);
    if (st) return st;
    Off o = offsets(m->n_in, m->H, m->n_out);
    mlp_forward_kernel<<<(unsigned)B, m->H, 0, s>>>(m->d_params, m->n_in, m->H, m->n_out, o, x, B, m->d_y, m->d_act);
    mlp_backward_kernel<<<(unsigned)B, m->H, 0, s>>>(m->d_params, m->n_in, m->H, m->n_out, o, x, t, B, m->d_y,
                                                     m->d_act, m->d_rows, m->d_loss_rows);
    column_sum_kernel<<<(unsigned)((o.n + 255) / 256), 256, 0, s>>>(m->d_rows, B, o.n, grad);
    if (loss) column_sum_kernel<<<1, 32, 0, s>>>(m->d_loss_rows, B, 1, loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_mlp kernels");
}

}  // namespace
}  // namespace hp

using namespace hp;

extern "C" {

hp_status hp_mlp_create(int n_in, int n_hidden, int n_out, uint64_t seed, int device, hp_mlp* out) {
    if (!out || n_in < 1 || n_in > kMaxIn || n_hidden < 32 || n_hidden > kMaxH || n_hidden % 32 || n_out < 1 ||
        n_out > kMaxOut) {
        set_error("hp_mlp_create: sizes out of range (n_in 1..16, hidden 32..256 multiple of 32, n_out 1..8)");
        return HP_ERR_ARG;
    }
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("hp_mlp_create: no such CUDA device");
        return HP_ERR_ARG;
    }
    cudaSetDevice(device);
    auto m = new hp_mlp_s();
    m->device = device;
    m->n_in = n_in;
    m->H = n_hidden;
    m->n_out = n_out;
    Off o = offsets(n_in, n_hidden, n_out);
    m->n_params = o.n;
    // He-uniform weights from a counter-based generator, zero biases
    std::vector<float> p(o.n, 0.f);
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        float a = std::sqrt(6.0f / (float)fan_in);
        for (int64_t j = 0; j < count; ++j) {
            double u = (double)(mix64(seed * 0x100000000ull + (uint64_t)(off + j)) >> 11) * (1.0 / 9007199254740992.0);
            p[off + j] = (float)((2.0 * u - 1.0) * a);
        }
    };
    fill(o.W1, (int64_t)n_hidden * n_in, n_in);
    fill(o.W2, (int64_t)n_hidden * n_hidden, n_hidden);
    fill(o.W3, (int64_t)n_out * n_hidden, n_hidden);
    cudaError_t e = cudaMalloc(&m->d_params, sizeof(float) * o.n);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m, sizeof(float) * o.n);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_v, sizeof(float) * o.n);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_grad, sizeof(float) * o.n);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_params, p.data(), sizeof(float) * o.n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, sizeof(float) * o.n);
    if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, sizeof(float) * o.n);
    if (e != cudaSuccess) {
        hp_status st = cuda_fail(e, "hp_mlp_create");
        hp_mlp_destroy(m);
        return st;
    }
    *out = m;
    return HP_OK;
}

hp_status hp_mlp_params(hp_mlp m, float* host, int64_t n, int set) {
    if (!m || !host || n != m->n_params) { set_error("hp_mlp_params: bad argument"); return HP_ERR_ARG; }
    cudaSetDevice(m->device);
    cudaError_t e = set ? cudaMemcpy(m->d_params, host, sizeof(float) * n, cudaMemcpyHostToDevice)
                        : cudaMemcpy(host, m->d_params, sizeof(float) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "hp_mlp_params");
    if (set) {
        cudaMemset(m->d_m, 0, sizeof(float) * n);
        cudaMemset(m->d_v, 0, sizeof(float) * n);
        m->step = 0;
    }
    return HP_OK;
}

hp_status hp_mlp_info(hp_mlp m, int* n_in, int* n_hidden, int* n_out, int64_t* n_params) {
    if (!m) { set_error("hp_mlp_info: null"); return HP_ERR_ARG; }
    if (n_in) *n_in = m->n_in;
    if (n_hidden) *n_hidden = m->H;
    if (n_out) *n_out = m->n_out;
    if (n_params) *n_params = m->n_params;
    return HP_OK;
}

hp_status hp_mlp_forward(hp_mlp m, const float* x, int64_t batch, float* y, void* stream) {
    if (!m || !x || !y || batch < 1 || batch > 65535) { set_error("hp_mlp_forward: bad argument"); return HP_ERR_ARG; }
    cudaSetDevice(m->device);
    Off o = offsets(m->n_in, m->H, m->n_out);
    mlp_forward_kernel<<<(unsigned)batch, m->H, 0, (cudaStream_t)stream>>>(m->d_params, m->n_in, m->H, m->n_out, o,
                                                                           x, batch, y, nullptr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_mlp_forward");
}

hp_status hp_mlp_grad(hp_mlp m, const float* x, const float* t, int64_t batch, float* grad, float* loss,
                      void* stream) {
    if (!m || !x || !t || !grad || batch < 1 || batch > 65535) { set_error("hp_mlp_grad: bad argument"); return HP_ERR_ARG; }
    cudaSetDevice(m->device);
    return grad_impl(m, x, t, batch, grad, loss, (cudaStream_t)stream);
}

hp_status hp_mlp_adam_step(hp_mlp m, const float* x, const float* t, int64_t batch, float lr, float* loss,
                           void* stream) {
    if (!m || !x || !t || batch < 1 || batch > 65535 || !(lr > 0.f)) { set_error("hp_mlp_adam_step: bad argument"); return HP_ERR_ARG; }
    cudaSetDevice(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    hp_status st = grad_impl(m, x, t, batch, m->d_grad, loss, s);
    if (st) return st;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    adam_kernel<<<(unsigned)((m->n_params + 255) / 256), 256, 0, s>>>(m->d_params, m->d_m, m->d_v, m->d_grad,
                                                                    m->n_params, lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_mlp_adam_step");
}

void hp_mlp_destroy(hp_mlp m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaFree(m->d_params);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_grad);
    cudaFree(m->d_rows);
    cudaFree(m->d_act);
    cudaFree(m->d_y);
    cudaFree(m->d_loss_rows);
    delete m;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradient entry point that allocates nothing (see hp_mlp_grad_noalloc in
// include/hp.h).  Its scratch -- per-sample gradient rows, activations,
// outputs and per-sample losses -- lives in this fixed-size device array,
// which every GPU that loads the library holds until the process exits.
static constexpr int64_t kNoAllocScratchFloats = int64_t(1) << 20;   // 4 MiB per device
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

namespace hp {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace
}  // namespace hp

extern "C" hp_status hp_mlp_grad_noalloc(const float* params, int n_in, int n_hidden, int n_out, const float* x,
                                         const float* t, int64_t batch, float* grad, float* loss, void* stream) {
    if (!params || !x || !t || !grad || batch < 1 || batch > 65535 || n_in < 1 || n_in > kMaxIn ||
        n_hidden < 32 || n_hidden > kMaxH || n_hidden % 32 || n_out < 1 || n_out > kMaxOut) {
        set_error("hp_mlp_grad_noalloc: bad argument");
        return HP_ERR_ARG;
    }
    Off o = offsets(n_in, n_hidden, n_out);
    const int64_t need = batch * (o.n + 2 * (int64_t)n_hidden + n_out + 1);
    if (need > kNoAllocScratchFloats) {
        set_error("hp_mlp_grad_noalloc: batch * (n_params + 2 n_hidden + n_out + 1) = " + std::to_string(need) +
                  " floats exceeds the fixed scratch of " + std::to_string(kNoAllocScratchFloats) +
                  " floats; use a smaller batch or hp_mlp_grad");
        return HP_ERR_ARG;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "hp_mlp_grad_noalloc");
    if (dev < 0 || dev >= kMaxDevices) { set_error("hp_mlp_grad_noalloc: device index out of range"); return HP_ERR_ARG; }
    float* base = nullptr;
    {
        // set-up on the first call on this device (the device is current):
        // the host-side name of the array is not a device address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "hp_mlp_grad_noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[dev] = static_cast<float*>(p);
        }
        base = g_noalloc_ptr[dev];
    }
    // every scratch entry read below is written first in the same call
    // (rows by the backward kernel, activations and outputs by the forward one),
    // so nothing needs clearing between calls
    float* rows = base;
    float* act = rows + batch * o.n;
    float* y = act + batch * 2 * (int64_t)n_hidden;
    float* loss_rows = y + batch * n_out;
    cudaStream_t s = (cudaStream_t)stream;
    mlp_forward_kernel<<<(unsigned)batch, n_hidden, 0, s>>>(params, n_in, n_hidden, n_out, o, x, batch, y, act);
    mlp_backward_kernel<<<(unsigned)batch, n_hidden, 0, s>>>(params, n_in, n_hidden, n_out, o, x, t, batch, y, act,
                                                            rows, loss_rows);
    column_sum_kernel<<<(unsigned)((o.n + 255) / 256), 256, 0, s>>>(rows, batch, o.n, grad);
    if (loss) column_sum_kernel<<<1, 32, 0, s>>>(loss_rows, batch, 1, loss);
    e = cudaGetLastError();
    return e == cudaSuccess ? HP_OK : cuda_fail(e, "hp_mlp_grad_noalloc");
}
