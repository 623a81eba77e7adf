// Persistent work-list form of the FP64 sum-factorised operators: one launch
// covers every block of an operator (all shapes, orders up to
// kWorklistMaxP, affine and curved), for p-adaptive meshes whose many blocks
// are each too small to fill the GPU.  The host cuts each block's element
// groups into work items and orders them by decreasing cost; every CTA takes
// the next item from a device counter, stages that block's reference tables
// (one bulk copy on a barrier it reuses) and runs the block's body over the
// item's groups.  Dynamic shared memory is the largest of the bodies present.
#include <algorithm>

#include "hp_sf.cuh"

namespace hp {
namespace {

// each body a function of its own (its own register allocation and code,
// called through the ABI), not one inlined union of all of them
template <int S, int PP, bool AFF>
__device__ __noinline__ bool wl_body(const SFDesc& a, unsigned char* smem, int64_t g0, int64_t g1, uint32_t* phase) {
    uint32_t ph = *phase;
    const bool ok = sf_groups<S, PP, double, AFF, 0>(a, smem, g0, 1, g1, ph);
    *phase = ph;
    return ok;
}

__global__ void __launch_bounds__(256, 3) sf_worklist_kernel(const SFDesc* __restrict__ desc,
                                                          const WorkItem* __restrict__ items, int n_items,
                                                          int* __restrict__ next, unsigned int* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    if (threadIdx.x == 0) mbar_init(reinterpret_cast<uint64_t*>(smem), 1);
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= n_items) return;
        const WorkItem w = items[it];
        const SFDesc& a = desc[w.block];
        bool ok;
        switch (w.key) {
#define HP_WL(S, PP)                                                                                     \
    case (S) * 32 + (PP) * 2:                                                                            \
        ok = wl_body<S, PP, false>(a, smem, w.g0, w.g1, &phase);                                         \
        break;                                                                                           \
    case (S) * 32 + (PP) * 2 + 1:                                                                        \
        ok = wl_body<S, PP, true>(a, smem, w.g0, w.g1, &phase);                                          \
        break;
#define HP_WL_SHAPE(S) HP_WL(S, 1) HP_WL(S, 2) HP_WL(S, 3) HP_WL(S, 4) HP_WL(S, 5) HP_WL(S, 6) HP_WL(S, 7) HP_WL(S, 8)
            HP_WL_SHAPE(0) HP_WL_SHAPE(1) HP_WL_SHAPE(2) HP_WL_SHAPE(3)
#undef HP_WL_SHAPE
#undef HP_WL
            default:
                if (threadIdx.x == 0) atomicOr(err, DERR_BOUNDS);
                ok = false;
        }
        if (!ok) return;
    }
}

template <int S>
int smem_of(int P) {
    switch (P) {
        case 1: return sf_smem_bytes<S, 1, double, 0>();
        case 2: return sf_smem_bytes<S, 2, double, 0>();
        case 3: return sf_smem_bytes<S, 3, double, 0>();
        case 4: return sf_smem_bytes<S, 4, double, 0>();
        case 5: return sf_smem_bytes<S, 5, double, 0>();
        case 6: return sf_smem_bytes<S, 6, double, 0>();
        case 7: return sf_smem_bytes<S, 7, double, 0>();
        case 8: return sf_smem_bytes<S, 8, double, 0>();
        default: return -1;
    }
}

}  // namespace

int sf_worklist_epb(int P) { return sf_epb<double>(P, 0); }

int sf_worklist_smem(int shape, int P) {
    switch (shape) {
        case HP_HEX: return smem_of<HP_HEX>(P);
        case HP_PRISM: return smem_of<HP_PRISM>(P);
        case HP_PYR: return smem_of<HP_PYR>(P);
        case HP_TET: return smem_of<HP_TET>(P);
        default: return -1;
    }
}

cudaError_t sf_worklist_grid(int smem, int* grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sf_worklist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sf_worklist_kernel, 256, smem);
    if (e != cudaSuccess) return e;
    *grid = sms * std::max(per, 1);
    return cudaSuccess;
}

cudaError_t sf_worklist_launch(const SFDesc* desc, const WorkItem* items, int n_items, int* next, int smem, int grid,
                               unsigned int* err, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    sf_worklist_kernel<<<std::min(grid, n_items), 256, smem, s>>>(desc, items, n_items, next, err);
    return cudaGetLastError();
}

}  // namespace hp
