// Ragged batches (sm_103a): one persistent launch over frames of several
// plans, 128^2 and 256^2 grids mixed. Each CTA walks its own list of frames
// (built on the host by a longest-processing-time-first schedule, grouped by
// plan); when the plan changes it reloads that plan's tables into shared
// memory, then runs the frame through the main kernel's per-frame path
// (128^2) or the slab path (256^2, with this CTA's scratch area). Both paths
// run on 512 threads.

#include <cuda_runtime.h>
#include <stdint.h>

#include "fwr_internal.h"

namespace fwr {

#include "fwr_fft.cuh"
#include "fwr_fused.cuh"
#include "fwr_slab.cuh"

static_assert(4 * 128 == SNT, "both paths of the ragged kernel run on 512 threads");

template <int GROUPS>
__global__ void __launch_bounds__(512, 1)
ragged_kernel(RaggedParams rp) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the 128^2 frames' LSQ coefficients live in tensor memory, as in the main
    // kernel (recomputed at each change of plan; one CTA per SM)
    __shared__ uint32_t s_tmem;
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         uint32_t(__cvta_generic_to_shared(&s_tmem))),
                     "r"(FUSED_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int b = blockIdx.x;
    const int i0 = rp.cta_off[b], i1 = rp.cta_off[b + 1];
    float2* G = rp.scratch ? rp.scratch + size_t(b) * SN * SN : nullptr;
    FusedCtx<float, 128> fc;
    SlabCtx sc;
    int cur = -1;
    for (int i = i0; i < i1; ++i) {
        const int f = rp.order[i];
        const int pl = rp.frame_plan[f];
        if (pl < 0 || pl >= rp.n_plans) {
            // a frame table rewritten with an invalid index: skip the frame
            if (threadIdx.x == 0) atomicOr(rp.plans[0].status, STATUS_BADINDEX);
            continue;
        }
        const RaggedPlan P = rp.plans[pl];
        if (pl != cur) {
            if (P.N == 128) fused_setup<float, 128, true>(fc, smem, P.tab, P.mask, P.n, P.off, P.periodic, false, tmem);
            else slab_setup<256>(sc, smem, P.tab, P.mask, P.n, P.off, P.periodic);
            cur = pl;
        }
        bool ok;
        if (P.N == 128)
            ok = fused_frame<float, 128, true>(fc, rp.slopes[f], nullptr, nullptr, rp.phase[f], nullptr, rp.iters);
        else ok = slab_frame<256, GROUPS>(sc, P.tab, rp.slopes[f], nullptr, rp.phase[f], rp.iters, G);
        if (!ok) atomicOr(P.status, STATUS_NONFINITE);
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(FUSED_TMEM_COLS)
                     : "memory");
    }
}

size_t ragged_smem_bytes(int N, int n) {
    if (N == 128) return Layout<float, 128>::bytes(n);
    if (N == 256) return slab_layout_bytes(n);
    return 0;
}

cudaError_t ragged_prepare(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(ragged_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(ragged_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

cudaError_t launch_ragged(const RaggedParams& p, int grid, size_t smem, cudaStream_t s) {
    if (p.shape == 1) ragged_kernel<1><<<grid, 512, smem, s>>>(p);
    else ragged_kernel<2><<<grid, 512, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fwr
