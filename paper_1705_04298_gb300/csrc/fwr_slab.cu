// Gerchberg kernel for 256^2 and 512^2 grids (sm_103a): kernels and launchers. The
// slab-streamed device code is in fwr_slab.cuh.

#include <cuda_runtime.h>
#include <stdint.h>

#include "fwr_internal.h"

namespace fwr {

#include "fwr_fft.cuh"
#include "fwr_slab.cuh"

template <int N, int GROUPS>
__global__ void __launch_bounds__(SNT, 1)
slab_kernel(Params<float> p, float2* scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    SlabCtx c;
    slab_setup<N>(c, smem, p.tab, p.mask, p.n, p.off, p.periodic);
    float2* G = scratch + size_t(blockIdx.x) * N * N;
    const int nn = p.n * p.n;
    bool finite = true;
    for (int f = blockIdx.x; f < p.F; f += gridDim.x) {
        finite &= slab_frame<N, GROUPS>(c, p.tab, p.slopes + size_t(f) * 2 * nn,
                                        p.ext_init ? p.ext_init + size_t(f) * 2 * N * N : nullptr,
                                        p.phase + size_t(f) * N * N, p.iters, G, p.hud);
        __syncthreads();
    }
    if (!finite) atomicOr(&s_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(p.status, STATUS_NONFINITE);
}

namespace {

typedef void (*SlabKernel)(Params<float>, float2*);

// the kernel of grid N and a shape (1 or 2 warp groups; 0 is 2) with its
// shared-memory limit set for n lenslets
cudaError_t slab_kernel_for(int N, int shape, int n, SlabKernel* k) {
    if (N == 512) *k = shape == 1 ? slab_kernel<512, 1> : slab_kernel<512, 2>;
    else *k = shape == 1 ? slab_kernel<256, 1> : slab_kernel<256, 2>;
    return cudaFuncSetAttribute(*k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(slab_layout_bytes_n(N, n)));
}

}  // namespace

size_t slab_smem_bytes(int N, int n) { return slab_layout_bytes_n(N, n); }

size_t slab_scratch_elems_per_cta(int N) { return size_t(N) * N; }

int slab_max_ctas() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

cudaError_t launch_slab(int N, const Params<float>& p, float2* scratch, int max_ctas, cudaStream_t s) {
    if (N != 256 && N != 512) return cudaErrorInvalidValue;
    SlabKernel kern = nullptr;
    cudaError_t e = slab_kernel_for(N, p.shape, p.n, &kern);
    if (e != cudaSuccess) return e;
    int grid = max_ctas;
    if (p.ctas > 0 && p.ctas < grid) grid = p.ctas;
    if (grid > p.F) grid = p.F;
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (p.l2_bytes == 0) {
        kern<<<grid, SNT, slab_smem_bytes(N, p.n), s>>>(p, scratch);
        return cudaGetLastError();
    }
    // the scratch's lines persist in L2 (the context's set-aside holds them)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SNT);
    cfg.dynamicSmemBytes = slab_smem_bytes(N, p.n);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow.base_ptr = scratch;
    attr[0].val.accessPolicyWindow.num_bytes = p.l2_bytes;
    attr[0].val.accessPolicyWindow.hitRatio = p.l2_hit;
    attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p, scratch);
}

// ---------------------------------------------------------------------------
// Variant without any allocation: the scratch is this file-scope array, sized
// for STATIC_SLAB_GRIDS concurrent frames (8 MB). It exists on every GPU that
// loads the library, for the life of the process.
// ---------------------------------------------------------------------------
static __device__ __align__(256) float2 g_static_slab_scratch[STATIC_SLAB_GRIDS * 256 * 256];

// Host code cannot use the array's name as a device address: look the address
// up with the device current (this also loads the module on that device, so a
// later call does no loading) and set the kernel's shared-memory limit.
cudaError_t static_slab_prepare(int n, float2** addr) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_slab_scratch);
    if (e != cudaSuccess) return e;
    SlabKernel kern = nullptr;
    if ((e = slab_kernel_for(256, 1, n, &kern)) != cudaSuccess || (e = slab_kernel_for(256, 2, n, &kern)) != cudaSuccess)
        return e;
    *addr = static_cast<float2*>(ptr);
    return cudaSuccess;
}

cudaError_t launch_slab_static(const Params<float>& p, float2* scratch, int ctas, cudaStream_t s) {
    if (ctas < 1 || ctas > STATIC_SLAB_GRIDS || !scratch) return cudaErrorInvalidValue;
    const int grid = ctas < p.F ? ctas : p.F;
    auto kern = p.shape == 1 ? slab_kernel<256, 1> : slab_kernel<256, 2>;
    kern<<<grid, SNT, slab_smem_bytes(256, p.n), s>>>(p, scratch);
    return cudaGetLastError();
}

}  // namespace fwr
