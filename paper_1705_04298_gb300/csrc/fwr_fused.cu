// Main fused persistent Gerchberg kernel for sm_103a: kernels and launchers.
// The device code (layout, passes, per-frame path) is in fwr_fused.cuh.

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "fwr_internal.h"

namespace fwr {

#include "fwr_fft.cuh"
#include "fwr_fused.cuh"

// HUD: the Hudgin extension as the initial extension (a separate
// instantiation, so that the default one carries none of its code)
template <typename T, int N, bool HUD>
__global__ void __launch_bounds__(4 * N)
fused_kernel(Params<T> p) {
    // FP32 on 128^2 (one CTA per SM): the LSQ coefficients live in tensor memory
    constexpr bool TMC = sizeof(T) == 4 && N == 128;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_bad;
    __shared__ uint32_t s_tmem;
    if (threadIdx.x == 0) s_bad = 0;
    if constexpr (TMC) {
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
    }
    FusedCtx<T, N> c;
    fused_setup<T, N, TMC>(c, smem, p.tab, p.mask, p.n, p.off, p.periodic, p.wf_smem != 0, TMC ? s_tmem : 0u);
    // launched as a dependent (Params::pdl): the set-up above used only the
    // plan's tables; the frames' inputs are read after the producer completes
    pdl_wait();
    const int nn = p.n * p.n;
    bool finite = true;
    for (int f = blockIdx.x; f < p.F; f += gridDim.x) {
        // the CTA's next frame's slopes into L2 while this one is worked
        if (f + int(gridDim.x) < p.F) prefetch_l2(p.slopes + size_t(f + gridDim.x) * 2 * nn, 2 * nn * sizeof(T));
        finite &= fused_frame<T, N, TMC>(c, p.slopes + size_t(f) * 2 * nn,
                                    p.ext_init ? p.ext_init + size_t(f) * 2 * N * N : nullptr,
                                    p.ext_init_h ? p.ext_init_h + size_t(f) * 2 * N * N : nullptr,
                                    p.phase ? p.phase + size_t(f) * N * N : nullptr,
                                    p.ext_out ? p.ext_out + size_t(f) * 2 * N * N : nullptr, p.iters,
                                    HUD ? p.hud : nullptr);
        __syncthreads();
    }
    if (!finite) atomicOr(&s_bad, 1);
    if constexpr (TMC) asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(p.status, STATUS_NONFINITE);
    if constexpr (TMC) {
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s_tmem),
                         "r"(FUSED_TMEM_COLS)
                         : "memory");
        }
    }
}

// Standalone batched 2-D FFT through the same three passes (test entry):
// natural-order input and output.
template <int N, bool INV>
__global__ void __launch_bounds__(4 * N)
fused_fft2_kernel(const float2* in, float2* out, int F, const float2* twg) {
    typedef Layout<float, N> L;
    constexpr int R = N / 4, NT = 4 * N, S = L::S;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* Z = reinterpret_cast<float2*>(smem + L::z);
    float2* tw = reinterpret_cast<float2*>(smem + L::tw);
    float2* tw2 = reinterpret_cast<float2*>(smem + L::tw2);
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += NT) tw[i] = twg[i];
    __syncthreads();
    for (int i = tid; i < 3 * R; i += NT) tw2[i] = tw[(i % R) * (1 + i / R)];
    int r, n2;
    row_role<N>(tid, r, n2);
    float2* const rowp = Z + r * S + n2;
    float2* const colp = Z + R * (tid / N) * S + tid % N;
    __syncthreads();
    for (int f = blockIdx.x; f < F; f += gridDim.x) {
        const float2* src = in + size_t(f) * N * N;
        float2* dst = out + size_t(f) * N * N;
        float2 x[R];
        if (!INV) {
            for (int c = tid; c < N * N; c += NT) Z[(c / N) * S + c % N] = src[c];
            __syncthreads();
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) x[n1] = rowp[4 * n1];
            dft_reg<R, false>(x);
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) rowp[4 * k1] = x[k1];
            __syncthreads();
            pass2<false, N>(Z, tw, tw2);
            __syncthreads();
#pragma unroll
            for (int m2 = 0; m2 < R; ++m2) x[m2] = colp[S * m2];
            dft_reg<R, false>(x);
#pragma unroll
            for (int q2 = 0; q2 < R; ++q2) colp[S * q2] = x[q2];
            __syncthreads();
            for (int c = tid; c < N * N; c += NT) {
                const int ky = c / N, kx = c % N;
                dst[c] = Z[(R * (ky & 3) + (ky >> 2)) * S + 4 * (kx % R) + kx / R];
            }
        } else {
            for (int c = tid; c < N * N; c += NT) {
                const int ky = c / N, kx = c % N;
                Z[(R * (ky & 3) + (ky >> 2)) * S + 4 * (kx % R) + kx / R] = src[c];
            }
            __syncthreads();
#pragma unroll
            for (int q2 = 0; q2 < R; ++q2) x[q2] = colp[S * q2];
            dft_reg<R, true>(x);
#pragma unroll
            for (int m2 = 0; m2 < R; ++m2) colp[S * m2] = x[m2];
            __syncthreads();
            pass2<true, N>(Z, tw, tw2);
            __syncthreads();
#pragma unroll
            for (int k1 = 0; k1 < R; ++k1) x[k1] = rowp[4 * k1];
            dft_reg<R, true>(x);
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) rowp[4 * n1] = x[n1];
            __syncthreads();
            for (int c = tid; c < N * N; c += NT) dst[c] = Z[(c / N) * S + c % N];
        }
        __syncthreads();
    }
}

namespace {

template <int N>
cudaError_t launch_fft2_n(const float2* in, float2* out, int F, int inverse, const float2* tw, cudaStream_t s) {
    const size_t smem = Layout<float, N>::a;
    auto kern = inverse ? fused_fft2_kernel<N, true> : fused_fft2_kernel<N, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = F < sms ? F : sms;
    kern<<<grid, 4 * N, smem, s>>>(in, out, F, tw);
    return cudaGetLastError();
}

// Per (device, kernel, shared-memory size): the SM count and the resident CTAs
// per SM (these queries were on every call's path). The kernel's
// shared-memory limit is a property of the function, so it is tracked per
// (device, kernel) and only ever raised: a smaller launch never lowers it
// below what a cached larger launch needs.
struct KernelLimit {
    int dev;
    const void* kern;
    size_t smem_max;
};
struct LaunchShape {
    int dev;
    const void* kern;
    size_t smem;
    int sms, per_sm;
};

cudaError_t launch_shape(const void* kern, size_t smem, int threads, int* sms, int* per_sm) {
    static std::mutex mu;
    static std::vector<KernelLimit> limits;
    static std::vector<LaunchShape> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    KernelLimit* lim = nullptr;
    for (KernelLimit& l : limits)
        if (l.dev == dev && l.kern == kern) lim = &l;
    if (!lim || lim->smem_max < smem) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem))) != cudaSuccess)
            return e;
        if (lim) {
            lim->smem_max = smem;
        } else {
            limits.push_back(KernelLimit{dev, kern, smem});
        }
    }
    for (const LaunchShape& c : cache)
        if (c.dev == dev && c.kern == kern && c.smem == smem) {
            *sms = c.sms;
            *per_sm = c.per_sm;
            return cudaSuccess;
        }
    LaunchShape c{dev, kern, smem, 0, 0};
    if ((e = cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.per_sm, kern, threads, smem)) != cudaSuccess) return e;
    cache.push_back(c);
    *sms = c.sms;
    *per_sm = c.per_sm;
    return cudaSuccess;
}

template <typename T, int N>
cudaError_t launch_n(const Params<T>& p0, cudaStream_t s) {
    // keep the final-filter table in shared memory when it still fits
    Params<T> p = p0;
    p.wf_smem = p.shape != 2 && Layout<T, N>::bytes_wf(p.n) <= size_t(227) * 1024 ? 1 : 0;
    const size_t smem = p.wf_smem ? Layout<T, N>::bytes_wf(p.n) : Layout<T, N>::bytes(p.n);
    auto kern = p.hud ? fused_kernel<T, N, true> : fused_kernel<T, N, false>;
    int sms = 0, per_sm = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void*>(kern), smem, 4 * N, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * per_sm;
    if (p.ctas > 0 && p.ctas < grid) grid = p.ctas;
    if (grid > p.F) grid = p.F;
    if (!p.pdl) {
        kern<<<grid, 4 * N, smem, s>>>(p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(4 * N);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

size_t fused_bytes(int N, int elem_bytes, int n) {
    const bool d = elem_bytes == 8;
    switch (N) {
        case 16: return d ? Layout<double, 16>::bytes(n) : Layout<float, 16>::bytes(n);
        case 32: return d ? Layout<double, 32>::bytes(n) : Layout<float, 32>::bytes(n);
        case 64: return d ? Layout<double, 64>::bytes(n) : Layout<float, 64>::bytes(n);
        case 128: return d ? Layout<double, 128>::bytes(n) : Layout<float, 128>::bytes(n);
        default: return 0;
    }
}

}  // namespace

cudaError_t launch_fft2_f32(int N, const float2* in, float2* out, int F, int inverse, const float2* tw,
                            cudaStream_t s) {
    switch (N) {
        case 16: return launch_fft2_n<16>(in, out, F, inverse, tw, s);
        case 32: return launch_fft2_n<32>(in, out, F, inverse, tw, s);
        case 64: return launch_fft2_n<64>(in, out, F, inverse, tw, s);
        case 128: return launch_fft2_n<128>(in, out, F, inverse, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

bool fused_supported(int N, int elem_bytes, int n) {
    const size_t b = fused_bytes(N, elem_bytes, n);
    return b != 0 && b <= size_t(227) * 1024;
}

cudaError_t launch_fused_f32(int N, const Params<float>& p, cudaStream_t s) {
    switch (N) {
        case 16: return launch_n<float, 16>(p, s);
        case 32: return launch_n<float, 32>(p, s);
        case 64: return launch_n<float, 64>(p, s);
        case 128: return launch_n<float, 128>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_f64(int N, const Params<double>& p, cudaStream_t s) {
    switch (N) {
        case 16: return launch_n<double, 16>(p, s);
        case 32: return launch_n<double, 32>(p, s);
        case 64: return launch_n<double, 64>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fwr
