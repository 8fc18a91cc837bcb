// FP32 FMA throughput of the device (sm_103a): the denominator of the FFT
// path's roofline, measured rather than taken from the unit counts and the
// nominal clock.
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA latency
// with the 32 resident warps per SM of this launch: 2 CTAs of 512 threads per
// SM), ITER rounds of 8 FMAs each; the launch is timed with CUDA events. The
// chains' values feed one conditional store so that nothing is removed.

#include <cuda_runtime.h>

#include "../../include/fwr.h"
#include "fwr_plan.h"

namespace {

constexpr int PEAK_THREADS = 512, PEAK_CHAINS = 8;

__device__ float g_peak_sink;

__global__ void __launch_bounds__(PEAK_THREADS, 2) fma_peak_kernel(int iters, float a, float b) {
    float x[PEAK_CHAINS];
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = float(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
    if (s < -1e30f) g_peak_sink = s;  // never true for a = 1, b = 0 (the values stay >= 0)
}

}  // namespace

extern "C" fwr_status fwr_fp32_fma_peak(double* tflops, double* ms, void* stream) {
    if (!tflops) return FWR_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_fp32_fma_peak");
    const int blocks = 2 * sms, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fwr::cuda_fail(e, "fwr_fp32_fma_peak events");
    }
    // a = 1, b = 0 keep the values finite and unchanged (the compiler cannot
    // know them); the sink is never written
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        fma_peak_kernel<<<blocks, PEAK_THREADS, 0, s>>>(iters, 1.0f, 0.0f);
        cudaEventRecord(e1, s);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < best) best = t;  // the first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_fp32_fma_peak");
    const double flop = 2.0 * double(blocks) * PEAK_THREADS * double(iters) * 16.0 * PEAK_CHAINS;
    *tflops = flop / (double(best) * 1e-3) / 1e12;
    if (ms) *ms = best;
    return FWR_OK;
}
