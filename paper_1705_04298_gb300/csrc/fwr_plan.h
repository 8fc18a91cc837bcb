// Plan object shared by the C-ABI translation units (fwr_api.cpp,
// fwr_batch.cpp). Not installed.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fwr.h"
#include "fwr_internal.h"

namespace fwr {

// Device copies of one precision's tables.
template <typename T> struct DevTables {
    typedef typename cvec<T>::type V;
    V* tw = nullptr;
    V* A = nullptr;
    V* Tt = nullptr;
    T* pt = nullptr;
    T* iota = nullptr;
    T* wfin = nullptr;
};

// Record a CUDA error as the thread's last error; returns FWR_ERR_CUDA.
fwr_status cuda_fail(cudaError_t e, const char* where);
// Record a message as the thread's last error.
void set_last_error(const char* msg);
// The persisting-L2 set-aside of a device before the library first raised it
// (FWR_OPT_L2_PERSIST): note records it once; before returns false if never raised.
void l2_setaside_note(int device, size_t before);
bool l2_setaside_before(int device, size_t* before);

}  // namespace fwr

struct fwr_plan;

namespace fwr {
// The FP32 path of plan p through the fused kernel with a BF16 warm start
// ([F][2][N][N] bit patterns, 8-byte aligned); cudaErrorNotSupported when the
// plan does not take the fused path (N = 256, the DFT-GEMM transform, grids
// the fused kernel does not cover). pdl: launched as a programmatic
// dependent of the kernel before it on s, which must be the producer of
// ext_init_h (its set-up then overlaps that kernel's tail).
cudaError_t launch_warm_bf16(fwr_plan* p, const float* slopes, const uint16_t* ext_init_h, int n_frames, int iters,
                             float* phase, cudaStream_t s, bool pdl = false);
}  // namespace fwr

struct fwr_plan {
    int n = 0, N = 0, off = 0, filter = 0, periodic = FWR_PERIODIC_BEFORE_EACH_FFT, nvalid = 0;
    int transform = FWR_TRANSFORM_FFT;
    int g_model = FWR_G_AVERAGED;   // measurement model of the filter tables
    int extension = FWR_EXT_ZERO;   // initial extension without a warm start
    int shape = 0;                  // kernel shape (FWR_OPT_SHAPE)
    int l2_persist = 0;             // FWR_OPT_L2_PERSIST
    size_t l2_bytes = 0;            // its access-policy window over d_scratch
    float l2_hit = 0.f;
    int ctas = 0;                   // persistent CTAs (FWR_OPT_CTAS; 0 = every SM)
    int16_t* d_hud = nullptr;       // [4][n]: pupil edges per column and row (Hudgin extension)
    double pixel = 0.0;             // d_px / d of the filter tables
    int device = 0;
    double noise_var = 0, r0 = 0, L0 = 0;
    uint8_t* d_mask = nullptr;
    std::vector<uint8_t> h_mask;  // host copy of the pupil mask (0/1)
    unsigned* d_status = nullptr;
    fwr::DevTables<float> f32;
    fwr::DevTables<double> f64;
    // 256^2 grids: per-CTA global scratch of the slab kernel
    float2* d_scratch = nullptr;
    // 256^2 grids: device address of the library's static scratch array on the
    // plan's device (looked up at plan creation; nullptr if that failed)
    float2* d_static_scratch = nullptr;
    // DFT-as-GEMM transform on 64^2 / 128^2 / 256^2 grids: operands and chunk buffers
    void* d_dftws = nullptr;
    int dftws_terms = 0;  // split products the workspace was built for (3 or 6)
    int scratch_ctas = 0;
    // host-path staging
    float* d_stage_in = nullptr;
    float* d_stage_out = nullptr;
    int stage_frames = 0;
    // host path: copy streams (H2D, D2H) and the events that join them to the
    // caller's stream, created with the staging
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in = nullptr, ev_k = nullptr, ev_done = nullptr;
    int sms = 0;
};
