// Internal interface between the C ABI (fwr_api.cpp) and the kernels
// (fwr_gerchberg.cu). Not installed; the public interface is include/fwr.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fwr {

template <typename T> struct cvec;
template <> struct cvec<float> { typedef float2 type; };
template <> struct cvec<double> { typedef double2 type; };

// Per-plan filter tables, built in FP64 on the host (Eqs. 3-4, Sec. 3.3) and
// rounded to T. Spectral tables cover rows ky = 0 .. N/2 only: both weights
// are even in k, and the kernels visit each (k, -k) pair once from that half.
template <typename T> struct Tables {
    const typename cvec<T>::type* tw;  // [N]   e^{-2 i pi j / N}
    const typename cvec<T>::type* A;   // [N]   a(u) = e^{2 i pi u} - 1
    const typename cvec<T>::type* Tt;  // [N]   T(u) = sinc(u) e^{i pi u}, 0 at u = -1/2
    const T* pt;                       // [N][4]  p(u) = a(u) conj(T(u)) (re, im), |a(u)|^2, |T(u)|^2
    const T* iota;                     // [(N/2+1) N] 1/|G|^2 / N^2 (0 at nulls)
    const T* wfin;                     // [(N/2+1) N] final weight / N^2 (LSQ or Wiener)
};

template <typename T> struct Params {
    Tables<T> tab;
    const uint8_t* mask = nullptr;       // [n n] device copy of the pupil mask
    const T* slopes = nullptr;           // [F][2][n][n]
    const T* ext_init = nullptr;         // [F][2][N][N] or nullptr
    const uint16_t* ext_init_h = nullptr;  // the same in BF16 (bit patterns; fused kernel only) or nullptr
    T* phase = nullptr;                  // [F][N][N] or nullptr
    T* ext_out = nullptr;                // [F][2][N][N] or nullptr
    int n = 0, off = 0, F = 0, iters = 0, periodic = 0;
    unsigned* status = nullptr;          // sticky device status bits
    int wf_smem = 0;                     // fused kernel: final weights resident in shared memory (set by its launcher)
    // Hudgin extension as the initial extension (no warm start given): per
    // lenslet column j the first / last pupil row, hud[j] / hud[n + j], per
    // row i the first / last pupil column, hud[2n + i] / hud[3n + i]; -1 where
    // the column or row has no pupil cell. nullptr: zero extension.
    const int16_t* hud = nullptr;
    // kernel shape (the plan's FWR_OPT_SHAPE; results are bitwise the same for
    // every value): 256^2 slab kernel: warp groups, 1 or 2 (0: 2); fused
    // kernel: final-filter weights 1 = in shared memory where they fit, 2 =
    // read from L2 (0: 1)
    int shape = 0;
    int ctas = 0;   // persistent CTAs (0: every SM, times the resident CTAs per SM)
    // slab kernel: an L2 access-policy window over the scratch (FWR_OPT_L2_PERSIST),
    // persisting hits for l2_hit of its l2_bytes; l2_bytes = 0: none
    size_t l2_bytes = 0;
    float l2_hit = 0.f;
    // fused kernel: launched as a programmatic dependent of the kernel before
    // it on the stream (its table set-up overlaps that kernel's tail; frames
    // start after it completes). Only for launches whose stream predecessor is
    // the library's own producer of this launch's inputs.
    int pdl = 0;
};

// Programmatic dependent launch (sm_90+): wait for the grids this one depends
// on to complete and their writes to be visible (no-op without a dependency);
// allow the dependent grid to launch once every CTA of this grid has signalled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Where Eq. PC is applied (same values as FWR_PERIODIC_* in fwr.h).
enum : int { PERIODIC_BEFORE_EACH_FFT = 0, PERIODIC_FINAL_ONLY = 1, PERIODIC_NONE = 2 };

// Status bits written by kernels.
enum : unsigned { STATUS_NONFINITE = 1u, STATUS_TIMEOUT = 2u, STATUS_BADINDEX = 4u };

// Shared-memory bytes of the generic kernel (fwr_basic.cu) for grid N.
size_t basic_smem_bytes(int N, int elem_bytes, int n);

// Generic kernel (fwr_basic.cu): one persistent launch over all frames.
cudaError_t launch_basic_f32(int N, const Params<float>& p, cudaStream_t s);
cudaError_t launch_basic_f64(int N, const Params<double>& p, cudaStream_t s);
// The generic kernel with every 2-D transform done as split-BF16 tensor-core
// DFT products (N in {32, 64}).
cudaError_t launch_basic_gemm_f32(int N, const Params<float>& p, cudaStream_t s);
// Standalone batched split-BF16 DFT (test entry), N in {32, 64}.
cudaError_t launch_dft2_gemm_f32(int N, const float2* in, float2* out, int F, int inverse, const float2* tw,
                                 cudaStream_t s);

// 256^2 and 512^2 grids (fwr_slab.cu): the grid lives in a per-CTA global
// scratch area of slab_scratch_elems_per_cta(N) float2 and is streamed
// through shared memory. launch_slab uses at most max_ctas CTAs (scratch must
// hold that many).
size_t slab_smem_bytes(int N, int n);
size_t slab_scratch_elems_per_cta(int N);
int slab_max_ctas();
cudaError_t launch_slab(int N, const Params<float>& p, float2* scratch, int max_ctas, cudaStream_t s);
// The same kernel on the library's static scratch array (no allocation):
// at most STATIC_SLAB_GRIDS CTAs; cudaErrorInvalidValue for ctas outside
// 1..STATIC_SLAB_GRIDS. static_slab_prepare (current device) returns the
// array's device address and sets the kernel's shared-memory limit for n
// lenslets; launch_slab_static takes that address.
enum : int { STATIC_SLAB_GRIDS = 16 };
cudaError_t static_slab_prepare(int n, float2** addr);
cudaError_t launch_slab_static(const Params<float>& p, float2* scratch, int ctas, cudaStream_t s);

// Ragged batches (fwr_ragged.cu): one launch over frames of several plans
// with N in {128, 256}. cta_off[grid + 1] / order[] list each CTA's frames;
// slopes[f] / phase[f] are the frame's device pointers.
struct RaggedPlan {
    Tables<float> tab;
    const uint8_t* mask;
    unsigned* status;
    int N, n, off, periodic;
};
struct RaggedParams {
    const RaggedPlan* plans;
    const int* frame_plan;
    const int* cta_off;
    const int* order;
    const float* const* slopes;
    float* const* phase;
    float2* scratch;  // grid x 256^2 (only when a 256^2 plan is present)
    int iters;
    int shape;        // warp groups of the 256^2 path (1 or 2)
    int n_plans;      // frames whose plan index is outside 0..n_plans-1 are skipped (STATUS_BADINDEX)
};
size_t ragged_smem_bytes(int N, int n);  // 0 if the plan cannot join a ragged batch
cudaError_t ragged_prepare(size_t smem);  // both shapes
cudaError_t launch_ragged(const RaggedParams& p, int grid, size_t smem, cudaStream_t s);

// Grids of any even size 16 <= N <= 64 (fwr_anygrid.cu): direct-DFT kernel
// for the paper's small windows around the pupil.
size_t anygrid_smem_bytes(int N, int elem_bytes, int n);
cudaError_t launch_anygrid_f32(int N, const Params<float>& p, cudaStream_t s);
cudaError_t launch_anygrid_f64(int N, const Params<double>& p, cudaStream_t s);

// Main fused kernel (fwr_fused.cu). fused_supported() says whether its
// shared-memory layout fits grid N with n lenslets for the element size.
bool fused_supported(int N, int elem_bytes, int n);
cudaError_t launch_fused_f32(int N, const Params<float>& p, cudaStream_t s);
cudaError_t launch_fused_f64(int N, const Params<double>& p, cudaStream_t s);

// Standalone batched 2-D FFT (test entry), FP32.
cudaError_t launch_fft2_f32(int N, const float2* in, float2* out, int F, int inverse,
                            const float2* tw, cudaStream_t s);

// tcgen05 GEMM (fwr_linws.cu): D [M][ldd] = A [M][K] B [N][K]^T, A and B
// BF16 row-major device arrays (16-byte aligned rows), K a multiple of 8, N
// of 128; FP32 or BF16 output; a pipeline wait that runs out sets bit 2 of
// *status.
cudaError_t tc_gemm(const void* A, int M, int K, const void* B, long long N, void* D, bool bf16_out, long long ldd,
                    int* status, cudaStream_t s);
// The same product (M = 2n) with its output split into BF16 terms and written
// as the next product's B operand: output (i, (f, x)), column (f, x) = f n + x,
// goes to row f n + (i mod n) of Bout [.][kout = 2 n terms], column x (+ n for
// i >= n), in each term region (3 terms: hi, lo, hi; 6: h, m, h, l, m, h).
// Bout must not be the operand B of the same call.
cudaError_t tc_gemm_split(const void* A, int M, int K, const void* B, long long N, void* Bout, int n, int kout,
                          int terms, int* status, cudaStream_t s);

// Batched split-BF16 DFT-as-GEMM path for N = 64, 128 and 256 (fwr_dftgemm_tc.cu):
// every 2-D transform of Algorithm 1 and of the final reconstruction as two
// tcgen05 GEMMs over a chunk of frames. Workspace: dftgemm_ws_bytes(N) bytes.
// terms: 3 or 6 split products (FWR_TRANSFORM_DFT_BF16X3 / X6).
size_t dftgemm_ws_bytes(int N, int terms);
int dftgemm_chunk(int N);
cudaError_t dftgemm_setup(int N, int terms, const float2* tw, void* ws);  // fills the DFT operand matrices of ws
cudaError_t launch_dftgemm_f32(int N, int terms, const Params<float>& p, void* ws, cudaStream_t s);

}  // namespace fwr
