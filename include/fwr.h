/*
 * fwr.h - C ABI of the GB300 (sm_103a) iterative Fourier wave-front
 * reconstructor: Gerchberg slope extension coupled to a Fourier-domain
 * least-squares / Wiener reconstructor (Bond et al., "Iterative wave-front
 * reconstruction in the Fourier domain", arXiv:1705.04298).
 *
 * The library computes, for every frame of Shack-Hartmann x/y slopes measured
 * inside a pupil:
 *   1. embed the n x n slopes in an N x N periodic grid at the centred offset
 *      off = (N - n) / 2, zero outside the pupil             (Sec. 3.2)
 *   2. optionally enforce the periodic condition: the last column of x slopes
 *      takes minus the sum of its row, the last row of y slopes minus the sum
 *      of its column                                          (Eq. PC)
 *   3. FFT, least-squares phase estimate through the discrete measurement
 *      model G, slopes re-synthesised through G, inverse FFT  (Algorithm 1,
 *      steps 1-3; the LSQ formula of Sec. 3.3)
 *   4. put the measured slopes back inside the pupil          (Algorithm 1,
 *      step 4); repeat 2-4 `iters` times
 *   5. final phase: FFT, Wiener or LSQ filter R, inverse FFT   (Eqs. 2-3)
 *
 * Conventions
 *   - Grid index [m][c]: m is the row (y), c the column (x). Slopes are phase
 *     differences across one lenslet, in radians; phase sample [m][c] is the
 *     lower-left corner of slope cell [m][c]; lenslet (i, j) of the dense
 *     input is grid cell (off + i, off + j).
 *   - Measurement model (Eq. 4, lenslet sampling x averaging x gradient),
 *     u = kx/N, v = ky/N in [-1/2, 1/2):
 *       Gx = (e^{2 i pi u} - 1) sinc(v) e^{i pi v},
 *       Gy = sinc(u) e^{i pi u} (e^{2 i pi v} - 1),
 *     with the transverse factor 0 on the Nyquist row/column. 1/|G|^2 is 0 at
 *     its nulls (piston and the waffle bin), so every output phase has zero
 *     mean over the N x N grid.
 *   - Wiener filter (Eq. 3, gamma = 1): R = G* / (|G|^2 + noise_var / W_phi)
 *     with W_phi = 0.023 (r0/d)^(-5/3) (kappa^2 + (d/L0)^2)^(-11/6), kappa in
 *     cycles per pitch. LSQ: R = G* / |G|^2. The filter inside the loop is
 *     always LSQ (Sec. 3.3); `filter` selects the final one.
 *   - All filter tables are built once per plan in FP64 on the host and
 *     rounded to the kernel's precision.
 *
 * Memory and errors
 *   - The caller owns every buffer it passes. `_dev` pointers are CUDA device
 *     pointers on the plan's device; `_host` pointers are host memory (pinned
 *     memory gives asynchronous copies).
 *   - A plan owns its device tables. fwr_reconstruct* allocate nothing and
 *     are asynchronous on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream).
 *   - Invalid arguments return FWR_ERR_ARG or FWR_ERR_UNSUPPORTED before any
 *     launch. A failed launch returns FWR_ERR_CUDA. Conditions found on the
 *     device (non-finite input slopes) set a sticky per-plan status word read
 *     by fwr_get_status; the kernels never trap.
 *   - A plan may be used from one host thread at a time.
 */
#ifndef FWR_H
#define FWR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fwr_plan fwr_plan;

typedef enum {
    FWR_LSQ = 0,     /* R = G* / |G|^2 (gamma = 0 in Eq. 3) */
    FWR_WIENER = 1   /* R = G* / (|G|^2 + noise_var / W_phi) (gamma = 1) */
} fwr_filter;

typedef enum {
    FWR_OK = 0,
    FWR_ERR_ARG = 1,          /* invalid argument; nothing launched */
    FWR_ERR_UNSUPPORTED = 2,  /* valid but not supported by the library (grid size, precision, path) */
    FWR_ERR_CUDA = 3,         /* CUDA runtime error (allocation, launch) */
    FWR_ERR_NONFINITE = 4,    /* a measured slope was NaN or Inf (device status) */
    FWR_ERR_TIMEOUT = 5       /* a bounded device wait gave up (device status) */
} fwr_status;

/* Option keys for fwr_plan_set_option. */
#define FWR_OPT_PERIODIC 1
#define FWR_OPT_TRANSFORM 2
/* Values of FWR_OPT_TRANSFORM: how the FP32 entry points take 2-D transforms. */
#define FWR_TRANSFORM_FFT 0         /* shared-memory FFT (default) */
#define FWR_TRANSFORM_DFT_BF16X3 1  /* dense DFT products on the tensor cores with split-BF16
                                       operands (x = hi + lo, products hi*hi + hi*lo + lo*hi,
                                       FP32 accumulation). N = 32: per-frame mma.sync
                                       products in one kernel. N = 64, 128 or 256: batched tcgen05
                                       GEMMs over chunks of frames (two per 2-D transform; the
                                       first writes the second's split operand from its
                                       epilogue) with element-wise kernels between transforms;
                                       setting the option allocates the plan's workspace
                                       (about 270 MB) and the
                                       reconstruct calls allocate nothing; no ext_out (returns
                                       FWR_ERR_UNSUPPORTED). Other N: FWR_ERR_UNSUPPORTED.
                                       About 2e-5 relative phase error (stated by the tests) */
#define FWR_TRANSFORM_DFT_BF16X6 2  /* the batched tcgen05 DFT-as-GEMM path of N = 64, 128 and 256
                                       with a three-way BF16 split (x = hi + mid + lo) and six
                                       products (hh + hm + mh + hl + mm + lh) over K = 12N: twice
                                       the GEMM work of DFT_BF16X3 for the same measured error
                                       (about 2e-5: the tensor core's FP32 accumulation over K,
                                       not the operand split, sets it). Other N:
                                       FWR_ERR_UNSUPPORTED.
                                       Setting it allocates its own workspace (about 480 MB),
                                       replacing a DFT_BF16X3 one (the plan falls back to
                                       the FFT transform if that allocation fails) */
/* Values of FWR_OPT_PERIODIC: where Eq. PC is applied. */
#define FWR_PERIODIC_BEFORE_EACH_FFT 0 /* before every forward FFT, the final one included (default) */
#define FWR_PERIODIC_FINAL_ONLY 1      /* once, before the final reconstruction (Algorithm 1 step 5) */
#define FWR_PERIODIC_NONE 2            /* never */
/*
 * Measurement model G of Eq. 4 (Sec. 2); both keys rebuild the plan's filter
 * tables in FP64. The new tables are uploaded, then the device is
 * synchronised before the old ones are freed (running launches may read
 * them); on failure the plan keeps its previous model and tables. Batches and
 * warm starts made from the plan keep the tables they were made with.
 *   FWR_OPT_G_MODEL: the transverse factor of G, i.e. how a slope averages
 *     across the lenslet. FWR_G_AVERAGED (default): the lenslet-averaged
 *     gradient, Gx = a(u) sinc(v) e^{i pi v}. FWR_G_FRIED: phase known at the
 *     lenslet corners, each slope the mean of the two edge differences,
 *     Gx = a(u) cos(pi v) e^{i pi v}. (Gy: u and v exchanged.)
 *   FWR_OPT_PIXEL: d_px / d in [0, 0.5], the detector pixel over the lenslet
 *     pitch. The slope is the difference of the transverse averages over
 *     d - d_px (the pixel correction of Sec. 2), per lenslet:
 *     a(u) = 2i sin(pi u (1 - d_px/d)) / (1 - d_px/d) e^{i pi u}; 0 (default)
 *     gives a(u) = e^{2 i pi u} - 1. Six pixels per lenslet: 1/6.
 */
#define FWR_OPT_G_MODEL 3
#define FWR_OPT_PIXEL 4
#define FWR_G_AVERAGED 0
#define FWR_G_FRIED 1
/*
 * FWR_OPT_EXTENSION: the slopes outside the pupil before the first iteration
 * when no warm start is passed. FWR_EXT_ZERO (default): zero. FWR_EXT_HUDGIN:
 * the Hudgin extension of Sec. 3.2 (after Poyneer et al.): every x slope
 * outside the pupil takes the measured x slope at the top or bottom pupil
 * edge of its column (up or down to the grid edge), every y slope the
 * measured y slope at the left or right pupil edge of its row; gaps inside a
 * column or row and columns or rows without pupil cells stay 0. With 0
 * iterations and the periodic condition this is the paper's Hudgin method;
 * with more, a Gerchberg loop started from it. Computed inside the kernels
 * from the staged slopes (no extra memory traffic). Supported by the FFT
 * paths of fwr_reconstruct_ex / fwr_reconstruct_f64 / fwr_reconstruct_host /
 * fwr_reconstruct_static; the DFT-as-GEMM transform and the generic kernel
 * for large pupils on 128x128 grids return FWR_ERR_UNSUPPORTED; batches and
 * warm-start objects start from their own extension.
 */
#define FWR_OPT_EXTENSION 5
#define FWR_EXT_ZERO 0
#define FWR_EXT_HUDGIN 1
/*
 * Launch shape of the FP32 FFT kernels (not part of the method: every value
 * gives bitwise the same result, only the speed differs; fwr_plan_autotune
 * picks them by timing).
 *   FWR_OPT_SHAPE: 256x256 grids: the CTA's 16 warps work the slabs as one
 *     group on 64-line slabs (1) or as two groups of 8 on 32-line slabs at
 *     the same time (2, the default 0). N <= 128: the final filter's weights
 *     are kept in shared memory where they fit (1, the default 0) or read from
 *     L2 (2). Values 0..2.
 *   FWR_OPT_CTAS: persistent CTAs of one launch, 0 (default) = every SM times
 *     the CTAs that fit on one; a larger value is clamped to that.
 */
#define FWR_OPT_SHAPE 6
#define FWR_OPT_CTAS 7
/*
 * FWR_OPT_L2_PERSIST (256x256 and 512x512 plans; FWR_ERR_UNSUPPORTED for
 * others): 1 marks the plan's working memory (one grid per SM) as persisting
 * in L2 for the slab kernel's launches (an access-policy window launch
 * attribute; CUDA-graph capturable), so its lines are not evicted by the
 * phase output and the slopes. Setting it raises the calling process's
 * persisting-L2 set-aside (cudaLimitPersistingL2CacheSize, a limit of the
 * CUDA context, released when the process exits; never lowered) to the
 * working memory's size or the device's maximum, whichever is smaller; the
 * persisting lines stay in L2 after the launches until other persisting
 * data displaces them or fwr_l2_persist_reset is called. The set-aside also
 * takes L2 from the process's other kernels: measured on the GB300, split-BF16
 * DFT and warm-start GEMMs run after a windowed 256x256 plan were 25-40 %
 * slower until the reset. 0 (default): no window. Results are bitwise the
 * same either way. Opt-in only: fwr_plan_autotune keeps the caller's setting.
 */
#define FWR_OPT_L2_PERSIST 8

/*
 * Create a plan for an n x n lenslet array (Sec. 2; Algorithm 1 input).
 *   n_lenslets  n >= 2
 *   pad_factor  N = next power of two >= ceil(pad_factor * n); N must be in
 *               {16, 32, 64, 128, 256} and N >= n + 2 (the fill column/row
 *               and the grid's last phase corners lie outside the pupil)
 *   pupil_mask  HOST, n*n bytes row-major, nonzero = valid lenslet; copied
 *               into the plan. At least one entry must be nonzero.
 *   filter      final filter (fwr_filter)
 *   noise_var   slope noise variance, rad^2 (>= 0; used by FWR_WIENER)
 *   r0, L0      Fried parameter and outer scale IN LENSLET PITCHES (> 0 for
 *               FWR_WIENER; ignored for FWR_LSQ)
 * Allocates the plan's device tables on the current CUDA device.
 * Returns FWR_OK and *out, or an error with *out = NULL.
 */
fwr_status fwr_plan_create(fwr_plan** out, int n_lenslets, double pad_factor,
                           const uint8_t* pupil_mask, int filter, double noise_var,
                           double r0, double L0);

/*
 * As fwr_plan_create, with the grid size N given instead of a pad factor:
 * the paper's small windows of w lenslets around the pupil (N = n + 2w,
 * Sec. 4.1: w = 3 and 6). N >= n + 2. A power of two in {16, ..., 256} gives
 * the same plan as fwr_plan_create. Any other N must be even and in
 * [16, 64]: such plans run the direct-DFT kernel (every 1-D transform a
 * direct sum over the line, O(N) per output) in FP32 and FP64 through
 * fwr_reconstruct, _ex, _f64 and _host, with every periodic mode, both
 * filters, warm starts and ext_out; the Hudgin extension, the DFT-as-GEMM
 * transform, ragged batches, the static-scratch call and warm-start objects
 * return FWR_ERR_UNSUPPORTED for them. FWR_ERR_UNSUPPORTED for other N.
 */
fwr_status fwr_plan_create_grid(fwr_plan** out, int n_lenslets, int N, const uint8_t* pupil_mask, int filter,
                                double noise_var, double r0, double L0);

/* Free a plan and its device tables (NULL is ignored). Not stream-ordered:
 * the caller makes sure no work using the plan is still running. */
void fwr_plan_destroy(fwr_plan* plan);

/* Padded grid size N of the plan, or -1 for NULL. */
int fwr_plan_grid(const fwr_plan* plan);

/* Number of valid lenslets in the plan's mask, or -1 for NULL. */
int fwr_plan_valid_count(const fwr_plan* plan);

/* Set a plan option (FWR_OPT_*). FWR_ERR_ARG for an unknown key or value. */
fwr_status fwr_plan_set_option(fwr_plan* plan, int key, double value);

/*
 * Reconstruct n_frames frames in FP32 (Algorithm 1 + Eqs. 2-3).
 *   slopes_dev  [n_frames][2][n][n] float, x slopes then y slopes; entries
 *               outside the mask are ignored
 *   iters       Gerchberg iterations, 0 <= iters <= 64 (0 = zero padding,
 *               plus the periodic fill where the option asks for it)
 *   phase_dev   [n_frames][N][N] float output, radians, zero mean; 16-byte
 *               aligned (FWR_ERR_ARG otherwise; all entry points that write
 *               a phase)
 * n_frames = 0 is a no-op. All work is one persistent kernel launch. For
 * N = 256 the grid of each frame is streamed through shared memory from a
 * plan-owned global scratch area (one 512 KB area per SM, allocated by
 * fwr_plan_create), so two calls on one plan must not run concurrently.
 */
fwr_status fwr_reconstruct(fwr_plan* plan, const float* slopes_dev, int n_frames, int iters,
                           float* phase_dev, void* stream);

/*
 * As fwr_reconstruct, with two optional extras (ext_out needs N <= 128).
 *   ext_init_dev  [n_frames][2][N][N] initial slopes used OUTSIDE the pupil
 *                 before the first iteration (a warm start), or NULL for 0;
 *                 16-byte aligned (FWR_ERR_ARG otherwise; same for the FP64
 *                 entry point)
 *   phase_dev     may be NULL (no final reconstruction)
 *   ext_out_dev   [n_frames][2][N][N] output: the extended slopes that enter
 *                 the final reconstruction (after the periodic fill where it
 *                 applies), or NULL
 */
fwr_status fwr_reconstruct_ex(fwr_plan* plan, const float* slopes_dev, const float* ext_init_dev,
                              int n_frames, int iters, float* phase_dev, float* ext_out_dev,
                              void* stream);

/*
 * The same computation in FP64 throughout (tables, transforms, filters). Same
 * layouts with double elements. Supported for N <= 64 (an FP64 grid of
 * 128^2 does not fit in one SM's shared memory): FWR_ERR_UNSUPPORTED
 * otherwise. Meant for parity checks, not throughput.
 */
fwr_status fwr_reconstruct_f64(fwr_plan* plan, const double* slopes_dev, const double* ext_init_dev,
                               int n_frames, int iters, double* phase_dev, double* ext_out_dev,
                               void* stream);

/*
 * End-to-end FP32 call on HOST buffers: copies slopes_host
 * ([n_frames][2][n][n]) to plan-owned device staging, reconstructs and copies
 * the phase back to phase_host ([n_frames][N][N]), ordered on `stream`.
 * The frames go in chunks of whole SM-waves (at least two, at most four
 * chunks): the plan's two copy streams move chunk c + 1 in and chunk c - 1
 * out while chunk c is reconstructed on `stream`, joined to `stream` by
 * events, so work enqueued on `stream` afterwards sees the whole result.
 * Host buffers should be pinned for the copies to overlap (pageable buffers
 * give the same result without overlap). The staging grows on demand
 * (cudaMalloc on the first call with a larger n_frames; fwr_plan_reserve does
 * it ahead and creates the copy streams). Calls on one plan must not run
 * concurrently from several host threads. Returns after enqueueing; the
 * caller synchronises `stream` before reading phase_host.
 */
fwr_status fwr_reconstruct_host(fwr_plan* plan, const float* slopes_host, int n_frames, int iters,
                                float* phase_host, void* stream);

/*
 * Choose the plan's launch shape (FWR_OPT_SHAPE, FWR_OPT_CTAS) by timing the
 * candidates on the caller's data: fwr_reconstruct_ex of n_frames frames
 * (slopes_dev, phase_dev as there) with `iters` iterations, one warm-up and
 * three timed launches per candidate, on `stream` (synchronises it). The
 * fastest is set on the plan and appended to the JSON-lines file cache_path
 * (NULL: no cache) under a key of the device (name, SM count), the driver and
 * runtime versions, the plan's geometry and options, n_frames and iters; an
 * entry for the same key is applied without timing. Candidates: the shapes
 * the plan's grid has (two for 256x256 and for N <= 128 when the final weights
 * fit shared memory) times the CTA counts {all, 3/4, 1/2 of the SMs} (times
 * the CTAs per SM). FWR_OPT_L2_PERSIST is not a candidate (it stays as
 * set); a cached entry's value is applied. Every candidate gives bitwise the
 * same phase.
 */
fwr_status fwr_plan_autotune(fwr_plan* plan, const float* slopes_dev, int n_frames, int iters, float* phase_dev,
                             void* stream, const char* cache_path);
/* The plan's current FWR_OPT_SHAPE, FWR_OPT_CTAS and FWR_OPT_L2_PERSIST (-1 for NULL). */
int fwr_plan_shape(const fwr_plan* plan);
int fwr_plan_ctas(const fwr_plan* plan);
int fwr_plan_l2_persist(const fwr_plan* plan);
/*
 * Give the whole L2 of `device` back to the process's other work: every line
 * that FWR_OPT_L2_PERSIST launches left persisting returns to normal status
 * (cudaCtxResetPersistingL2Cache in that device's context) and the
 * persisting set-aside returns to its value before the library first raised
 * it. Plans keep their window option; setting FWR_OPT_L2_PERSIST to 1 again
 * raises the set-aside again. Call with no launch in flight on the device.
 * FWR_ERR_ARG for an invalid device.
 */
fwr_status fwr_l2_persist_reset(int device);

/* Pre-allocate host-path staging for n_frames frames (and the copy streams). */
fwr_status fwr_plan_reserve(fwr_plan* plan, int n_frames);

/*
 * Ragged batches: frames of several plans (128x128 and 256x256 grids mixed,
 * e.g. pupils of 40, 64, 80 and 128 lenslets across) reconstructed by ONE
 * persistent kernel launch. The batch fixes which plan each frame uses and
 * the number of iterations; it owns a schedule (the frames each CTA
 * processes, balanced on the host by longest-processing-time-first with a
 * per-frame cost of 1 for 128x128 and `cost_ratio` for 256x256) and, when a
 * 256x256 plan is present, the working memory of its frames (512 KB per SM).
 *
 * fwr_batch_create
 *   plans        HOST array of n_plans plans on one device; each must have
 *                N = 128 (n <= 85) or N = 256 (FWR_ERR_UNSUPPORTED otherwise).
 *                The plans must outlive the batch; their options are read at
 *                creation.
 *   frame_plan   HOST array of n_frames plan indices, copied
 *   iters        Gerchberg iterations for every frame (0..64)
 * fwr_batch_run: one launch on `stream`, no allocation, no host
 * synchronisation (CUDA-graph capturable).
 *   slopes_dev   DEVICE array of n_frames device pointers; frame f points to
 *                [2][n][n] floats of its plan
 *   phase_dev    DEVICE array of n_frames device pointers to [N][N] floats
 * Runs on one batch must not overlap on the GPU (shared working memory).
 * fwr_batch_schedule re-balances with `ctas` persistent CTAs (1 .. SM count)
 * and a 256x256/128x128 cost ratio; fwr_batch_autotune times candidate
 * (ctas, cost_ratio, shape) triples on the caller's data (synchronises
 * `stream`), keeps the fastest and appends it to the JSON-lines file
 * cache_path (NULL: no cache); a cached entry for the same device, driver and
 * runtime versions, plans, frame counts and iterations is applied without
 * timing.
 */
typedef struct fwr_batch fwr_batch;
fwr_status fwr_batch_create(fwr_batch** out, fwr_plan* const* plans, int n_plans, const int* frame_plan,
                            int n_frames, int iters);
fwr_status fwr_batch_run(fwr_batch* batch, const float* const* slopes_dev, float* const* phase_dev,
                         void* stream);
fwr_status fwr_batch_schedule(fwr_batch* batch, int ctas, double cost_ratio);
fwr_status fwr_batch_autotune(fwr_batch* batch, const float* const* slopes_dev, float* const* phase_dev,
                              void* stream, const char* cache_path);
int fwr_batch_ctas(const fwr_batch* batch);
double fwr_batch_cost_ratio(const fwr_batch* batch);
/* The 256x256 frames' kernel shape (as FWR_OPT_SHAPE: 1 or 2 warp groups;
 * default 2), also chosen by fwr_batch_autotune when a 256x256 plan is
 * present; bitwise the same result either way. */
int fwr_batch_shape(const fwr_batch* batch);
fwr_status fwr_batch_set_shape(fwr_batch* batch, int shape);
void fwr_batch_destroy(fwr_batch* batch);

/*
 * One-call ragged reconstruction: every frame f goes through plan
 * plans[frame_plan_dev[f]] (Algorithm 1 and Eqs. 2-3 per frame, as
 * fwr_reconstruct), all frames in ONE persistent kernel launch on `stream`.
 *   plans           HOST array of n_plans plans on one device, each N = 128
 *                   (n <= 85) or N = 256 (FWR_ERR_UNSUPPORTED otherwise)
 *   frame_plan_dev  DEVICE int array [n_frames] of plan indices
 *   slopes_dev      DEVICE array of n_frames device pointers, frame f's
 *                   [2][n][n] floats of its plan
 *   phase_dev       DEVICE array of n_frames device pointers to [N][N]
 *                   floats (16-byte aligned)
 *   iters           Gerchberg iterations of every frame, 0..64
 * The schedule (frames per CTA, longest first, grouped by plan; the batch
 * object above with its default schedule) is built on the first call for a
 * given (plans, their tables and periodic modes, frame_plan_dev, n_frames,
 * iters) and kept: that first call reads frame_plan_dev after the caller's
 * earlier work on `stream` (synchronising it), validates every index
 * (FWR_ERR_ARG) and allocates the schedule and, with a 256x256 plan, 512 KB
 * of working memory per SM. Later calls with the same key allocate nothing
 * and do not synchronise (CUDA-graph capturable). The kernel reads each
 * frame's plan from frame_plan_dev at run time, so rewriting its contents
 * keeps results correct (only the load balance is the first call's); a frame
 * whose index has become invalid is skipped and sets FWR_ERR_ARG in the
 * status word of plans[0] (fwr_get_status). Calls with one key must not
 * overlap on the GPU (shared working memory). The plans must outlive the
 * kept schedules: fwr_ragged_release frees all of them (synchronises the
 * devices through cudaFree).
 */
fwr_status fwr_reconstruct_ragged(fwr_plan* const* plans, int n_plans, const int* frame_plan_dev,
                                  const float* const* slopes_dev, int n_frames, int iters,
                                  float* const* phase_dev, void* stream);
void fwr_ragged_release(void);

/*
 * Learned warm start (the paper has no learned component; this is the
 * project's addition). A small U-Net predicts the slopes outside the pupil
 * from the measured ones; passed as ext_init to fwr_reconstruct_ex it lets
 * one or two Gerchberg iterations approach the result of many.
 * Definition: input 3 x 32 x 32 (x and y slopes inside the pupil, times 0.5,
 * and the pupil indicator, on the 128 x 128 grid averaged over 4 x 4 blocks);
 * 4 levels of widths (w, 2w, 4w, 4w), two 3 x 3 convolutions with bias and
 * ReLU per level, 2 x 2 average pooling, nearest 2 x upsampling, skip
 * concatenation [upsampled, skip]; 1 x 1 convolution to 2 channels; the
 * output divided by 0.5 and repeated over 4 x 4 blocks is the warm start.
 * BF16 weights and activations, FP32 accumulation, FP32 master weights and
 * Adam. Weights are a flat FP32 vector, layer by layer (e1a e1b e2a e2b e3a
 * e3b ba bb d3a d3b d2a d2b d1a d1b out), each W[cout][dy][dx][cin] then the
 * bias[cout].
 *
 * fwr_net_create     width w (1..32), largest batch, optional HOST initial
 *                    weights (count must equal fwr_net_param_count; NULL:
 *                    zeros). Allocates all buffers.
 * fwr_net_forward    plan must have N = 128; slopes_dev [F][2][n][n];
 *                    ext_init_dev [F][2][128][128] output (F <= largest batch)
 * fwr_net_gradients  forward, masked MSE against the 4 x 4 block means of
 *                    target_ext_dev [F][2][128][128] over blocks without pupil
 *                    cells (last block row/column excluded), backward;
 *                    optional HOST outputs: the gradient (param_count floats)
 *                    and the loss. Synchronises `stream`.
 * fwr_net_train_step fwr_net_gradients then one Adam step (lr; betas 0.9,
 *                    0.999; eps 1e-8).
 * fwr_net_set_option FWR_NET_OPT_CONV: FWR_NET_CONV_AUTO (default) runs the
 *                    forward 3 x 3 convolutions whose input channel groups are
 *                    multiples of 16 and output channels multiples of 8 on the
 *                    tensor cores (implicit GEMM, BF16 in, FP32 accumulate);
 *                    FWR_NET_CONV_SIMT keeps every convolution on the CUDA
 *                    cores. Both sum in FP32 and round the stored activation to
 *                    BF16; they differ only in summation order. Unknown option
 *                    or value: FWR_ERR_ARG.
 * fwr_net_tc_layers  how many layers are eligible for the tensor-core forward
 *                    (-1 for NULL).
 */
#define FWR_NET_OPT_CONV 1
#define FWR_NET_CONV_AUTO 0
#define FWR_NET_CONV_SIMT 1
typedef struct fwr_net fwr_net;
fwr_status fwr_net_create(fwr_net** out, int width, int max_batch, const float* init_weights, int count);
void fwr_net_destroy(fwr_net* net);
int fwr_net_param_count(const fwr_net* net);
fwr_status fwr_net_get_weights(fwr_net* net, float* host, int count);
fwr_status fwr_net_set_weights(fwr_net* net, const float* host, int count);
fwr_status fwr_net_forward(fwr_net* net, const fwr_plan* plan, const float* slopes_dev, int n_frames,
                           float* ext_init_dev, void* stream);
fwr_status fwr_net_gradients(fwr_net* net, const fwr_plan* plan, const float* slopes_dev,
                             const float* target_ext_dev, int n_frames, float* grad_host, float* loss_host,
                             void* stream);
fwr_status fwr_net_train_step(fwr_net* net, const fwr_plan* plan, const float* slopes_dev,
                              const float* target_ext_dev, int n_frames, float lr, float* loss_host,
                              void* stream);
fwr_status fwr_net_set_option(fwr_net* net, int option, int value);
int fwr_net_tc_layers(const fwr_net* net);

/*
 * The schedule of ragged batches, on the host only: assign n jobs with
 * costs[i] >= 0 to `ctas` workers, longest first to the least loaded worker.
 * Output: worker c runs order[cta_off[c] .. cta_off[c+1]) (cta_off has
 * ctas + 1 entries, order has n).
 */
fwr_status fwr_schedule_lpt(const double* costs, int n, int ctas, int* cta_off, int* order);

/*
 * fwr_reconstruct without any device allocation, for 256x256 grids.
 * (The paper has no counterpart: this is a deployment convenience.)
 *
 * For callers that must not allocate GPU memory once they are running: a
 * real-time control loop that forbids allocation after start-up (an
 * allocation can stall for milliseconds), or a process whose device memory
 * belongs to another allocator or to a fixed budget. Reconstructing a
 * 256x256 grid needs 512 KB of working memory per frame in flight, which
 * fwr_reconstruct takes from the plan (one area per SM, allocated when the
 * plan is created). This entry point instead uses an array that is part of
 * the library itself: room for FWR_STATIC_SCRATCH_GRIDS frames in flight
 * (8 MB), present on every GPU that loads the library until the process
 * exits. It calls no cudaMalloc or cudaFree, and loads nothing: creating a
 * 256x256 plan loads the library's device code on the plan's device and
 * looks up the array's address there, so do that at start-up (a plan made
 * before a cudaDeviceReset is unusable after it, like all its memory).
 *
 *   plan          a plan with N = 256 and the shared-memory FFT transform
 *                 (FWR_ERR_UNSUPPORTED otherwise: other grids have no scratch,
 *                 and FWR_TRANSFORM_DFT_BF16X3 has its own workspace)
 *   slopes_dev, n_frames, iters, phase_dev, stream   as for fwr_reconstruct
 *   ctas          frames processed concurrently, 1 .. FWR_STATIC_SCRATCH_GRIDS
 *                 (FWR_ERR_ARG otherwise; fwr_last_error() says why); any
 *                 n_frames is accepted, the CTAs loop over the frames
 *
 * The kernel is fwr_reconstruct's, on the same tables and options (periodic
 * mode, measurement model, Hudgin extension), so the results are bitwise
 * equal to fwr_reconstruct's. The array is shared by all calls on a device and
 * keeps the last call's contents; nothing in it needs to start at zero,
 * because every frame writes its whole area before reading it. Calls that
 * overlap on the GPU (other streams, other threads, other plans) race on the
 * array: serialise them.
 */
#define FWR_STATIC_SCRATCH_GRIDS 16
fwr_status fwr_reconstruct_static(fwr_plan* plan, const float* slopes_dev, int n_frames, int iters,
                                  float* phase_dev, int ctas, void* stream);

/*
 * Batched 2-D FFT of n_frames complex N x N grids with the kernels' own
 * shared-memory FFT (the transform used inside the loop), FP32 interleaved
 * complex (re, im). Forward: X[ky][kx] = sum x[m][c] e^{-2 i pi (ky m + kx c)/N};
 * inverse (inverse != 0) uses +i and no 1/N^2 scaling. N in {16,...,128};
 * in_dev and out_dev may be the same buffer.
 */
fwr_status fwr_fft2(int N, const float* in_dev, float* out_dev, int n_frames, int inverse,
                    void* stream);

/*
 * Batched 2-D DFT of n_frames complex N x N grids as dense products on the
 * tensor cores with split-BF16 operands (the transform of
 * FWR_TRANSFORM_DFT_BF16X3). Same layouts and sign conventions as fwr_fft2;
 * N in {32, 64}.
 */
fwr_status fwr_dft2_bf16x3(int N, const float* in_dev, float* out_dev, int n_frames, int inverse,
                           void* stream);

/*
 * Read and clear the plan's sticky device status word. Synchronises the
 * plan's device. FWR_OK, FWR_ERR_NONFINITE, FWR_ERR_TIMEOUT or (ragged
 * launches given an invalid plan index) FWR_ERR_ARG.
 */
fwr_status fwr_get_status(fwr_plan* plan);

/*
 * Linear warm start (the project's addition; Algorithm 1, Sec. 3.3, is linear
 * in the slopes, so the extension the loop reaches after k iterations from a
 * zero start is one fixed matrix E_k applied to the measured slopes).
 *
 * fwr_linws_create   plan: the geometry (its mask fixes the valid cells);
 *                    rank r: a multiple of 128 in [128, 8192];
 *                    A_host [2 n_valid][r] and V_host [2 N^2][r], FP32, HOST,
 *                    a factorisation E ~ A V^T (copied and rounded to BF16; the
 *                    caller keeps ownership). Slope index j < n_valid is the x
 *                    slope of the j-th valid lenslet in row-major order, j >=
 *                    n_valid the y slope of lenslet j - n_valid; the extension
 *                    index is the flat [2][N][N] index of ext_init.
 *                    max_batch: largest F. 2 N^2 must be a multiple of 128.
 * fwr_linws_forward  slopes_dev [F][2][n][n] FP32 -> ext_init_dev [F][2][N][N]
 *                    FP32 (16-byte aligned) = (X A) V^T with X the gathered
 *                    slopes, on the tcgen05 tensor cores (BF16 operands, FP32
 *                    accumulation; X A rounded to BF16). Asynchronous on
 *                    `stream`; a pipeline wait that runs out is recorded and
 *                    reported by fwr_linws_status (synchronises the device).
 *                    The result feeds fwr_reconstruct_ex as ext_init.
 * fwr_linws_reconstruct
 *                    the warm start and the reconstruction in one call:
 *                    fwr_linws_forward into a BF16 buffer owned by `ws`
 *                    ([max_batch][2 N^2], allocated at creation), then the
 *                    fused kernel of fwr_reconstruct_ex reading it (iters
 *                    0..64, phase_dev [F][N][N]). `plan` must have the grid and
 *                    the pupil mask `ws` was created with (its filter may
 *                    differ); FWR_ERR_ARG otherwise, FWR_ERR_UNSUPPORTED for
 *                    plans that do not take the fused path (N = 256, the
 *                    DFT-GEMM transform). Asynchronous on `stream`.
 * fwr_gemm_bf16_tc   the tensor-core GEMM on its own (synchronous): D [M][N]
 *                    FP32 = A [M][K] B[N][K]^T, A and B BF16 row-major device
 *                    arrays (16-byte aligned), K a positive multiple of 8, N a
 *                    multiple of 128; FWR_ERR_TIMEOUT if a wait ran out.
 * The GEMM kernel allocates up to 512 TMEM columns per CTA (one CTA per SM);
 * it is not meant to share an SM with other TMEM users on another stream.
 */
typedef struct fwr_linws fwr_linws;
fwr_status fwr_linws_create(fwr_linws** out, const fwr_plan* plan, int rank, const float* A_host,
                            const float* V_host, int max_batch);
void fwr_linws_destroy(fwr_linws* ws);
int fwr_linws_valid_count(const fwr_linws* ws);
fwr_status fwr_linws_forward(fwr_linws* ws, const float* slopes_dev, int n_frames, float* ext_init_dev,
                             void* stream);
fwr_status fwr_linws_reconstruct(fwr_linws* ws, fwr_plan* plan, const float* slopes_dev, int n_frames,
                                 int iters, float* phase_dev, void* stream);
fwr_status fwr_linws_status(fwr_linws* ws);
fwr_status fwr_gemm_bf16_tc(const void* A_dev, const void* B_dev, int M, int N, int K, float* D_dev, void* stream);
/*
 * fwr_gemm_bf16_tc with the MMA issuer's and the epilogue's mbarrier waits
 * bounded by wait_cycles (1 .. 4e9 SM clock cycles; fwr_gemm_bf16_tc uses
 * 4e9, about two seconds) instead of the default. For testing the timeout
 * path: with a few cycles the issuer gives up before the first operand tiles
 * land, the kernel drains its loads in flight (those waits keep the full
 * bound), frees its tensor memory and the call returns FWR_ERR_TIMEOUT with
 * the context intact. D is then undefined.
 */
fwr_status fwr_gemm_bf16_tc_limit(const void* A_dev, const void* B_dev, int M, int N, int K, float* D_dev,
                                  long long wait_cycles, void* stream);

/*
 * Measured FP32 FMA throughput of the current device, the peak of the FFT
 * path's roofline: 2 CTAs of 512 threads per SM, each thread 8 independent
 * FMA chains, best of five timed launches (about 2 ms each) after a warm-up,
 * synchronous on `stream`. *tflops = 2 x FMAs / time in TFLOP/s; *ms (may be
 * NULL) the launch time.
 */
fwr_status fwr_fp32_fma_peak(double* tflops, double* ms, void* stream);

/* Static, human-readable name of a status code. */
const char* fwr_status_string(fwr_status status);

/* Text of the last CUDA error seen by the library on this thread ("" if none). */
const char* fwr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FWR_H */
