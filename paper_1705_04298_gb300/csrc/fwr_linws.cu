// Linear warm start of the Gerchberg loop (Algorithm 1, Sec. 3.3) on the
// tcgen05 tensor cores, and the BF16 GEMM entry point it is built from.
//
// The loop is linear in the measured slopes, so the extension it reaches
// after k iterations from a zero start is E_k s for one fixed matrix E_k
// (2 n_valid slopes -> 2 N^2 extended slopes). The warm start stores a rank-r
// factorisation E ~ A V^T (A: [2 n_valid][r], V: [2 N^2][r], fitted off line
// from the operator and training frames) in BF16 and evaluates, per batch,
//   X  = the measured slopes, gathered  [F][K]   (BF16, K = 2 n_valid padded)
//   C  = X A                              [F][r]   (tcgen05 GEMM, BF16 out)
//   x0 = C V^T                            [F][2N^2] (tcgen05 GEMM, FP32 out)
// x0 is the ext_init of fwr_reconstruct_ex. The paper has no such component;
// it trades a dense contraction on the tensor cores for FP32 FFT iterations.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/fwr.h"
#include "fwr_internal.h"
#include "fwr_plan.h"
#include "fwr_umma.cuh"

namespace {

using fwr::umma::BM;

// K elements per pipeline stage of the tensor-core GEMM (32: 64-byte swizzle)
constexpr int GEMM_BK = 64;


typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// BF16 matrix [rows][ld] (ld elements per row, ld * 2 a multiple of 16) read
// as {cols, rows} in boxes of GEMM_BK x box_rows with the matching swizzle
bool make_map(CUtensorMap* map, const void* ptr, uint64_t cols, uint64_t rows, uint64_t ld, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {uint32_t(GEMM_BK), uint32_t(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, GEMM_BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, typename OutT, bool SPLIT = false, bool ARES = false>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(fwr::umma::gemm_kernel<BN, GEMM_BK, OutT, SPLIT, ARES>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(fwr::umma::Cfg<BN, GEMM_BK>::SMEM));
}

// per device: the kernels' shared-memory limit is raised once; SM count
int device_sms(int device) {
    static std::mutex mu;
    static std::vector<std::pair<int, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (auto& d : done)
        if (d.first == device) return d.second;
    int sms = 0;
    if (set_smem<128, float>() != cudaSuccess || set_smem<256, float>() != cudaSuccess ||
        set_smem<128, __nv_bfloat16>() != cudaSuccess || set_smem<256, __nv_bfloat16>() != cudaSuccess ||
        set_smem<128, float, true>() != cudaSuccess || set_smem<256, float, true>() != cudaSuccess ||
        set_smem<128, float, false, true>() != cudaSuccess || set_smem<256, float, false, true>() != cudaSuccess ||
        set_smem<128, __nv_bfloat16, false, true>() != cudaSuccess ||
        set_smem<256, __nv_bfloat16, false, true>() != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
        return 0;
    done.push_back({device, sms});
    return sms;
}

// D = A B^T. mb128 / mb256: B with boxes of 128 / 256 rows. 256-wide tiles
// when N allows them and they still give every SM a tile, else 128-wide.
// pdl: launched as a programmatic dependent of the previous kernel on the
// stream (only where that kernel is the library's producer of A).
template <typename OutT>
cudaError_t launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb128, const CUtensorMap& mb256, int M,
                        long long N, int K, OutT* D, long long ldd, int* status, cudaStream_t s,
                        long long wait_limit = fwr::umma::WAIT_LIMIT, bool pdl = false,
                        fwr::umma::SplitDst sd = fwr::umma::SplitDst()) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = device_sms(dev);
    if (sms < 1) return cudaErrorInvalidValue;
    const long long tm = (M + BM - 1) / BM;
    const int bn = (N % 256 == 0 && tm * (N / 256) >= sms) ? 256 : 128;
    const long long tiles = tm * (N / bn);
    const unsigned grid = unsigned(tiles < sms ? tiles : sms);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(fwr::umma::THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const int n32 = int(N);
    const bool split = sd.B != nullptr;
    // A resident in shared memory when every tile of a CTA has the same A rows
    // (tiles walk M fastest, so a grid that is a multiple of the M tiles keeps
    // each CTA on one row block) and K fits its k-blocks
    const int kblocks = (K + GEMM_BK - 1) / GEMM_BK;
    const bool ares = !split && kblocks <= fwr::umma::Cfg<128, GEMM_BK>::ARES_KB &&
                      (grid % unsigned(tm) == 0 || tiles <= (long long)grid);
    using namespace fwr::umma;
    if (bn == 256) {
        cfg.dynamicSmemBytes = Cfg<256, GEMM_BK>::SMEM;
        if (split)
            return cudaLaunchKernelEx(&cfg, gemm_kernel<256, GEMM_BK, OutT, true>, ma, mb256, M, n32, K, D, ldd,
                                      status, wait_limit, sd);
        if (ares)
            return cudaLaunchKernelEx(&cfg, gemm_kernel<256, GEMM_BK, OutT, false, true>, ma, mb256, M, n32, K, D,
                                      ldd, status, wait_limit, sd);
        return cudaLaunchKernelEx(&cfg, gemm_kernel<256, GEMM_BK, OutT, false>, ma, mb256, M, n32, K, D, ldd, status,
                                  wait_limit, sd);
    }
    cfg.dynamicSmemBytes = Cfg<128, GEMM_BK>::SMEM;
    if (split)
        return cudaLaunchKernelEx(&cfg, gemm_kernel<128, GEMM_BK, OutT, true>, ma, mb128, M, n32, K, D, ldd, status,
                                  wait_limit, sd);
    if (ares)
        return cudaLaunchKernelEx(&cfg, gemm_kernel<128, GEMM_BK, OutT, false, true>, ma, mb128, M, n32, K, D, ldd,
                                  status, wait_limit, sd);
    return cudaLaunchKernelEx(&cfg, gemm_kernel<128, GEMM_BK, OutT, false>, ma, mb128, M, n32, K, D, ldd, status,
                              wait_limit, sd);
}

}  // namespace

// D [M][ldd] = A [M][K] B [N][K]^T (BF16 in, FP32 accumulate, FP32 or BF16
// out), maps built per call; the library's other tensor-core users call this.
cudaError_t fwr::tc_gemm(const void* A, int M, int K, const void* B, long long N, void* D, bool bf16_out,
                         long long ldd, int* status, cudaStream_t s) {
    if (M < 1 || K < 8 || K % 8 != 0 || N < 128 || N % 128 != 0) return cudaErrorInvalidValue;
    CUtensorMap ma, mb128, mb256;
    if (!make_map(&ma, A, uint64_t(K), uint64_t(M), uint64_t(K), BM) ||
        !make_map(&mb128, B, uint64_t(K), uint64_t(N), uint64_t(K), 128) ||
        !make_map(&mb256, B, uint64_t(K), uint64_t(N), uint64_t(K), 256))
        return cudaErrorInvalidValue;
    return bf16_out ? launch_gemm<__nv_bfloat16>(ma, mb128, mb256, M, N, K, static_cast<__nv_bfloat16*>(D), ldd,
                                                 status, s)
                    : launch_gemm<float>(ma, mb128, mb256, M, N, K, static_cast<float*>(D), ldd, status, s);
}

// The same product with the split-BF16 epilogue (fwr_umma.cuh SplitDst):
// output (i, (f, x)) -> BF16 terms in row f n + (i mod n) of Bout [.][kout].
cudaError_t fwr::tc_gemm_split(const void* A, int M, int K, const void* B, long long N, void* Bout, int n, int kout,
                               int terms, int* status, cudaStream_t s) {
    if (M < 1 || M != 2 * n || K < 8 || K % 8 != 0 || N < 128 || N % 128 != 0 || n % 64 != 0 ||
        kout != 2 * n * terms || (terms != 3 && terms != 6) || !Bout)
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb128, mb256;
    if (!make_map(&ma, A, uint64_t(K), uint64_t(M), uint64_t(K), BM) ||
        !make_map(&mb128, B, uint64_t(K), uint64_t(N), uint64_t(K), 128) ||
        !make_map(&mb256, B, uint64_t(K), uint64_t(N), uint64_t(K), 256))
        return cudaErrorInvalidValue;
    fwr::umma::SplitDst sd;
    sd.B = static_cast<__nv_bfloat16*>(Bout);
    sd.n = n;
    sd.k = kout;
    sd.terms = terms;
    return launch_gemm<float>(ma, mb128, mb256, M, N, K, nullptr, 0, status, s, fwr::umma::WAIT_LIMIT, false, sd);
}

namespace {

// slopes [F][2][n][n] -> X [F][ldx] BF16: column j takes the slope at
// offset src[j] of the frame's [2][n][n] block (x slopes of the valid cells in
// row-major order, then their y slopes), or 0 where src[j] < 0 (padding).
// One block per frame; pairs of columns per thread (ldx even).
__global__ void k_gather(const float* __restrict__ sl, const int2* __restrict__ src, int nn, int ldx,
                         __nv_bfloat16* __restrict__ X) {
    // the GEMM after this kernel may start its set-up (it waits for this grid)
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int f = blockIdx.x;
    const float* s = sl + size_t(f) * 2 * nn;
    __nv_bfloat162* x = reinterpret_cast<__nv_bfloat162*>(X + size_t(f) * ldx);
#pragma unroll 4
    for (int j = threadIdx.x; j < ldx / 2; j += blockDim.x) {
        const int2 o = __ldg(src + j);
        const float a = o.x >= 0 ? __ldg(s + o.x) : 0.f, b = o.y >= 0 ? __ldg(s + o.y) : 0.f;
        x[j] = __floats2bfloat162_rn(a, b);
    }
}

// src [rows][cols] FP32 -> dst [cols][ldd] BF16 (transposed), or, when
// !transpose, dst [rows][ldd]
__global__ void k_to_bf16_2d(const float* src, int rows, int cols, bool transpose, int ldd, __nv_bfloat16* dst) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const int r = int(i / cols), c = int(i - (long long)r * cols);
    const __nv_bfloat16 v = __float2bfloat16_rn(src[i]);
    if (transpose)
        dst[size_t(c) * ldd + r] = v;
    else
        dst[size_t(r) * ldd + c] = v;
}

inline unsigned nblocks(long long n, int t) { return unsigned((n + t - 1) / t); }

fwr_status fail(fwr_status code, const char* msg) {
    fwr::set_last_error(msg);
    return code;
}

}  // namespace

struct fwr_linws {
    int n = 0, N = 0, nv = 0, K = 0, Kpad = 0, rank = 0, max_batch = 0, device = 0;
    long long cells2 = 0;                 // 2 N^2
    int* d_src = nullptr;                 // [Kpad] source offset of every X column in a frame's slopes, or -1
    __nv_bfloat16* X = nullptr;           // [max_batch][Kpad]
    __nv_bfloat16* C = nullptr;           // [max_batch][rank]
    __nv_bfloat16* At = nullptr;          // [rank][Kpad]
    __nv_bfloat16* V = nullptr;           // [2 N^2][rank]
    __nv_bfloat16* Eh = nullptr;          // [max_batch][2 N^2]: the warm start of fwr_linws_reconstruct
    int* d_status = nullptr;
    std::vector<uint8_t> mask;            // the pupil the factors were fitted for
    CUtensorMap mX, mAt128, mAt256, mC, mV128, mV256;
};

namespace {

void free_ws(fwr_linws* w) {
    cudaFree(w->d_src);
    cudaFree(w->X);
    cudaFree(w->C);
    cudaFree(w->At);
    cudaFree(w->V);
    cudaFree(w->Eh);
    cudaFree(w->d_status);
    delete w;
}

// host FP32 [rows][cols] -> device BF16, in slices of at most 16M elements
cudaError_t upload_bf16(const float* host, int rows, int cols, bool transpose, int ldd, __nv_bfloat16* dst) {
    const int slice = std::max(1, (1 << 24) / std::max(1, cols));
    float* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, size_t(std::min(slice, rows)) * cols * sizeof(float));
    for (int r0 = 0; r0 < rows && e == cudaSuccess; r0 += slice) {
        const int nr = std::min(slice, rows - r0);
        e = cudaMemcpy(tmp, host + size_t(r0) * cols, size_t(nr) * cols * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        __nv_bfloat16* d = transpose ? dst + r0 : dst + size_t(r0) * ldd;
        k_to_bf16_2d<<<nblocks((long long)nr * cols, 256), 256>>>(tmp, nr, cols, transpose, ldd, d);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(tmp);
    return e;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

fwr_status fwr_gemm_bf16_tc(const void* A, const void* B, int M, int N, int K, float* D, void* stream) {
    return fwr_gemm_bf16_tc_limit(A, B, M, N, K, D, fwr::umma::WAIT_LIMIT, stream);
}

fwr_status fwr_gemm_bf16_tc_limit(const void* A, const void* B, int M, int N, int K, float* D, long long wait_cycles,
                                  void* stream) {
    if (wait_cycles < 1 || wait_cycles > fwr::umma::WAIT_LIMIT)
        return fail(FWR_ERR_ARG, "fwr_gemm_bf16_tc_limit: wait_cycles outside 1 .. 4e9");
    if (M < 0 || N < 0 || K < 0) return fail(FWR_ERR_ARG, "fwr_gemm_bf16_tc: negative size");
    if (M == 0 || N == 0) return FWR_OK;
    if (K < 1 || K % 8 != 0 || N % 128 != 0)
        return fail(FWR_ERR_ARG, "fwr_gemm_bf16_tc: K must be a positive multiple of 8, N of 128");
    if (!A || !B || !D || !aligned16(A) || !aligned16(B) || !aligned16(D))
        return fail(FWR_ERR_ARG, "fwr_gemm_bf16_tc: null or unaligned pointer");
    CUtensorMap ma, mb128, mb256;
    if (!make_map(&ma, A, uint64_t(K), uint64_t(M), uint64_t(K), BM) ||
        !make_map(&mb128, B, uint64_t(K), uint64_t(N), uint64_t(K), 128) ||
        !make_map(&mb256, B, uint64_t(K), uint64_t(N), uint64_t(K), 256))
        return fail(FWR_ERR_CUDA, "fwr_gemm_bf16_tc: tensor map encoding failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* st = nullptr;
    cudaError_t e = cudaMalloc(&st, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_gemm<float>(ma, mb128, mb256, M, N, K, D, N, st, s, wait_cycles);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(st);
    if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_gemm_bf16_tc");
    if (h) return fail(FWR_ERR_TIMEOUT, "fwr_gemm_bf16_tc: a pipeline wait ran out");
    return FWR_OK;
}

fwr_status fwr_linws_create(fwr_linws** out, const fwr_plan* plan, int rank, const float* A_host,
                            const float* V_host, int max_batch) {
    if (!out) return FWR_ERR_ARG;
    *out = nullptr;
    if (!plan || !A_host || !V_host) return fail(FWR_ERR_ARG, "fwr_linws_create: null argument");
    if (rank < 128 || rank % 128 != 0 || rank > 8192)
        return fail(FWR_ERR_ARG, "fwr_linws_create: rank must be a multiple of 128 in [128, 8192]");
    if (max_batch < 1 || max_batch > 65536)
        return fail(FWR_ERR_ARG, "fwr_linws_create: max_batch must be in [1, 65536]");
    if ((2LL * plan->N * plan->N) % 128 != 0)
        return fail(FWR_ERR_UNSUPPORTED, "fwr_linws_create: 2 N^2 must be a multiple of 128");
    fwr_linws* w = new (std::nothrow) fwr_linws();
    if (!w) return FWR_ERR_CUDA;
    w->n = plan->n;
    w->N = plan->N;
    w->rank = rank;
    w->max_batch = max_batch;
    w->cells2 = 2LL * plan->N * plan->N;
    cudaGetDevice(&w->device);
    w->mask = plan->h_mask;
    cudaError_t e = cudaSuccess;
    std::vector<int> cells;
    for (int i = 0; i < w->n * w->n; ++i)
        if (w->mask[i]) cells.push_back(i);
    w->nv = int(cells.size());
    w->K = 2 * w->nv;
    w->Kpad = (w->K + 63) / 64 * 64;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc(reinterpret_cast<void**>(&w->d_src), size_t(w->Kpad) * sizeof(int));
    alloc(reinterpret_cast<void**>(&w->X), size_t(max_batch) * w->Kpad * 2);
    alloc(reinterpret_cast<void**>(&w->C), size_t(max_batch) * rank * 2);
    alloc(reinterpret_cast<void**>(&w->At), size_t(rank) * w->Kpad * 2);
    alloc(reinterpret_cast<void**>(&w->V), size_t(w->cells2) * rank * 2);
    alloc(reinterpret_cast<void**>(&w->Eh), size_t(max_batch) * w->cells2 * 2);
    alloc(reinterpret_cast<void**>(&w->d_status), sizeof(int));
    std::vector<int> src(size_t(w->Kpad), -1);
    for (int j = 0; j < w->nv; ++j) {
        src[j] = cells[j];
        src[w->nv + j] = w->n * w->n + cells[j];
    }
    if (e == cudaSuccess) e = cudaMemcpy(w->d_src, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(w->At, 0, size_t(rank) * w->Kpad * 2);
    if (e == cudaSuccess) e = cudaMemset(w->d_status, 0, sizeof(int));
    // A [K][rank] -> At [rank][Kpad]; V [2 N^2][rank] as is
    if (e == cudaSuccess) e = upload_bf16(A_host, w->K, rank, true, w->Kpad, w->At);
    if (e == cudaSuccess) e = upload_bf16(V_host, int(w->cells2), rank, false, rank, w->V);
    if (e != cudaSuccess) {
        free_ws(w);
        return fwr::cuda_fail(e, "fwr_linws_create");
    }
    if (!make_map(&w->mX, w->X, uint64_t(w->Kpad), uint64_t(max_batch), uint64_t(w->Kpad), BM) ||
        !make_map(&w->mAt128, w->At, uint64_t(w->Kpad), uint64_t(rank), uint64_t(w->Kpad), 128) ||
        !make_map(&w->mAt256, w->At, uint64_t(w->Kpad), uint64_t(rank), uint64_t(w->Kpad), 256) ||
        !make_map(&w->mC, w->C, uint64_t(rank), uint64_t(max_batch), uint64_t(rank), BM) ||
        !make_map(&w->mV128, w->V, uint64_t(rank), uint64_t(w->cells2), uint64_t(rank), 128) ||
        !make_map(&w->mV256, w->V, uint64_t(rank), uint64_t(w->cells2), uint64_t(rank), 256)) {
        free_ws(w);
        return fail(FWR_ERR_CUDA, "fwr_linws_create: tensor map encoding failed");
    }
    *out = w;
    return FWR_OK;
}

void fwr_linws_destroy(fwr_linws* w) {
    if (w) free_ws(w);
}

int fwr_linws_valid_count(const fwr_linws* w) { return w ? w->nv : -1; }

}  // extern "C"

namespace {

// gather, X A, (X A) V^T -> out [F][2 N^2] (FP32 or BF16)
template <typename OutT>
cudaError_t run_ws(fwr_linws* w, const float* slopes, int F, OutT* out, cudaStream_t s) {
    k_gather<<<F, 256, 0, s>>>(slopes, reinterpret_cast<const int2*>(w->d_src), w->n * w->n, w->Kpad, w->X);
    cudaError_t e = cudaGetLastError();
    // the GEMMs are programmatic dependents of their producers (gather, X A)
    if (e == cudaSuccess)
        e = launch_gemm<__nv_bfloat16>(w->mX, w->mAt128, w->mAt256, F, w->rank, w->Kpad, w->C, w->rank, w->d_status,
                                       s, fwr::umma::WAIT_LIMIT, true);
    if (e == cudaSuccess)
        e = launch_gemm<OutT>(w->mC, w->mV128, w->mV256, F, w->cells2, w->rank, out, w->cells2, w->d_status, s,
                              fwr::umma::WAIT_LIMIT, true);
    return e;
}

}  // namespace

extern "C" {

fwr_status fwr_linws_forward(fwr_linws* w, const float* slopes_dev, int n_frames, float* ext_init_dev,
                             void* stream) {
    if (!w || n_frames < 0 || n_frames > w->max_batch) return FWR_ERR_ARG;
    if (n_frames == 0) return FWR_OK;
    if (!slopes_dev || !ext_init_dev || !aligned16(ext_init_dev))
        return fail(FWR_ERR_ARG, "fwr_linws_forward: null or unaligned pointer");
    const cudaError_t e = run_ws<float>(w, slopes_dev, n_frames, ext_init_dev, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_linws_forward");
}

fwr_status fwr_linws_reconstruct(fwr_linws* w, fwr_plan* plan, const float* slopes_dev, int n_frames, int iters,
                                 float* phase_dev, void* stream) {
    if (!w || !plan || n_frames < 0 || n_frames > w->max_batch || iters < 0 || iters > 64) return FWR_ERR_ARG;
    if (plan->n != w->n || plan->N != w->N || plan->h_mask != w->mask)
        return fail(FWR_ERR_ARG, "fwr_linws_reconstruct: the plan's pupil or grid differs from the warm start's");
    if (n_frames == 0) return FWR_OK;
    if (!slopes_dev || !phase_dev || !aligned16(phase_dev))
        return fail(FWR_ERR_ARG, "fwr_linws_reconstruct: null or unaligned pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = run_ws<__nv_bfloat16>(w, slopes_dev, n_frames, w->Eh, s);
    if (e == cudaSuccess)
        e = fwr::launch_warm_bf16(plan, slopes_dev, reinterpret_cast<const uint16_t*>(w->Eh), n_frames, iters,
                                  phase_dev, s, true);
    if (e == cudaErrorNotSupported)
        return fail(FWR_ERR_UNSUPPORTED, "fwr_linws_reconstruct: the plan does not take the fused path");
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_linws_reconstruct");
}

fwr_status fwr_linws_status(fwr_linws* w) {
    if (!w) return FWR_ERR_ARG;
    int h = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, w->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(w->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return fwr::cuda_fail(e, "fwr_linws_status");
    return h ? fail(FWR_ERR_TIMEOUT, "fwr_linws_forward: a pipeline wait ran out") : FWR_OK;
}

}  // extern "C"
