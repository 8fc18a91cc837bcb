// Generic fused Gerchberg kernel for sm_103a (fallback for pupils too large for
// the shared-memory layout of fwr_fused.cu, and the FFT test entry).
//
// One CTA owns one frame at a time and keeps the frame's whole N x N complex
// grid Z = sx + i sy in shared memory for all iterations of Algorithm 1
// (Sec. 3.3) and for the final reconstruction (Eqs. 2-3); HBM is touched only
// to read the measured slopes and to write the phase. The CTA then moves on
// to frame blockIdx.x + gridDim.x (persistent grid sized to the SMs).
//
// 2-D FFT: a 1-D transform of length N = R1 * R2 is two register passes
// (Cooley-Tukey four-step): pass A does R1-point DFTs on elements R2 apart
// and applies the twiddles w_N^(n2 k1) in place; pass B does R2-point DFTs on
// contiguous groups and writes natural order. The grid's row stride is N + 1
// (odd), so a warp that walks 32 consecutive rows or 32 consecutive columns
// hits distinct banks. Rows and columns use the same code with the strides
// swapped.
//
// Packing: both slope fields go through one complex FFT; the spectral step
// visits each (k, -k) pair once, unpacks Sx, Sy, applies the LSQ projection
// of Sec. 3.3 (phi = (Gx* Sx + Gy* Sy) / |G|^2, S' = G phi) and repacks.

#include <cuda_runtime.h>
#include <stdint.h>

#include "fwr_internal.h"

namespace fwr {

#include "fwr_fft.cuh"
#include "fwr_dftgemm.cuh"

template <int N> struct Split;
template <> struct Split<16> { static constexpr int R1 = 4, R2 = 4, NT = 64; };
template <> struct Split<32> { static constexpr int R1 = 8, R2 = 4, NT = 128; };
template <> struct Split<64> { static constexpr int R1 = 8, R2 = 8, NT = 256; };
template <> struct Split<128> { static constexpr int R1 = 16, R2 = 8, NT = 512; };

// ---------------------------------------------------------------------------
// 1-D passes over all N lines of the grid. ROWS: lines are rows (elements
// contiguous); otherwise lines are columns (elements S apart).
// ---------------------------------------------------------------------------
template <int N, int NT, bool INV, bool ROWS, typename V>
__device__ __forceinline__ void fft_pass_a(V* Z, const V* tw) {
    constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2, S = N + 1;
    constexpr int LS = ROWS ? S : 1, PS = ROWS ? 1 : S;
    constexpr int TASKS = N * R2;
    static_assert(TASKS % NT == 0, "pass A tasks must divide evenly");
#pragma unroll
    for (int i = 0; i < TASKS / NT; ++i) {
        const int t = threadIdx.x + i * NT;
        const int line = t % N, n2 = t / N;
        V* base = Z + line * LS + n2 * PS;
        V x[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) x[n1] = base[n1 * R2 * PS];
        dft_reg<R1, INV>(x);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            V w = tw[n2 * k1];
            if (INV) w.y = -w.y;
            x[k1] = cmul(x[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) base[k1 * R2 * PS] = x[k1];
    }
}

template <int N, int NT, bool INV, bool ROWS, typename V>
__device__ __forceinline__ void fft_pass_b(V* Z) {
    constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2, S = N + 1;
    constexpr int LS = ROWS ? S : 1, PS = ROWS ? 1 : S;
    constexpr int TASKS = N * R1;
    static_assert(TASKS % NT == 0, "pass B tasks must divide evenly");
    constexpr int PER = TASKS / NT;
    V y[PER][R2];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = threadIdx.x + i * NT;
        const int line = t % N, k1 = t / N;
        const V* base = Z + line * LS + (R2 * k1) * PS;
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) y[i][n2] = base[n2 * PS];
        dft_reg<R2, INV>(y[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = threadIdx.x + i * NT;
        const int line = t % N, k1 = t / N;
        V* base = Z + line * LS + k1 * PS;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) base[(R1 * k2) * PS] = y[i][k2];
    }
}

// Full 2-D transform in place; ends with a barrier.
template <int N, int NT, bool INV, typename V>
__device__ __forceinline__ void fft2(V* Z, const V* tw) {
    fft_pass_a<N, NT, INV, true>(Z, tw);
    __syncthreads();
    fft_pass_b<N, NT, INV, true>(Z);
    __syncthreads();
    fft_pass_a<N, NT, INV, false>(Z, tw);
    __syncthreads();
    fft_pass_b<N, NT, INV, false>(Z);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Spectral steps. Pairs (k, -k): rows ky = 1 .. N/2-1 with every kx, plus
// rows 0 and N/2 with kx = 0 .. N/2 (their partners lie in the same row).
// FINAL = false: LSQ projection onto range(G) (Algorithm 1 step 2).
// FINAL = true : phi = R_x Sx + R_y Sy (Eq. 2) with R = G* wfin (Eq. 3),
//                stored as a Hermitian spectrum.
// ---------------------------------------------------------------------------
template <int N, int NT, bool FINAL, typename T, typename V>
__device__ __forceinline__ void spectral(V* Z, const V* A, const V* Tt, const T* wtab) {
    constexpr int S = N + 1, H = N / 2;
    constexpr int NP = (H - 1) * N + 2 * (H + 1);
    const T half = T(0.5);
    for (int p = threadIdx.x; p < NP; p += NT) {
        int ky, kx;
        if (p < (H - 1) * N) {
            ky = 1 + p / N;
            kx = p % N;
        } else {
            const int q = p - (H - 1) * N;
            ky = (q <= H) ? 0 : H;
            kx = (q <= H) ? q : q - (H + 1);
        }
        const int my = (N - ky) & (N - 1), mx = (N - kx) & (N - 1);
        const V z1 = Z[ky * S + kx], z2 = Z[my * S + mx];
        // Sx = (z1 + conj z2) / 2, Sy = (z1 - conj z2) / (2i)
        const V sx = mk(half * (z1.x + z2.x), half * (z1.y - z2.y));
        const V sy = mk(half * (z1.y + z2.y), half * (z2.x - z1.x));
        const V gx = cmul(A[kx], Tt[ky]);
        const V gy = cmul(Tt[kx], A[ky]);
        const T w = wtab[ky * N + kx];
        V ph = cadd(cmulc(gx, sx), cmulc(gy, sy));
        ph = mk(ph.x * w, ph.y * w);
        if (!FINAL) {
            const V ox = cmul(gx, ph), oy = cmul(gy, ph);
            Z[my * S + mx] = mk(ox.x + oy.y, oy.x - ox.y);  // conj(ox) + i conj(oy)
            Z[ky * S + kx] = mk(ox.x - oy.y, ox.y + oy.x);  // ox + i oy
        } else {
            Z[my * S + mx] = mk(ph.x, -ph.y);
            Z[ky * S + kx] = ph;
        }
    }
}


// Eq. PC: Z.x[m][N-1] = -sum_{c<N-1} Z.x[m][c]; Z.y[N-1][c] = -sum_{m<N-1} Z.y[m][c].
// The x and y fills touch different components, so they run together.
template <int N, int NT, typename T, typename V>
__device__ __forceinline__ void periodic_fill(V* Z) {
    constexpr int S = N + 1, NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = warp; r < N; r += NW) {
        T s = T(0);
        for (int c = lane; c < N - 1; c += 32) s += Z[r * S + c].x;
        s = warp_sum(s);
        if (lane == 0) Z[r * S + N - 1].x = -s;
    }
    for (int c = warp; c < N; c += NW) {
        T s = T(0);
        for (int r = lane; r < N - 1; r += 32) s += Z[r * S + c].y;
        s = warp_sum(s);
        if (lane == 0) Z[(N - 1) * S + c].y = -s;
    }
}

// Algorithm 1 step 4: the measured slopes replace the grid inside the pupil.
template <int N, int NT, typename T, typename V>
__device__ __forceinline__ bool reinsert(V* Z, const uint8_t* mask, const T* sl, int n, int off) {
    constexpr int S = N + 1;
    const int nn = n * n;
    bool finite = true;
    for (int c = threadIdx.x; c < nn; c += NT) {
        if (mask[c]) {
            const int i = c / n, j = c - i * n;
            const T vx = sl[c], vy = sl[nn + c];
            finite &= isfinite(vx) && isfinite(vy);
            Z[(off + i) * S + off + j] = mk(vx, vy);
        }
    }
    return finite;
}

template <typename T> __host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, int N>
__host__ __device__ constexpr size_t smem_layout_bytes(int n) {
    typedef typename cvec<T>::type V;
    return align16<T>(size_t(N) * (N + 1) * sizeof(V) + 3 * size_t(N) * sizeof(V) +
                      2 * size_t(N / 2 + 1) * N * sizeof(T)) +
           align16<T>(size_t(n) * n);
}

// extra shared memory of the DFT-GEMM transforms: 4 N^2 split operands and
// the 6 N^2 split DFT matrix, BF16
template <int N> __host__ __device__ constexpr size_t gemm_extra_bytes() { return size_t(10) * N * N * 2; }

// 2-D transform of the generic kernel: the shared-memory FFT, or (GEMM) the
// split-BF16 tensor-core DFT. Both end with a barrier.
template <int N, int NT, bool INV, bool GEMM, typename V>
__device__ __forceinline__ void transform2(V* Z, const V* tw, bf16_t* xb, const bf16_t* Fm) {
    if constexpr (GEMM) dft2_gemm<N, NT, INV>(Z, N + 1, xb, Fm);
    else fft2<N, NT, INV>(Z, tw);
}

template <typename T, int N, bool GEMM>
__global__ void __launch_bounds__(Split<N>::NT)
basic_kernel(Params<T> p) {
    typedef typename cvec<T>::type V;
    constexpr int NT = Split<N>::NT, S = N + 1, H = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* Z = reinterpret_cast<V*>(smem_raw);
    V* tw = Z + N * S;
    V* A = tw + N;
    V* Tt = A + N;
    T* iota = reinterpret_cast<T*>(Tt + N);
    T* wfin = iota + (H + 1) * N;
    uint8_t* mask = reinterpret_cast<uint8_t*>(smem_raw) +
                    align16<T>(size_t(N) * S * sizeof(V) + 3 * size_t(N) * sizeof(V) +
                               2 * size_t(H + 1) * N * sizeof(T));
    bf16_t* xb = reinterpret_cast<bf16_t*>(smem_raw + smem_layout_bytes<T, N>(p.n));
    bf16_t* Fm = xb + 4 * N * N;
    __shared__ int s_bad;

    const int n = p.n, off = p.off, nn = n * n;
    for (int i = threadIdx.x; i < N; i += NT) {
        tw[i] = p.tab.tw[i];
        A[i] = p.tab.A[i];
        Tt[i] = p.tab.Tt[i];
    }
    for (int i = threadIdx.x; i < (H + 1) * N; i += NT) {
        iota[i] = p.tab.iota[i];
        wfin[i] = p.tab.wfin[i];
    }
    for (int i = threadIdx.x; i < nn; i += NT) mask[i] = p.mask[i];
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    if constexpr (GEMM) {
        dft_matrix_split<N, NT>(Fm, tw);
        __syncthreads();
    }

    bool finite = true;
    for (int f = blockIdx.x; f < p.F; f += gridDim.x) {
        const T* sl = p.slopes + size_t(f) * 2 * nn;
        // embed: initial extension (zero or the caller's warm start) ...
        const T* ext = p.ext_init ? p.ext_init + size_t(f) * 2 * N * N : nullptr;
        for (int idx = threadIdx.x; idx < N * N; idx += NT) {
            const int m = idx / N, c = idx % N;
            Z[m * S + c] = ext ? mk(ext[idx], ext[N * N + idx]) : mk(T(0), T(0));
        }
        __syncthreads();
        // ... and the measurement inside the pupil
        finite &= reinsert<N, NT>(Z, mask, sl, n, off);
        __syncthreads();

        for (int it = 0; it < p.iters; ++it) {
            if (p.periodic == PERIODIC_BEFORE_EACH_FFT) {
                periodic_fill<N, NT, T>(Z);
                __syncthreads();
            }
            transform2<N, NT, false, GEMM>(Z, tw, xb, Fm);
            spectral<N, NT, false, T>(Z, A, Tt, iota);
            __syncthreads();
            transform2<N, NT, true, GEMM>(Z, tw, xb, Fm);
            reinsert<N, NT>(Z, mask, sl, n, off);
            __syncthreads();
        }
        if (p.periodic != PERIODIC_NONE) {
            periodic_fill<N, NT, T>(Z);
            __syncthreads();
        }
        if (p.ext_out) {
            T* eo = p.ext_out + size_t(f) * 2 * N * N;
            for (int idx = threadIdx.x; idx < N * N; idx += NT) {
                const V z = Z[(idx / N) * S + idx % N];
                eo[idx] = z.x;
                eo[N * N + idx] = z.y;
            }
            __syncthreads();
        }
        if (p.phase) {
            transform2<N, NT, false, GEMM>(Z, tw, xb, Fm);
            spectral<N, NT, true, T>(Z, A, Tt, wfin);
            __syncthreads();
            transform2<N, NT, true, GEMM>(Z, tw, xb, Fm);
            T* ph = p.phase + size_t(f) * N * N;
            for (int idx = threadIdx.x; idx < N * N; idx += NT) ph[idx] = Z[(idx / N) * S + idx % N].x;
        }
        __syncthreads();
    }
    if (!finite) atomicOr(&s_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(p.status, STATUS_NONFINITE);
}

size_t basic_smem_bytes(int N, int elem_bytes, int n) {
    const bool d = elem_bytes == 8;
    switch (N) {
        case 16: return d ? smem_layout_bytes<double, 16>(n) : smem_layout_bytes<float, 16>(n);
        case 32: return d ? smem_layout_bytes<double, 32>(n) : smem_layout_bytes<float, 32>(n);
        case 64: return d ? smem_layout_bytes<double, 64>(n) : smem_layout_bytes<float, 64>(n);
        case 128: return d ? smem_layout_bytes<double, 128>(n) : smem_layout_bytes<float, 128>(n);
        default: return 0;
    }
}

template <typename T, int N, bool GEMM = false>
static cudaError_t launch_one(const Params<T>& p, cudaStream_t s) {
    constexpr int NT = Split<N>::NT;
    const size_t smem = smem_layout_bytes<T, N>(p.n) + (GEMM ? gemm_extra_bytes<N>() : 0);
    auto kern = basic_kernel<T, N, GEMM>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * per_sm;
    if (p.ctas > 0 && p.ctas < grid) grid = p.ctas;
    if (grid > p.F) grid = p.F;
    kern<<<grid, NT, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_basic_f32(int N, const Params<float>& p, cudaStream_t s) {
    switch (N) {
        case 16: return launch_one<float, 16>(p, s);
        case 32: return launch_one<float, 32>(p, s);
        case 64: return launch_one<float, 64>(p, s);
        case 128: return launch_one<float, 128>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_basic_f64(int N, const Params<double>& p, cudaStream_t s) {
    switch (N) {
        case 16: return launch_one<double, 16>(p, s);
        case 32: return launch_one<double, 32>(p, s);
        case 64: return launch_one<double, 64>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_basic_gemm_f32(int N, const Params<float>& p, cudaStream_t s) {
    switch (N) {
        case 32: return launch_one<float, 32, true>(p, s);
        case 64: return launch_one<float, 64, true>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

// Standalone batched 2-D DFT through the split-BF16 tensor-core products (test entry).
template <int N, bool INV>
__global__ void __launch_bounds__(Split<N>::NT)
dft2_gemm_kernel(const float2* in, float2* out, int F, const float2* twg) {
    constexpr int NT = Split<N>::NT, S = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* Z = reinterpret_cast<float2*>(smem_raw);
    float2* tw = Z + N * S;
    bf16_t* xb = reinterpret_cast<bf16_t*>(smem_raw + align16<float>(size_t(N) * S * 8 + size_t(N) * 8));
    bf16_t* Fm = xb + 4 * N * N;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = twg[i];
    __syncthreads();
    dft_matrix_split<N, NT>(Fm, tw);
    for (int f = blockIdx.x; f < F; f += gridDim.x) {
        const float2* src = in + size_t(f) * N * N;
        for (int idx = threadIdx.x; idx < N * N; idx += NT) Z[(idx / N) * S + idx % N] = src[idx];
        __syncthreads();
        dft2_gemm<N, NT, INV>(Z, S, xb, Fm);
        float2* dst = out + size_t(f) * N * N;
        for (int idx = threadIdx.x; idx < N * N; idx += NT) dst[idx] = Z[(idx / N) * S + idx % N];
        __syncthreads();
    }
}

template <int N>
static cudaError_t launch_dft2_gemm_n(const float2* in, float2* out, int F, int inverse, const float2* tw,
                                      cudaStream_t s) {
    const size_t smem = align16<float>(size_t(N) * (N + 1) * 8 + size_t(N) * 8) + gemm_extra_bytes<N>();
    auto kern = inverse ? dft2_gemm_kernel<N, true> : dft2_gemm_kernel<N, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int grid = F < 4 * sms ? F : 4 * sms;
    kern<<<grid, Split<N>::NT, smem, s>>>(in, out, F, tw);
    return cudaGetLastError();
}

cudaError_t launch_dft2_gemm_f32(int N, const float2* in, float2* out, int F, int inverse, const float2* tw,
                                 cudaStream_t s) {
    switch (N) {
        case 32: return launch_dft2_gemm_n<32>(in, out, F, inverse, tw, s);
        case 64: return launch_dft2_gemm_n<64>(in, out, F, inverse, tw, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fwr
