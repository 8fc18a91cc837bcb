// Gerchberg kernel for grids of any even size 16 <= N <= 64 (sm_103a): the
// paper's small windows, where the pupil of n lenslets is padded by w cells
// on each side (N = n + 2w, e.g. 46 and 52 for 40 lenslets with w = 3 and 6,
// Sec. 4.1) instead of to a power of two.
//
// One CTA owns one frame at a time; the whole N x N packed grid Z = sx + i sy
// stays in shared memory for every iteration of Algorithm 1 (Sec. 3.3) and
// the final reconstruction (Eqs. 2-3), as in the power-of-two kernels. The
// 1-D transforms are direct DFTs: output k of a line is
//   X[k] = sum_n x[n] w^(n k mod N),  w = e^{-2 i pi / N}  (e^{+} inverse),
// with w^j from an FP64-built table in shared memory and the index n k mod N
// advanced exactly in integers (no recurrence error). A warp takes one line
// at a time: its lanes hold outputs k = lane and lane + 32, and every input
// x[n] is one broadcast shared-memory read for the whole warp. Rows go from Z
// into a second grid Y, columns from Y back into Z.
//
// The spectral step visits each (k, -k) pair once (partners (N - k) mod N),
// unpacks Sx, Sy, applies the LSQ projection of Sec. 3.3 inside the loop and
// the final filter (Eq. 2) at the end; Eq. PC and the reinsertion are the
// same element-wise steps as in the other kernels.

#include <cuda_runtime.h>
#include <stdint.h>

#include "fwr_internal.h"

namespace fwr {

#include "fwr_fft.cuh"

namespace {

constexpr int AG_NT = 256;  // threads per CTA (8 warps)

template <typename T> struct AgLayout {
    typedef typename cvec<T>::type V;
    // Z and Y: N x (N + 1) cells each; tw, A, Tt: N cells; iota, wfin:
    // (N/2 + 1) x N weights; the mask: n x n bytes
    __host__ __device__ static size_t grid_bytes(int N) { return size_t(N) * (N + 1) * sizeof(V); }
    __host__ __device__ static size_t bytes(int N, int n) {
        return 2 * grid_bytes(N) + 3 * size_t(N) * sizeof(V) + 2 * size_t(N / 2 + 1) * N * sizeof(T) +
               ((size_t(n) * n + 15) & ~size_t(15));
    }
};

// One direct-DFT pass over all N lines: dst line l = DFT of src line l.
// ROWS: lines are rows (elements contiguous), else columns (elements S apart).
template <bool INV, bool ROWS, typename V>
__device__ __forceinline__ void dft_lines(const V* __restrict__ src, V* __restrict__ dst, const V* tw, int N) {
    typedef decltype(V().x) T;
    const int S = N + 1, LS = ROWS ? S : 1, PS = ROWS ? 1 : S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k1 = lane, k2 = lane + 32;
    const bool has2 = k2 < N;
    for (int l = warp; l < N; l += AG_NT / 32) {
        if (k1 >= N) break;  // N >= 16: lanes N .. 31 of a short line idle (N < 32 only)
        const V* x = src + l * LS;
        V acc1 = mk(T(0), T(0)), acc2 = acc1;
        int i1 = 0, i2 = 0;  // n k mod N for the two outputs
        for (int n = 0; n < N; ++n) {
            const V v = x[n * PS];
            V w1 = tw[i1];
            if (INV) w1.y = -w1.y;
            acc1 = mk(fmadd(v.x, w1.x, fmadd(-v.y, w1.y, acc1.x)), fmadd(v.x, w1.y, fmadd(v.y, w1.x, acc1.y)));
            i1 += k1;
            if (i1 >= N) i1 -= N;
            if (has2) {
                V w2 = tw[i2];
                if (INV) w2.y = -w2.y;
                acc2 = mk(fmadd(v.x, w2.x, fmadd(-v.y, w2.y, acc2.x)), fmadd(v.x, w2.y, fmadd(v.y, w2.x, acc2.y)));
                i2 += k2 - N;  // k2 - N in [-N, 0): one correction keeps i2 in range
                if (i2 < 0) i2 += N;
            }
        }
        V* y = dst + l * LS;
        y[k1 * PS] = acc1;
        if (has2) y[k2 * PS] = acc2;
    }
}

// 2-D transform Z -> Z through Y; ends with a barrier.
template <bool INV, typename V>
__device__ __forceinline__ void dft2_any(V* Z, V* Y, const V* tw, int N) {
    dft_lines<INV, true>(Z, Y, tw, N);
    __syncthreads();
    dft_lines<INV, false>(Y, Z, tw, N);
    __syncthreads();
}

// Spectral step over the (k, -k) pairs: rows ky = 1 .. N/2 - 1 with every kx,
// and rows 0 and N/2 with kx = 0 .. N/2 (their partners lie in the same row).
template <bool FINAL, typename T, typename V>
__device__ __forceinline__ void spectral_any(V* Z, const V* A, const V* Tt, const T* wtab, int N) {
    const int S = N + 1, H = N / 2;
    const int NP = (H - 1) * N + 2 * (H + 1);
    const T half = T(0.5);
    for (int p = threadIdx.x; p < NP; p += AG_NT) {
        int ky, kx;
        if (p < (H - 1) * N) {
            ky = 1 + p / N;
            kx = p % N;
        } else {
            const int q = p - (H - 1) * N;
            ky = (q <= H) ? 0 : H;
            kx = (q <= H) ? q : q - (H + 1);
        }
        const int my = ky == 0 ? 0 : N - ky, mx = kx == 0 ? 0 : N - kx;
        const V z1 = Z[ky * S + kx], z2 = Z[my * S + mx];
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

// Eq. PC on the packed grid (x and y parts touch different components)
template <typename T, typename V>
__device__ __forceinline__ void fill_any(V* Z, int N) {
    const int S = N + 1, NW = AG_NT / 32;
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

template <typename T, typename V>
__device__ __forceinline__ bool reinsert_any(V* Z, const uint8_t* mask, const T* sl, int n, int off, int N) {
    const int S = N + 1, nn = n * n;
    bool finite = true;
    for (int c = threadIdx.x; c < nn; c += AG_NT) {
        if (mask[c]) {
            const int i = c / n, j = c - i * n;
            const T vx = sl[c], vy = sl[nn + c];
            finite &= isfinite(vx) && isfinite(vy);
            Z[(off + i) * S + off + j] = mk(vx, vy);
        }
    }
    return finite;
}

template <typename T>
__global__ void __launch_bounds__(AG_NT) anygrid_kernel(Params<T> p, int N) {
    typedef typename cvec<T>::type V;
    const int S = N + 1, H = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* Z = reinterpret_cast<V*>(smem_raw);
    V* Y = Z + N * S;
    V* tw = Y + N * S;
    V* A = tw + N;
    V* Tt = A + N;
    T* iota = reinterpret_cast<T*>(Tt + N);
    T* wfin = iota + (H + 1) * N;
    uint8_t* mask = reinterpret_cast<uint8_t*>(wfin + (H + 1) * N);
    __shared__ int s_bad;

    const int n = p.n, off = p.off, nn = n * n;
    for (int i = threadIdx.x; i < N; i += AG_NT) {
        tw[i] = p.tab.tw[i];
        A[i] = p.tab.A[i];
        Tt[i] = p.tab.Tt[i];
    }
    for (int i = threadIdx.x; i < (H + 1) * N; i += AG_NT) {
        iota[i] = p.tab.iota[i];
        wfin[i] = p.tab.wfin[i];
    }
    for (int i = threadIdx.x; i < nn; i += AG_NT) mask[i] = p.mask[i];
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();

    bool finite = true;
    for (int f = blockIdx.x; f < p.F; f += gridDim.x) {
        const T* sl = p.slopes + size_t(f) * 2 * nn;
        const T* ext = p.ext_init ? p.ext_init + size_t(f) * 2 * N * N : nullptr;
        for (int idx = threadIdx.x; idx < N * N; idx += AG_NT) {
            const int m = idx / N, c = idx - m * N;
            Z[m * S + c] = ext ? mk(ext[idx], ext[N * N + idx]) : mk(T(0), T(0));
        }
        __syncthreads();
        finite &= reinsert_any<T>(Z, mask, sl, n, off, N);
        __syncthreads();
        for (int it = 0; it < p.iters; ++it) {
            if (p.periodic == PERIODIC_BEFORE_EACH_FFT) {
                fill_any<T>(Z, N);
                __syncthreads();
            }
            dft2_any<false>(Z, Y, tw, N);
            spectral_any<false, T>(Z, A, Tt, iota, N);
            __syncthreads();
            dft2_any<true>(Z, Y, tw, N);
            reinsert_any<T>(Z, mask, sl, n, off, N);
            __syncthreads();
        }
        if (p.periodic != PERIODIC_NONE) {
            fill_any<T>(Z, N);
            __syncthreads();
        }
        if (p.ext_out) {
            T* eo = p.ext_out + size_t(f) * 2 * N * N;
            for (int idx = threadIdx.x; idx < N * N; idx += AG_NT) {
                const V z = Z[(idx / N) * S + idx % N];
                eo[idx] = z.x;
                eo[N * N + idx] = z.y;
            }
            __syncthreads();
        }
        if (p.phase) {
            dft2_any<false>(Z, Y, tw, N);
            spectral_any<true, T>(Z, A, Tt, wfin, N);
            __syncthreads();
            dft2_any<true>(Z, Y, tw, N);
            T* ph = p.phase + size_t(f) * N * N;
            for (int idx = threadIdx.x; idx < N * N; idx += AG_NT) ph[idx] = Z[(idx / N) * S + idx % N].x;
        }
        __syncthreads();
    }
    if (!finite) atomicOr(&s_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(p.status, STATUS_NONFINITE);
}

template <typename T>
cudaError_t launch_any(int N, const Params<T>& p, cudaStream_t s) {
    if (N < 16 || N > 64 || (N & 1)) return cudaErrorInvalidValue;
    const size_t smem = AgLayout<T>::bytes(N, p.n);
    auto kern = anygrid_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, AG_NT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * per_sm;
    if (p.ctas > 0 && p.ctas < grid) grid = p.ctas;
    if (grid > p.F) grid = p.F;
    kern<<<grid, AG_NT, smem, s>>>(p, N);
    return cudaGetLastError();
}

}  // namespace

size_t anygrid_smem_bytes(int N, int elem_bytes, int n) {
    return elem_bytes == 8 ? AgLayout<double>::bytes(N, n) : AgLayout<float>::bytes(N, n);
}

cudaError_t launch_anygrid_f32(int N, const Params<float>& p, cudaStream_t s) { return launch_any<float>(N, p, s); }
cudaError_t launch_anygrid_f64(int N, const Params<double>& p, cudaStream_t s) { return launch_any<double>(N, p, s); }

}  // namespace fwr
