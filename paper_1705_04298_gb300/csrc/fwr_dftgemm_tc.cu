// Split-BF16 DFT-as-GEMM path for 64^2, 128^2 and 256^2 grids on the tcgen05 tensor
// cores: Algorithm 1 (Sec. 3.3) and the final reconstruction (Eqs. 2-3) with
// every 2-D DFT computed as dense products, Z <- F Z F with F[j][k] =
// e^{-2 i pi j k / N} (the conjugate for the inverse; no scaling: 1/N^2 is in
// the spectral weights).
//
// The frames of a chunk are the columns of two GEMMs per 2-D transform (D =
// A B^T, fwr_umma.cuh). A complex N x N product is one real 2N x 2N product:
// [Re; Im] <- [[Fr, -Fi], [Fi, Fr]] [Re; Im]. Every FP32 operand x is split
// into BF16 terms, and the products of the terms are one GEMM over K = 2N per
// product, FP32 accumulation in TMEM:
//   3 products (FWR_TRANSFORM_DFT_BF16X3): x = hi + lo (hi = bf16(x), lo =
//     bf16(x - hi)); hi hi + hi lo + lo hi over K = 6N with A = [Ah | Ah | Al]
//     and B rows [hi | lo | hi] (lo lo, about 2^-16 relative, dropped);
//   6 products (FWR_TRANSFORM_DFT_BF16X6): x = hi + mid + lo, each the BF16
//     rounding of what the previous terms leave; hh + hm + mh + hl + mm + lh
//     over K = 12N with A = [Ah | Ah | Am | Ah | Am | Al] and B rows
//     [h | m | h | l | m | h] (the dropped terms are about 2^-24 relative).
//     Measured against the FP64 oracle it gives the error of the three
//     products: the tensor core's FP32 accumulation over K sets the error.
//
// Per transform, with the chunk's frames f and row (or column) index x:
//   right product  B rows (f, r) = row r of Z_f        -> D [2N][(f, r)] = (Z_f F)^T
//   left product   B rows (f, i) = column i of Z_f F   -> D [2N][(f, k)] = F Z_f F
// so D's rows are output rows (real parts, then imaginary parts) and its
// columns run over frames and the other index. The right product's epilogue
// writes its result straight into the left product's operand, split into BF16
// terms (B row (f, i) = [Re D[i][(f, .)], Im D[N + i][(f, .)]]; no FP32 D in
// between). After the left products, element-wise kernels rebuild B from D:
// the spectral step (LSQ projection or final filter, with the y part of Eq.
// PC as a spectral correction; it needs the partner bins (-ky, -kx), which
// lie in other tiles) and, in direct space, reinsertion of the measured
// slopes and the x part of Eq. PC (row sums over whole rows).

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fwr_internal.h"

namespace fwr {

#include "fwr_fft.cuh"

namespace {

typedef __nv_bfloat16 bf16;

// frames per chunk: the chunk's GEMMs have 2^23 / N columns
__host__ __device__ inline int chunk_frames(int N) { return (1 << 23) / (N * N); }

// K of the GEMMs: 2N per product
__host__ __device__ inline int gemm_k(int N, int terms) { return 2 * N * terms; }

struct Ws {
    bf16* Af;  // [2N][K] forward operand
    bf16* Ai;  // [2N][K] inverse operand
    bf16* B;   // [chunk N][K]: operand of each transform's right product
    bf16* B2;  // [chunk N][K]: operand of its left product (the right product's split epilogue)
    float* D;  // [2N][chunk N]
};

Ws carve(int N, int terms, void* ws) {
    Ws w;
    uint8_t* p = static_cast<uint8_t*>(ws);
    const size_t K = size_t(gemm_k(N, terms));
    const size_t a = size_t(2 * N) * K * sizeof(bf16);
    const size_t cols = size_t(chunk_frames(N)) * N;
    const size_t b = cols * K * sizeof(bf16);
    w.Af = reinterpret_cast<bf16*>(p);
    w.Ai = reinterpret_cast<bf16*>(p + a);
    w.B = reinterpret_cast<bf16*>(p + 2 * a);
    w.B2 = reinterpret_cast<bf16*>(p + 2 * a + b);
    w.D = reinterpret_cast<float*>(p + 2 * a + 2 * b);
    return w;
}

__device__ __forceinline__ void split(float x, bf16& hi, bf16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
__device__ __forceinline__ void split3(float x, bf16& hi, bf16& mid, bf16& lo) {
    hi = __float2bfloat16_rn(x);
    const float r = x - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r);
    lo = __float2bfloat16_rn(r - __bfloat162float(mid));
}

// entry k of a B row: 3 products [hi | lo | hi] (K = 6N); 6 products
// [h | m | h | l | m | h] (K = 12N)
__device__ __forceinline__ void put_split(bf16* row, int N, int k, float x, int terms) {
    if (terms == 3) {
        bf16 h, l;
        split(x, h, l);
        row[k] = h;
        row[2 * N + k] = l;
        row[4 * N + k] = h;
    } else {
        bf16 h, m, l;
        split3(x, h, m, l);
        row[k] = h;
        row[2 * N + k] = m;
        row[4 * N + k] = h;
        row[6 * N + k] = l;
        row[8 * N + k] = m;
        row[10 * N + k] = h;
    }
}

// A operands from the twiddle table: forward [[Fr, -Fi], [Fi, Fr]], inverse
// with Fi -> -Fi; rows [Ah | Ah | Al] (3 products) or [Ah | Ah | Am | Ah | Am
// | Al] (6 products).
__device__ __forceinline__ void put_a(bf16* row, int N, int c, float v, int terms) {
    if (terms == 3) {
        bf16 h, l;
        split(v, h, l);
        row[c] = h;
        row[2 * N + c] = h;
        row[4 * N + c] = l;
    } else {
        bf16 h, m, l;
        split3(v, h, m, l);
        row[c] = h;
        row[2 * N + c] = h;
        row[4 * N + c] = m;
        row[6 * N + c] = h;
        row[8 * N + c] = m;
        row[10 * N + c] = l;
    }
}

__global__ void k_dg_operands(const float2* tw, int N, int terms, bf16* Af, bf16* Ai) {
    const int i = blockIdx.x;  // output row 0 .. 2N
    const size_t K = size_t(gemm_k(N, terms));
    for (int c = threadIdx.x; c < 2 * N; c += blockDim.x) {
        const int io = i % N, co = c % N;
        const float2 f = tw[(long long)io * co % N];  // (cos, -sin) of 2 pi io co / N
        const bool im_out = i >= N, im_in = c >= N;
        // forward: Re out = Fr Re - Fi Im, Im out = Fi Re + Fr Im (Fi = f.y)
        const float vf = im_out == im_in ? f.x : (im_out ? f.y : -f.y);
        const float vi = im_out == im_in ? f.x : (im_out ? -f.y : f.y);
        put_a(Af + (size_t)i * K, N, c, vf, terms);
        put_a(Ai + (size_t)i * K, N, c, vi, terms);
    }
}

// Direct-space rows -> B rows (f, r) of the right product. Source: the embed
// (first pass: measured slopes in the pupil, warm start or 0 outside) or D in
// the direct-space layout of the previous inverse (then the measured slopes
// are reinserted). Then the x part of Eq. PC when `fill`. One block of N / 2
// threads per row.
__global__ void k_dg_rows(const float* D, long long ldd, bool embed, const float* slopes, const float* ext,
                          const uint8_t* mask, int n, int off, int N, int f0, bool fill, bf16* B,
                          unsigned* status, int terms) {
    const int row = blockIdx.x;  // (f, r) in the chunk
    const int fl = row / N, r = row % N, f = f0 + fl;
    const int nn = n * n;
    const float* sl = slopes + (size_t)f * 2 * nn;
    __shared__ float red[32];
    float xs[2], ys[2];
    float part = 0.f;
    bool bad = false;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int c = threadIdx.x + u * (N / 2);
        float vx, vy;
        if (embed) {
            const float* e = ext ? ext + (size_t)f * 2 * N * N : nullptr;
            vx = e ? e[r * N + c] : 0.f;
            vy = e ? e[N * N + r * N + c] : 0.f;
        } else {
            vx = D[(size_t)r * ldd + (size_t)fl * N + c];
            vy = D[(size_t)(N + r) * ldd + (size_t)fl * N + c];
        }
        const int i = r - off, j = c - off;
        if (i >= 0 && i < n && j >= 0 && j < n && mask[i * n + j]) {
            vx = sl[i * n + j];
            vy = sl[nn + i * n + j];
            bad |= !(isfinite(vx) && isfinite(vy));
        }
        xs[u] = vx;
        ys[u] = vy;
        if (c != N - 1) part += vx;
    }
    if (embed && bad) atomicOr(status, STATUS_NONFINITE);
    if (fill) {
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == N / 2 - 1) {
            float s = 0.f;
            for (int w = 0; w < N / 64; ++w) s += red[w];
            xs[1] = -s;  // column N - 1 is this thread's second cell
        }
    }
    bf16* b = B + (size_t)row * gemm_k(N, terms);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int c = threadIdx.x + u * (N / 2);
        put_split(b, N, c, xs[u], terms);
        put_split(b, N, N + c, ys[u], terms);
    }
}

// Spectral step on Y_f[ky][kx] = D[ky][(f, kx)] + i D[N + ky][(f, kx)], the
// packed spectrum of sx + i sy; writes B rows (f, ky) of the inverse's right
// product. Non-final: LSQ projection (Algorithm 1 steps 2-3); final: the
// filter of Eq. 2 (weights wfin). Both read the half-tables (rows ky <=
// N / 2, the rest from (-ky, -kx)) that hold 1/N^2. With `fill`, the y part
// of Eq. PC: Sy(ky, kx) -= Sy(0, kx) e^{2 i pi ky / N}.
__global__ void k_dg_spectral(const float* D, long long ldd, int N, const Tables<float> tab, bool final, bool fill,
                              bf16* B, int terms) {
    const int row = blockIdx.x;  // (f, ky)
    const int fl = row / N, ky = row % N, kyn = (N - ky) & (N - 1);
    const float* wt = final ? tab.wfin : tab.iota;
    bf16* b = B + (size_t)row * gemm_k(N, terms);
    const size_t cb = (size_t)fl * N;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int kx = threadIdx.x + u * (N / 2), kxn = (N - kx) & (N - 1);
        const float2 z1 = make_float2(D[(size_t)ky * ldd + cb + kx], D[(size_t)(N + ky) * ldd + cb + kx]);
        const float2 z2 = make_float2(D[(size_t)kyn * ldd + cb + kxn], D[(size_t)(N + kyn) * ldd + cb + kxn]);
        float2 sx = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
        float2 sy = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
        if (fill) {
            const float2 e0 = make_float2(D[cb + kx], D[(size_t)N * ldd + cb + kx]);
            const float2 e1 = make_float2(D[cb + kxn], D[(size_t)N * ldd + cb + kxn]);
            const float2 ey = make_float2(0.5f * (e0.y + e1.y), 0.5f * (e1.x - e0.x));
            const float2 t = tab.tw[ky];
            const float2 c = cmul(ey, make_float2(t.x, -t.y));
            sy = make_float2(sy.x - c.x, sy.y - c.y);
        }
        const float2 gx = cmul(tab.A[kx], tab.Tt[ky]);
        const float2 gy = cmul(tab.Tt[kx], tab.A[ky]);
        const float w = ky <= N / 2 ? wt[ky * N + kx] : wt[kyn * N + kxn];
        float2 ph = cadd(cmulc(gx, sx), cmulc(gy, sy));
        ph = make_float2(ph.x * w, ph.y * w);
        float2 out;
        if (!final) {
            const float2 ox = cmul(gx, ph), oy = cmul(gy, ph);
            out = make_float2(ox.x - oy.y, ox.y + oy.x);
        } else {
            out = ph;
        }
        put_split(b, N, kx, out.x, terms);
        put_split(b, N, N + kx, out.y, terms);
    }
}

// real phase of the chunk's frames out of the direct-space D
__global__ void k_dg_phase(const float* D, long long ldd, int N, int f0, int nf, float* phase) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nf * N * N) return;
    const int fl = int(i / ((long long)N * N)), rc = int(i % ((long long)N * N)), r = rc / N, c = rc % N;
    phase[(size_t)(f0 + fl) * N * N + rc] = D[(size_t)r * ldd + (size_t)fl * N + c];
}

}  // namespace

size_t dftgemm_ws_bytes(int N, int terms) {
    if ((N != 64 && N != 128 && N != 256) || (terms != 3 && terms != 6)) return 0;
    const size_t cols = size_t(chunk_frames(N)) * N, K = size_t(gemm_k(N, terms));
    return 2 * size_t(2 * N) * K * sizeof(bf16) + 2 * cols * K * sizeof(bf16) + size_t(2 * N) * cols * sizeof(float);
}

int dftgemm_chunk(int N) { return chunk_frames(N); }

cudaError_t dftgemm_setup(int N, int terms, const float2* tw, void* ws) {
    Ws w = carve(N, terms, ws);
    k_dg_operands<<<2 * N, 256>>>(tw, N, terms, w.Af, w.Ai);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? cudaDeviceSynchronize() : e;
}

cudaError_t launch_dftgemm_f32(int N, int terms, const Params<float>& p, void* ws, cudaStream_t s) {
    if ((N != 64 && N != 128 && N != 256) || (terms != 3 && terms != 6) || !ws) return cudaErrorInvalidValue;
    const Ws w = carve(N, terms, ws);
    const int K = gemm_k(N, terms);
    const int chunk = chunk_frames(N);
    const long long ldd = (long long)chunk * N;
    int* st = reinterpret_cast<int*>(p.status);
    for (int f0 = 0; f0 < p.F; f0 += chunk) {
        const int nf = p.F - f0 < chunk ? p.F - f0 : chunk;
        // GEMM columns: whole frames, rounded up to a multiple of 128 (at 64^2
        // an odd frame count adds one frame's columns, whose B rows hold stale
        // values: each output column depends on its own B row only, and no
        // kernel reads those columns back)
        const long long cols = ((long long)nf * N + 127) / 128 * 128;
        for (int it = 0; it <= p.iters; ++it) {
            const bool final = it == p.iters;
            const bool fill = p.periodic == PERIODIC_BEFORE_EACH_FFT || (p.periodic == PERIODIC_FINAL_ONLY && final);
            k_dg_rows<<<nf * N, N / 2, 0, s>>>(w.D, ldd, it == 0, p.slopes, p.ext_init, p.mask, p.n, p.off, N, f0,
                                               fill, w.B, p.status, terms);
            cudaError_t e = cudaGetLastError();
            // forward transform: right product (its epilogue splits the result
            // into the left product's operand B2), left product
            if (e == cudaSuccess) e = tc_gemm_split(w.Af, 2 * N, K, w.B, cols, w.B2, N, K, terms, st, s);
            if (e == cudaSuccess) e = tc_gemm(w.Af, 2 * N, K, w.B2, cols, w.D, false, ldd, st, s);
            if (e == cudaSuccess) {
                k_dg_spectral<<<nf * N, N / 2, 0, s>>>(w.D, ldd, N, p.tab, final, fill, w.B, terms);
                e = cudaGetLastError();
            }
            // inverse transform
            if (e == cudaSuccess) e = tc_gemm_split(w.Ai, 2 * N, K, w.B, cols, w.B2, N, K, terms, st, s);
            if (e == cudaSuccess) e = tc_gemm(w.Ai, 2 * N, K, w.B2, cols, w.D, false, ldd, st, s);
            if (e != cudaSuccess) return e;
        }
        if (p.phase) {
            const long long tot = (long long)nf * N * N;
            k_dg_phase<<<unsigned((tot + 255) / 256), 256, 0, s>>>(w.D, ldd, N, f0, nf, p.phase);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace fwr
