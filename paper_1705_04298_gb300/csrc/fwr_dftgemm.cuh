// 2-D DFT of an N x N complex grid as two dense complex matrix products on the
// tensor cores, Z <- F Z F with F[j][k] = e^{-2 i pi j k / N} = C - i S (the
// conjugate for the inverse), with split-BF16 operands: every FP32 operand x
// is held as hi + lo, hi = bf16(x), lo = bf16(x - hi), and a product is taken
// as hi*hi + hi*lo + lo*hi (the lo*lo term, about 2^-16 relative, dropped),
// accumulated in FP32 by mma.sync.m16n8k16 (BF16 in, FP32 out).
// Included inside namespace fwr after fwr_fft.cuh; N in {32, 64}.
#pragma once

#include <cuda_bf16.h>

namespace {

typedef __nv_bfloat16 bf16_t;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const bf16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragment (16 x 16, row-major M with row stride ld) at (r0, k0)
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const bf16_t* M, int ld, int r0, int k0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    a[0] = ld32(M + (r0 + g) * ld + k0 + 2 * t);
    a[1] = ld32(M + (r0 + g + 8) * ld + k0 + 2 * t);
    a[2] = ld32(M + (r0 + g) * ld + k0 + 2 * t + 8);
    a[3] = ld32(M + (r0 + g + 8) * ld + k0 + 2 * t + 8);
}

// B fragment (16 x 8) at (k0, n0) from Bt, the transpose of B, row-major with stride ld
__device__ __forceinline__ void frag_b(uint32_t (&b)[2], const bf16_t* Bt, int ld, int k0, int n0, int lane) {
    const int g = lane >> 2, t = lane & 3;
    b[0] = ld32(Bt + (n0 + g) * ld + k0 + 2 * t);
    b[1] = ld32(Bt + (n0 + g) * ld + k0 + 2 * t + 8);
}

__device__ __forceinline__ void split_bf16(float x, bf16_t& hi, bf16_t& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

}  // namespace

// Split factors of the DFT matrix: Fm[q * N * N + j * N + k] for q = 0..5 is
// C_hi, C_lo, S_hi, S_lo, (-S)_hi, (-S)_lo with C = cos, S = sin of 2 pi j k / N,
// taken from the twiddle table tw[j] = e^{-2 i pi j / N}.
template <int N, int NT>
__device__ __forceinline__ void dft_matrix_split(bf16_t* Fm, const float2* tw) {
    for (int i = threadIdx.x; i < N * N; i += NT) {
        const float2 w = tw[((i / N) * (i % N)) & (N - 1)];
        split_bf16(w.x, Fm[i], Fm[N * N + i]);
        split_bf16(-w.y, Fm[2 * N * N + i], Fm[3 * N * N + i]);
        split_bf16(w.y, Fm[4 * N * N + i], Fm[5 * N * N + i]);
    }
}

// Z (row stride S, FP32 complex) <- F Z F (INV: conjugate F, no scaling).
// xb: 4 N^2 BF16 scratch in shared memory. Ends with a barrier.
template <int N, int NT, bool INV>
__device__ __forceinline__ void dft2_gemm(float2* Z, int S, bf16_t* xb, const bf16_t* Fm) {
    static_assert(N == 32 || N == 64, "DFT-GEMM grids");
    constexpr int NN = N * N, TILES = (N / 16) * (N / 8), NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    const bf16_t* Ch = Fm;
    const bf16_t* Cl = Fm + NN;
    // +S or -S by direction: forward F = C - iS, inverse F* = C + iS
    const bf16_t* Ph = Fm + (INV ? 4 : 2) * NN;  // multiplies the "real gets imag" term
    const bf16_t* Pl = Fm + (INV ? 5 : 3) * NN;
    const bf16_t* Mh = Fm + (INV ? 2 : 4) * NN;  // multiplies the "imag gets real" term
    const bf16_t* Ml = Fm + (INV ? 3 : 5) * NN;

    // step 1: Y = F X, with X split and stored transposed (B operand)
    for (int i = threadIdx.x; i < NN; i += NT) {
        const int r = i / N, c = i % N;
        const float2 v = Z[r * S + c];
        split_bf16(v.x, xb[c * N + r], xb[NN + c * N + r]);
        split_bf16(v.y, xb[2 * NN + c * N + r], xb[3 * NN + c * N + r]);
    }
    __syncthreads();
    for (int tile = warp; tile < TILES; tile += NW) {
        const int r0 = (tile / (N / 8)) * 16, n0 = (tile % (N / 8)) * 8;
        float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < N; k0 += 16) {
            uint32_t ch[4], cl[4], ph[4], pl[4], mh[4], ml[4], xrh[2], xrl[2], xih[2], xil[2];
            frag_a(ch, Ch, N, r0, k0, lane);
            frag_a(cl, Cl, N, r0, k0, lane);
            frag_a(ph, Ph, N, r0, k0, lane);
            frag_a(pl, Pl, N, r0, k0, lane);
            frag_a(mh, Mh, N, r0, k0, lane);
            frag_a(ml, Ml, N, r0, k0, lane);
            frag_b(xrh, xb, N, k0, n0, lane);
            frag_b(xrl, xb + NN, N, k0, n0, lane);
            frag_b(xih, xb + 2 * NN, N, k0, n0, lane);
            frag_b(xil, xb + 3 * NN, N, k0, n0, lane);
            // Yr = C Xr + (+-S) Xi ; Yi = C Xi + (-+S) Xr
            mma_bf16(ar, ch, xrh);
            mma_bf16(ar, ch, xrl);
            mma_bf16(ar, cl, xrh);
            mma_bf16(ar, ph, xih);
            mma_bf16(ar, ph, xil);
            mma_bf16(ar, pl, xih);
            mma_bf16(ai, ch, xih);
            mma_bf16(ai, ch, xil);
            mma_bf16(ai, cl, xih);
            mma_bf16(ai, mh, xrh);
            mma_bf16(ai, mh, xrl);
            mma_bf16(ai, ml, xrh);
        }
        Z[(r0 + g) * S + n0 + 2 * t4] = make_float2(ar[0], ai[0]);
        Z[(r0 + g) * S + n0 + 2 * t4 + 1] = make_float2(ar[1], ai[1]);
        Z[(r0 + g + 8) * S + n0 + 2 * t4] = make_float2(ar[2], ai[2]);
        Z[(r0 + g + 8) * S + n0 + 2 * t4 + 1] = make_float2(ar[3], ai[3]);
    }
    __syncthreads();
    // step 2: Z = Y F, with Y split row-major (A operand); F is symmetric, so
    // its rows serve as the transposed B operand
    for (int i = threadIdx.x; i < NN; i += NT) {
        const int r = i / N, c = i % N;
        const float2 v = Z[r * S + c];
        split_bf16(v.x, xb[i], xb[NN + i]);
        split_bf16(v.y, xb[2 * NN + i], xb[3 * NN + i]);
    }
    __syncthreads();
    for (int tile = warp; tile < TILES; tile += NW) {
        const int r0 = (tile / (N / 8)) * 16, n0 = (tile % (N / 8)) * 8;
        float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k0 = 0; k0 < N; k0 += 16) {
            uint32_t yrh[4], yrl[4], yih[4], yil[4], ch[2], cl[2], ph[2], pl[2], mh[2], ml[2];
            frag_a(yrh, xb, N, r0, k0, lane);
            frag_a(yrl, xb + NN, N, r0, k0, lane);
            frag_a(yih, xb + 2 * NN, N, r0, k0, lane);
            frag_a(yil, xb + 3 * NN, N, r0, k0, lane);
            frag_b(ch, Ch, N, k0, n0, lane);
            frag_b(cl, Cl, N, k0, n0, lane);
            frag_b(ph, Ph, N, k0, n0, lane);
            frag_b(pl, Pl, N, k0, n0, lane);
            frag_b(mh, Mh, N, k0, n0, lane);
            frag_b(ml, Ml, N, k0, n0, lane);
            // Zr = Yr C + Yi (+-S) ; Zi = Yi C + Yr (-+S)
            mma_bf16(ar, yrh, ch);
            mma_bf16(ar, yrh, cl);
            mma_bf16(ar, yrl, ch);
            mma_bf16(ar, yih, ph);
            mma_bf16(ar, yih, pl);
            mma_bf16(ar, yil, ph);
            mma_bf16(ai, yih, ch);
            mma_bf16(ai, yih, cl);
            mma_bf16(ai, yil, ch);
            mma_bf16(ai, yrh, mh);
            mma_bf16(ai, yrh, ml);
            mma_bf16(ai, yrl, mh);
        }
        Z[(r0 + g) * S + n0 + 2 * t4] = make_float2(ar[0], ai[0]);
        Z[(r0 + g) * S + n0 + 2 * t4 + 1] = make_float2(ar[1], ai[1]);
        Z[(r0 + g + 8) * S + n0 + 2 * t4] = make_float2(ar[2], ai[2]);
        Z[(r0 + g + 8) * S + n0 + 2 * t4 + 1] = make_float2(ar[3], ai[3]);
    }
    __syncthreads();
}
