// Register-level FFT building blocks shared by the kernels (sm_103a).
// Included inside namespace fwr by each kernel translation unit.
#pragma once

#include "fwr_w32t.inc"

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <int R> struct Log2 { static constexpr int v = 1 + Log2<R / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 t32(float2, int i) { return c_t32f[i]; }
__device__ __forceinline__ double2 t32(double2, int i) { return c_t32d[i]; }

// Radix-2 decimation-in-time butterfly a, b <- a + w b, a - w b with
// w = w_32^IDX (conjugated for the inverse). Trivial twiddles (1, -i) take 4
// adds; the others use the tangent form w = s (1 + i r) or s (r + i) with
// |r| <= 1: 6 fused multiply-adds instead of 4 adds and a complex multiply.
template <bool INV, int IDX, typename V>
__device__ __forceinline__ void bfly(V& a, V& b) {
    if constexpr (IDX == 0) {
        const V t = b;
        b = csub(a, t);
        a = cadd(a, t);
    } else if constexpr (IDX == 8) {
        const V t = INV ? mk(-b.y, b.x) : mk(b.y, -b.x);
        b = csub(a, t);
        a = cadd(a, t);
    } else {
        constexpr bool cos_form = IDX <= 4 || IDX >= 12;
        const V f = t32(a, IDX);
        auto s = f.x, r = f.y;
        if (INV) {
            r = -r;
            if (!cos_form) s = -s;
        }
        V u;
        if (cos_form) u = mk(fmadd(-r, b.y, b.x), fmadd(r, b.x, b.y));
        else u = mk(fmadd(r, b.x, -b.y), fmadd(r, b.y, b.x));
        const V a0 = a;
        a = mk(fmadd(s, u.x, a0.x), fmadd(s, u.y, a0.y));
        b = mk(fmadd(-s, u.x, a0.x), fmadd(-s, u.y, a0.y));
    }
}

// All butterflies of a radix-2 DIT network, enumerated at compile time:
// stage S (half size h = 2^S), block start B, index J < h.
template <int R, bool INV, int S, int B, int J, typename V>
__device__ __forceinline__ void dit_net(V* y) {
    if constexpr (S < Log2<R>::v) {
        constexpr int h = 1 << S;
        if constexpr (B >= R) {
            dit_net<R, INV, S + 1, 0, 0>(y);
        } else if constexpr (J >= h) {
            dit_net<R, INV, S, B + 2 * h, 0>(y);
        } else {
            bfly<INV, J*(16 / h)>(y[B + J], y[B + J + h]);
            dit_net<R, INV, S, B, J + 1>(y);
        }
    }
}

template <int I, int R, typename V>
__device__ __forceinline__ void bitrev_copy(V* y, const V* x) {
    if constexpr (I < R) {
        y[I] = x[bitrev(I, Log2<R>::v)];
        bitrev_copy<I + 1, R>(y, x);
    }
}

// In-register R-point DFT (R <= 32), natural order in and out (the input
// bit reversal is a register renaming). Forward uses e^{-2 i pi / R}; INV the
// conjugate, without scaling.
template <int R, bool INV, typename V>
__device__ __forceinline__ void dft_reg(V* x) {
    V y[R];
    bitrev_copy<0, R>(y, x);
    dit_net<R, INV, 0, 0, 0>(y);
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] = y[i];
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
