// Device code of the 256^2 slab-streamed Gerchberg kernel (fwr_slab.cu),
// shared with the ragged-batch kernel (fwr_ragged.cu). Included inside
// namespace fwr after fwr_fft.cuh.
#pragma once

// Gerchberg kernel for 256^2 grids (sm_103a): slab-streamed through shared memory.
//
// A 256 x 256 complex grid (512 KB) does not fit one SM's shared memory, so
// each persistent CTA keeps its frame's packed grid Z = sx + i sy in its own
// area of a global scratch buffer (L2 resident: 512 KB per CTA) and streams
// it through shared memory in slabs of 64 lines:
//
//   row phase, 4 slabs of 64 rows:     inverse row FFTs, reinsertion of the
//                                      measured slopes (Algorithm 1 step 4),
//                                      x part of the periodic fill (Eq. PC),
//                                      forward row FFTs
//   column phase, 4 slabs of 64 cols:  forward column FFTs, y part of Eq. PC
//                                      as a spectral correction, the LSQ
//                                      projection (Sec. 3.3) or the final
//                                      filter (Eqs. 2-3), inverse column FFTs
//
// Column slab s holds the columns kx in [32 s, 32 s + 32) and their partners
// -kx (slab 0 also holds the self-paired column 128), so every (k, -k) pair of
// the spectral step lies in one slab. One iteration moves 2 MB between L2 and
// shared memory per frame.
//
// 256-point line FFTs: two register passes, 16-point DFTs over elements 16
// apart with twiddles w_256^(n2 k1), then 16-point DFTs over contiguous groups
// written back in natural order. Line stride 257 keeps warps that walk 32
// consecutive lines bank-conflict free.

namespace {

constexpr int SN = 256;        // grid size
constexpr int SL = 64;         // lines per slab
constexpr int SLS = SN + 1;    // line stride in shared memory
constexpr int SNT = 512;       // threads per CTA
constexpr int SH = SN / 2;
constexpr int WS = 33;         // row stride of the spectral weights of a column slab

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// asynchronous global -> shared copies (cp.async), completed by cp_wait_all
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// prefetch [p, p + bytes) into L2, one 128-byte line per thread and step
__device__ __forceinline__ void prefetch_lines_l2(const void* p, size_t bytes) {
    const char* b = static_cast<const char*>(p);
    for (size_t o = size_t(threadIdx.x) * 128; o < bytes; o += size_t(blockDim.x) * 128)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(b + o));
}

// Pass A over the 64 lines: 16-point DFT over n1 of elements 16 n1 + n2,
// then the twiddle w^(n2 k1) (conjugate for the inverse), in place.
template <bool INV>
__device__ __forceinline__ void line_pass_a(float2* Lb, const float2* tw) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int t = threadIdx.x + i * SNT;
        const int line = t % SL, n2 = t / SL;
        float2* base = Lb + line * SLS + n2;
        float2 x[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) x[n1] = base[16 * n1];
        dft_reg<16, INV>(x);
#pragma unroll
        for (int k1 = 1; k1 < 16; ++k1) {
            const float2 w = tw[n2 * k1];
            x[k1] = INV ? cmulc(w, x[k1]) : cmul(x[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) base[16 * k1] = x[k1];
    }
}

// Pass B: 16-point DFT over contiguous groups 16 k1 + n2, natural-order output.
template <bool INV>
__device__ __forceinline__ void line_pass_b(float2* Lb) {
    float2 y[2][16];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int t = threadIdx.x + i * SNT;
        const int line = t % SL, k1 = t / SL;
        const float2* base = Lb + line * SLS + 16 * k1;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) y[i][n2] = base[n2];
        dft_reg<16, INV>(y[i]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int t = threadIdx.x + i * SNT;
        const int line = t % SL, k1 = t / SL;
        float2* base = Lb + line * SLS + k1;
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) base[16 * k2] = y[i][k2];
    }
}

// 256-point FFT of all 64 lines of the slab; ends with a barrier.
template <bool INV>
__device__ __forceinline__ void line_fft(float2* Lb, const float2* tw) {
    line_pass_a<INV>(Lb, tw);
    __syncthreads();
    line_pass_b<INV>(Lb);
    __syncthreads();
}

// storage column of line j in column slab s: j < 32 -> 32 s + j; j >= 32 ->
// the partner -(32 s + j - 32), with the self-paired column 128 in place of
// the duplicate 0 in slab 0
__device__ __forceinline__ int slab_col(int s, int j) {
    if (j < 32) return 32 * s + j;
    const int jj = j - 32;
    return (s == 0 && jj == 0) ? SH : (SN - 32 * s - jj) & (SN - 1);
}
// partner line of line j < 32 in slab s (self-paired for column 0)
__device__ __forceinline__ int slab_partner(int s, int j) { return (s == 0 && j == 0) ? 0 : 32 + j; }

}  // namespace

// Shared-memory bytes of the slab path for n lenslets: the slab, the 1-D
// tables (twiddles, a(u), T(u), the separable factors p(u)), Sy(0, kx) per
// column pair, the spectral weights of the current column slab (256 rows x
// 33 columns) and the mask.
__host__ __device__ __forceinline__ size_t slab_layout_bytes(int n) {
    return size_t(SL) * SLS * sizeof(float2) + 3 * size_t(SN) * sizeof(float2) + 4 * size_t(SN) * sizeof(float) +
           33 * sizeof(float2) + WS * size_t(SN) * sizeof(float) + ((size_t(n) * n + 15) & ~size_t(15));
}

// Per-CTA state of the slab path for one plan.
struct SlabCtx {
    float2* Lb;
    float2* tw;
    float2* A;
    float2* Tt;
    float* pt;
    float2* eyv;
    float* wts;
    uint8_t* mask;
    int n, off, nn, mode;
    int pw;  // log2 of the lenslet count rounded up to a power of two
};

// Load a plan's 1-D tables and mask into shared memory; ends with a barrier.
__device__ __forceinline__ void slab_setup(SlabCtx& c, unsigned char* smem, const Tables<float>& tab,
                                           const uint8_t* mask_g, int n, int off, int mode) {
    c.Lb = reinterpret_cast<float2*>(smem);
    c.tw = c.Lb + SL * SLS;
    c.A = c.tw + SN;
    c.Tt = c.A + SN;
    c.pt = reinterpret_cast<float*>(c.Tt + SN);
    c.eyv = reinterpret_cast<float2*>(c.pt + 4 * SN);
    c.wts = reinterpret_cast<float*>(c.eyv + 33);
    c.mask = reinterpret_cast<uint8_t*>(c.wts + WS * SN);
    c.n = n;
    c.off = off;
    c.nn = n * n;
    c.mode = mode;
    c.pw = 0;
    while ((1 << c.pw) < n) ++c.pw;
    const int tid = threadIdx.x;
    for (int i = tid; i < SN; i += SNT) {
        c.tw[i] = tab.tw[i];
        c.A[i] = tab.A[i];
        c.Tt[i] = tab.Tt[i];
    }
    for (int i = tid; i < 4 * SN; i += SNT) c.pt[i] = tab.pt[i];
#pragma unroll 8
    for (int i = tid; i < c.nn; i += SNT) c.mask[i] = mask_g[i];
    __syncthreads();
}

// One frame through the whole path with the grid in G (this CTA's 256^2
// scratch area). sl: [2][n][n] slopes; ext: [2][N][N] warm start or nullptr;
// phase: [N][N] output. Called by every thread; returns false in the threads
// that saw a non-finite measured slope.
//
// Thread roles. Slab copies: a thread keeps one line (column slabs: line
// tid mod 64, rows tid / 64 + 8 i) or one column (row slabs: column tid mod 256,
// rows tid / 256 + 2 i), so its addresses advance by constant strides. Spectral
// step: a thread keeps one frequency row ky = tid mod 256 (and its partner -ky)
// and takes the lines j = tid / 256 + 2 i, so the ky factors stay in registers
// and the kx factors are warp-uniform.
__device__ __forceinline__ bool slab_frame(const SlabCtx& c, const Tables<float>& tab, const float* sl,
                                           const float* ext, float* phase, int iters, float2* G,
                                           const int16_t* hud = nullptr) {
    const int tid = threadIdx.x;
    float2* const Lb = c.Lb;
    const float2* const tw = c.tw;
    const float2* const A = c.A;
    const float2* const Tt = c.Tt;
    const float* const pt = c.pt;
    float2* const eyv = c.eyv;
    float* const wts = c.wts;
    const uint8_t* const mask = c.mask;
    const int n = c.n, off = c.off, nn = c.nn, mode = c.mode;
    bool finite = true;
    // spectral roles: frequency row ky and its partner -ky
    const int ky = tid & (SN - 1), kyn = (SN - ky) & (SN - 1);
    // column-slab copy roles: line jl, rows rb + 8 i
    const int jl = tid & (SL - 1), rb = tid >> 6;
    // row-slab copy roles: column cc, rows lb + 2 i
    const int cc = tid & (SN - 1), lb = tid >> 8;
    // it = -1: embed; it = 0 .. iters-1: Gerchberg; it = iters: final
    for (int it = -1; it <= iters; ++it) {
        const bool final = it == iters;
        if (it >= 0) {
            // ------------------------------------------------ column phase
            const bool fill = mode == PERIODIC_BEFORE_EACH_FFT || (mode == PERIODIC_FINAL_ONLY && final);
            // per-ky factors of the projection (LSQ) or of G (final filter)
            const float4 pv = *reinterpret_cast<const float4*>(pt + 4 * ky);
            const float2 Tky = Tt[ky], Aky = A[ky], twk = tw[ky];
            for (int s = 0; s < 4; ++s) {
                {
                    const float2* src = G + slab_col(s, jl) + rb * SN;
                    float2* dst = Lb + jl * SLS + rb;
#pragma unroll 8
                    for (int i = 0; i < SN / 8; ++i) cp_async8(dst + 8 * i, src + 8 * i * SN);
                }
                {
                    // spectral weights of the first-half columns: wts[ky][j] at
                    // (ky, kx) from the half-table (rows 0..N/2; (-ky, -kx) beyond);
                    // a warp reads 32 adjacent columns of one table row
                    const float* wt = final ? tab.wfin : tab.iota;
                    const int j = tid & 31, kx = slab_col(s, j), kxn = (SN - kx) & (SN - 1);
                    for (int k = tid >> 5; k < SN; k += SNT / 32)
                        cp_async4(wts + k * WS + j, wt + (k <= SH ? k * SN + kx : (SN - k) * SN + kxn));
                    if (s == 0 && tid < SN)  // line 32: the self-paired column 128
                        cp_async4(wts + tid * WS + 32, wt + (tid <= SH ? tid : SN - tid) * SN + SH);
                }
                cp_wait_all();
                __syncthreads();
                line_fft<false>(Lb, tw);
                if (fill && tid < 33) {
                    // Sy(0, kx) of every first-half column (and of column 128 in
                    // slab 0), read before the in-place spectral updates below
                    const int j = tid, pj = j < 32 ? slab_partner(s, j) : 32;
                    const float2 e0 = Lb[j * SLS], e1 = Lb[pj * SLS];
                    eyv[j] = make_float2(0.5f * (e0.y + e1.y), 0.5f * (e1.x - e0.x));
                }
                __syncthreads();
                // one (k, -k) pair per item: line j (kx) at row ky, partner line pj
                // (-kx) at row -ky; lines 0..31, plus line 32 (column 128) in slab 0
                const int jend = (s == 0 && tid <= SH) ? 34 : 32;
                for (int j = lb; j < jend; j += 2) {
                    const int jj = j < 32 ? j : 32;
                    const int pj = jj < 32 ? slab_partner(s, jj) : 32;
                    if (pj == jj && ky > SH) continue;  // self-paired column: half the rows
                    const int kx = slab_col(s, jj);
                    float2 z1 = Lb[jj * SLS + ky], z2 = Lb[pj * SLS + kyn];
                    if (fill) {
                        // y part of Eq. PC: Sy(ky,kx) -= Sy(0,kx) e^{2 i pi ky / N}, i.e.
                        // Z(k) -= i c and Z(-k) -= i conj(c), c = Sy(0,kx) e^{2 i pi ky / N}
                        const float2 c0 = cmul(eyv[jj], conjf2(twk));
                        z1 = make_float2(z1.x + c0.y, z1.y - c0.x);
                        z2 = make_float2(z2.x - c0.y, z2.y - c0.x);
                    }
                    const float w = wts[ky * WS + jj];
                    if (!final) {
                        // Algorithm 1 step 2 for both bins: Z'(k) = w (a z1 + b conj z2),
                        // Z'(-k) = w (a' z2 + b conj z1), a = |G|^2/2 + Im P, a' = |G|^2/2 - Im P,
                        // b = (|Gx|^2 - |Gy|^2)/2 + i Re P, P = p(u) conj p(v)
                        const float4 pu = *reinterpret_cast<const float4*>(pt + 4 * kx);
                        const float Px = pu.x * pv.x + pu.y * pv.y, Py = pu.y * pv.x - pu.x * pv.y;
                        const float h1 = 0.5f * pu.z * pv.w, h2 = 0.5f * pu.w * pv.z;
                        const float g = h1 + h2, br = h1 - h2, bi = Px;
                        const float a = g + Py, an = g - Py;
                        const float2 o1 = make_float2(a * z1.x + br * z2.x + bi * z2.y, a * z1.y + bi * z2.x - br * z2.y);
                        const float2 o2 = make_float2(an * z2.x + br * z1.x + bi * z1.y, an * z2.y + bi * z1.x - br * z1.y);
                        Lb[pj * SLS + kyn] = make_float2(w * o2.x, w * o2.y);
                        Lb[jj * SLS + ky] = make_float2(w * o1.x, w * o1.y);
                    } else {
                        // Eq. 2 with the final filter: phi = w (conj(Gx) Sx + conj(Gy) Sy)
                        const float2 z2c = conjf2(z2);
                        const float2 sx = make_float2(0.5f * (z1.x + z2c.x), 0.5f * (z1.y + z2c.y));
                        const float2 sy = make_float2(0.5f * (z1.y - z2c.y), 0.5f * (z2c.x - z1.x));
                        const float2 gx = cmul(A[kx], Tky);
                        const float2 gy = cmul(Tt[kx], Aky);
                        float2 ph = cadd(cmulc(gx, sx), cmulc(gy, sy));
                        ph = make_float2(ph.x * w, ph.y * w);
                        Lb[pj * SLS + kyn] = conjf2(ph);
                        Lb[jj * SLS + ky] = ph;
                    }
                }
                __syncthreads();
                line_fft<true>(Lb, tw);
                {
                    float2* dst = G + slab_col(s, jl) + rb * SN;
                    const float2* src = Lb + jl * SLS + rb;
#pragma unroll 8
                    for (int i = 0; i < SN / 8; ++i) __stcg(dst + 8 * i * SN, src[8 * i]);
                }
                __syncthreads();
            }
        }
        // --------------------------------------------------------- row phase
        const bool fill_next = !final && (mode == PERIODIC_BEFORE_EACH_FFT ||
                                          (mode == PERIODIC_FINAL_ONLY && it + 1 == iters));
        for (int b = 0; b < 4; ++b) {
            const int m0 = SL * b;
            {
                // this slab's measured slopes into L2 while it is loaded and transformed
                const int p0 = max(0, m0 - off), p1 = min(n, m0 + SL - off);
                if (p1 > p0) {
                    prefetch_lines_l2(sl + p0 * n, size_t(p1 - p0) * n * sizeof(float));
                    prefetch_lines_l2(sl + nn + p0 * n, size_t(p1 - p0) * n * sizeof(float));
                }
            }
            if (it < 0) {
                for (int l = lb; l < SL; l += 2) {
                    const int g = (m0 + l) * SN + cc;
                    float2 v = make_float2(0.f, 0.f);
                    if (ext) {
                        v = make_float2(ext[g], ext[SN * SN + g]);
                    } else if (hud) {
                        // Hudgin extension from the measured slopes of the pupil
                        // edges (the pupil cells are overwritten below)
                        const int i = m0 + l - off, j = cc - off;
                        if (j >= 0 && j < n) {
                            const int t = __ldg(hud + j), b2 = __ldg(hud + n + j);
                            if (t >= 0 && (i < t || i > b2)) v.x = __ldg(sl + (i < t ? t : b2) * n + j);
                        }
                        if (i >= 0 && i < n) {
                            const int le = __ldg(hud + 2 * n + i), rt = __ldg(hud + 3 * n + i);
                            if (le >= 0 && (j < le || j > rt)) v.y = __ldg(sl + nn + i * n + (j < le ? le : rt));
                        }
                    }
                    Lb[l * SLS + cc] = v;
                }
            } else {
                {
                    const float2* src = G + (m0 + lb) * SN + cc;
                    float2* dst = Lb + lb * SLS + cc;
#pragma unroll 8
                    for (int i = 0; i < SL / 2; ++i) cp_async8(dst + 2 * i * SLS, src + 2 * i * SN);
                }
                cp_wait_all();
                __syncthreads();
                line_fft<true>(Lb, tw);
                if (final) {
                    float* ph = phase + (m0 + lb) * SN + cc;
                    const float2* src = Lb + lb * SLS + cc;
#pragma unroll 8
                    for (int i = 0; i < SL / 2; ++i) __stcs(ph + 2 * i * SN, src[2 * i * SLS].x);
                    __syncthreads();
                    continue;
                }
            }
            __syncthreads();
            // Algorithm 1 step 4 (and the embedding): measurement in the pupil
            // the slope loads do not depend on the mask (every address is in
            // the frame), so unrolled iterations keep several L2 reads in flight
            // (thread: lenslet column tid mod 2^pw, rows tid >> pw + steps of 512 >> pw)
            const int i0 = max(0, m0 - off), i1 = min(n, m0 + SL - off);
            const int j = tid & ((1 << c.pw) - 1);
            if (j < n) {
#pragma unroll 16
                for (int i = i0 + (tid >> c.pw); i < i1; i += SNT >> c.pw) {
                    const float vx = __ldg(sl + i * n + j), vy = __ldg(sl + nn + i * n + j);
                    if (mask[i * n + j]) {
                        if (it < 0) finite &= isfinite(vx) && isfinite(vy);
                        Lb[(off + i - m0) * SLS + off + j] = make_float2(vx, vy);
                    }
                }
            }
            __syncthreads();
            if (fill_next) {
                // x part of Eq. PC: 8 lanes per row; a warp takes rows 8 apart so
                // its lanes read .x words in distinct bank pairs
                const int w = tid >> 5, lane = tid & 31;
                const int l = 32 * (w >> 3) + (w & 7) + 8 * (lane >> 3), part = lane & 7;
                float s = 0.f;
                for (int c = part; c < SN - 1; c += 8) s += Lb[l * SLS + c].x;
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                if (part == 0) Lb[l * SLS + SN - 1].x = -s;
                __syncthreads();
            }
            line_fft<false>(Lb, tw);
            {
                float2* dst = G + (m0 + lb) * SN + cc;
                const float2* src = Lb + lb * SLS + cc;
#pragma unroll 8
                for (int i = 0; i < SL / 2; ++i) __stcg(dst + 2 * i * SN, src[2 * i * SLS]);
            }
            __syncthreads();
        }
    }
    return finite;
}
