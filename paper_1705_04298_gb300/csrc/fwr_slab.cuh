// Device code of the 256^2 slab-streamed Gerchberg kernel (fwr_slab.cu),
// shared with the ragged-batch kernel (fwr_ragged.cu). Included inside
// namespace fwr after fwr_fft.cuh.
#pragma once

// Gerchberg kernel for 256^2 grids (sm_103a): slab-streamed through shared memory.
//
// A 256 x 256 complex grid (512 KB) does not fit one SM's shared memory, so
// each persistent CTA keeps its frame's packed grid Z = sx + i sy in its own
// area of a global scratch buffer (L2 resident: 512 KB per CTA) and works it
// in slabs of 32 lines:
//
//   row phase, 8 slabs of 32 rows:     inverse row FFTs, reinsertion of the
//                                      measured slopes (Algorithm 1 step 4),
//                                      x part of the periodic fill (Eq. PC),
//                                      forward row FFTs
//   column phase, 8 slabs of 32 cols:  forward column FFTs, y part of Eq. PC
//                                      as a spectral correction, the LSQ
//                                      projection (Sec. 3.3) or the final
//                                      filter (Eqs. 2-3), inverse column FFTs
//
// Column slab s holds the columns kx in [16 s, 16 s + 16) and their partners
// -kx (slab 0 also holds the self-paired column 128), so every (k, -k) pair of
// the spectral step lies in one slab.
//
// The CTA's 16 warps form two groups of 8 that work different slabs of the
// same phase at the same time (group g takes slabs g, g + 2, ...), each with
// its own shared-memory buffer and named barrier, so one group's L2 loads
// overlap the other's arithmetic; a CTA barrier separates the phases.
//
// 256-point line FFTs: two register passes (four-step), 16-point DFTs over
// elements 16 apart with twiddles w_256^(n2 k1), then 16-point DFTs over the
// other index. A task keeps 16 points of one line. The slab data move
// between the scratch area (L2) and registers directly (coalesced 8-byte
// loads and stores: the lanes of a warp take adjacent columns in the column
// phase, 16 adjacent cells of a row in the row phase), and shared memory is
// used only for the exchanges between the passes:
//   column phase: L2 -> pass A -> smem -> pass B -> smem (the partner bins of
//     the spectral step) -> spectral step and inverse pass A in registers ->
//     smem -> inverse pass B -> L2;
//   row phase: L2 -> inverse pass A -> smem -> inverse pass B, reinsertion,
//     x fill (row sums by warp shuffles) and forward pass A in registers (the
//     inverse pass B leaves each task the cells the forward pass A needs) ->
//     smem -> pass B -> L2.
// That is six crossings of shared memory per column slab and four per row
// slab. Column-phase exchanges use lines 257 cells apart, row-phase ones
// groups of 16 cells 17 apart: both bank-conflict free.

namespace {

constexpr int SN = 256;        // grid size
constexpr int SNT = 512;       // threads per CTA
constexpr int SH = SN / 2;
constexpr int CLS = SN + 1;    // column phase: line stride in shared memory (cells)
constexpr int RGS = 17;        // row phase: stride of the 16-cell groups of a line
constexpr int RLS = 16 * RGS;  // row phase: line stride
constexpr int SLAB_LINES = 64; // lines of all groups' slabs together

// Kernel shape: GROUPS warp groups (1 or 2) of 512 / GROUPS threads, each on
// its own slab of 64 / GROUPS lines at a time.
template <int GROUPS> struct SlabShape {
    static_assert(GROUPS == 1 || GROUPS == 2, "one or two groups");
    static constexpr int SL = SLAB_LINES / GROUPS;  // lines per slab
    static constexpr int SGT = SNT / GROUPS;        // threads per group
    static constexpr int SC = SL / 2;               // first-half columns of a column slab
    static constexpr int WS = SC + 1;               // row stride of a group's spectral weights
    static constexpr int LB_CELLS = SL * RLS;       // one group's buffer
    static_assert(SL * CLS <= LB_CELLS, "slab buffer");
};

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// barrier of one group's threads (named barrier 1 + g)
__device__ __forceinline__ void group_sync(int g, int threads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(g + 1), "r"(threads) : "memory");
}

// asynchronous global -> shared copies (cp.async), completed by cp_wait_all
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// prefetch [p, p + bytes) into L2, one 128-byte line per thread (of nthreads) and step
__device__ __forceinline__ void prefetch_lines_l2(const void* p, size_t bytes, int t, int nthreads) {
    const char* b = static_cast<const char*>(p);
    for (size_t o = size_t(t) * 128; o < bytes; o += size_t(nthreads) * 128)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(b + o));
}

// storage column of line j in column slab s (SC first-half columns per
// slab): j < SC -> SC s + j; j >= SC -> the partner -(SC s + j - SC), with the
// self-paired column 128 in place of the duplicate 0 in slab 0
template <int SC>
__device__ __forceinline__ int slab_col(int s, int j) {
    if (j < SC) return SC * s + j;
    const int jj = j - SC;
    return (s == 0 && jj == 0) ? SH : (SN - SC * s - jj) & (SN - 1);
}
// the line holding the partner column -kx of line j (self-paired: columns 0
// and 128, lines 0 and SC of slab 0)
template <int SC>
__device__ __forceinline__ int partner_line(int s, int j) { return (s == 0 && (j & (SC - 1)) == 0) ? j : (j ^ SC); }

// forward (INV = false) or inverse 16-point DFT of x with the twiddle
// w_256^(n2 k) (conjugated for the inverse) applied to output k; tw16 holds
// w_256^(n2 k) at [k][n2], so lanes with consecutive n2 read consecutive
// entries (the row phase) and lanes with one n2 read one entry (the column
// phase): no bank conflicts either way
template <bool INV>
__device__ __forceinline__ void dft16_tw(float2 (&x)[16], const float2* tw16, int n2) {
    dft_reg<16, INV>(x);
#pragma unroll
    for (int k = 1; k < 16; ++k) {
        const float2 w = tw16[16 * k + n2];
        x[k] = INV ? cmulc(w, x[k]) : cmul(x[k], w);
    }
}

}  // namespace

// Shared-memory bytes of the slab path for n lenslets: the two groups' slab
// exchange buffers and spectral weights (256 rows x 17 columns each), the 1-D
// tables (twiddles, a(u), T(u), the separable factors p(u)) and the mask.
// (The weights of one group's slab take WS x SN floats; two groups of 17
// columns need one column more than one group of 33, so the layout reserves
// the larger.)
constexpr int SLAB_WTS = 2 * SlabShape<2>::WS * SN > SlabShape<1>::WS * SN ? 2 * SlabShape<2>::WS * SN
                                                                               : SlabShape<1>::WS * SN;
__host__ __device__ __forceinline__ size_t slab_layout_bytes(int n) {
    return size_t(SLAB_LINES) * RLS * sizeof(float2) + 3 * size_t(SN) * sizeof(float2) + 256 * sizeof(float2) +
           4 * size_t(SN) * sizeof(float) + size_t(SLAB_WTS) * sizeof(float) + ((size_t(n) * n + 15) & ~size_t(15));
}

// Per-CTA state of the slab path for one plan.
struct SlabCtx {
    float2* Lb;   // the groups' buffers (64 lines of RLS cells in all)
    float2* tw;
    float2* A;
    float2* Tt;
    float2* tw16;  // w_256^(n2 k) at [k][n2], n2, k < 16
    float* pt;
    float* wts;   // the groups' weight tables (SLAB_WTS floats in all)
    uint8_t* mask;
    int n, off, nn, mode;
};

// Load a plan's 1-D tables and mask into shared memory; ends with a barrier.
__device__ __forceinline__ void slab_setup(SlabCtx& c, unsigned char* smem, const Tables<float>& tab,
                                           const uint8_t* mask_g, int n, int off, int mode) {
    c.Lb = reinterpret_cast<float2*>(smem);
    c.tw = c.Lb + SLAB_LINES * RLS;
    c.A = c.tw + SN;
    c.Tt = c.A + SN;
    c.tw16 = c.Tt + SN;
    c.pt = reinterpret_cast<float*>(c.tw16 + 256);
    c.wts = c.pt + 4 * SN;
    c.mask = reinterpret_cast<uint8_t*>(c.wts + SLAB_WTS);
    c.n = n;
    c.off = off;
    c.nn = n * n;
    c.mode = mode;
    const int tid = threadIdx.x;
    for (int i = tid; i < SN; i += SNT) {
        c.tw[i] = tab.tw[i];
        c.A[i] = tab.A[i];
        c.Tt[i] = tab.Tt[i];
    }
    for (int i = tid; i < 4 * SN; i += SNT) c.pt[i] = tab.pt[i];
    if (tid < 256) c.tw16[tid] = tab.tw[(tid & 15) * (tid >> 4)];
#pragma unroll 8
    for (int i = tid; i < c.nn; i += SNT) c.mask[i] = mask_g[i];
    __syncthreads();
}

// One frame through the whole path with the grid in G (this CTA's 256^2
// scratch area). sl: [2][n][n] slopes; ext: [2][N][N] warm start or nullptr;
// phase: [N][N] output. Called by every thread; returns false in the threads
// that saw a non-finite measured slope.
//
// Tasks: a thread works two tasks of 16 points in every pass. Column phase:
// line t mod SL (both tasks), pass index q = t / SL and q + 8 (t: the
// thread's index in its group). Row phase: cell group q = t mod 16 (both
// tasks), lines t / 16 and + SL / 2. Both shapes give bitwise the same
// result (each line transform and each bin's arithmetic is the same).
template <int GROUPS>
__device__ __forceinline__ bool slab_frame(const SlabCtx& c, const Tables<float>& tab, const float* sl,
                                           const float* ext, float* phase, int iters, float2* G,
                                           const int16_t* hud = nullptr) {
    typedef SlabShape<GROUPS> Sh;
    constexpr int SL = Sh::SL, SGT = Sh::SGT, SC = Sh::SC, WS = Sh::WS;
    const int g = threadIdx.x / SGT, tg = threadIdx.x % SGT;
    float2* const Lb = c.Lb + g * Sh::LB_CELLS;
    const float2* const tw = c.tw;
    const float2* const tw16 = c.tw16;
    const float2* const A = c.A;
    const float2* const Tt = c.Tt;
    const float* const pt = c.pt;
    float* const wts = c.wts + g * WS * SN;
    const uint8_t* const mask = c.mask;
    const int n = c.n, off = c.off, nn = c.nn, mode = c.mode;
    bool finite = true;
    // column-phase roles
    const int cl = tg & (SL - 1), cq = tg / SL;
    // row-phase roles
    const int rq = tg & 15, rl = tg >> 4;
    const unsigned half_mask = 0xFFFFu << (threadIdx.x & 16);  // the 16 lanes of this row group
    // it = -1: embed; it = 0 .. iters-1: Gerchberg; it = iters: final
    for (int it = -1; it <= iters; ++it) {
        const bool final = it == iters;
        if (it >= 0) {
            // ------------------------------------------------ column phase
            const bool fill = mode == PERIODIC_BEFORE_EACH_FFT || (mode == PERIODIC_FINAL_ONLY && final);
            for (int s = g; s < SN / SL; s += GROUPS) {
                const int kx = slab_col<SC>(s, cl);
                const int pl = partner_line<SC>(s, cl);
                {
                    // spectral weights of the first-half columns: wts[ky][j] at
                    // (ky, kx) from the half-table (rows 0..N/2; (-ky, -kx) beyond);
                    // 16 lanes read 16 adjacent columns of one table row
                    const float* wt = final ? tab.wfin : tab.iota;
                    const int j = tg & (SC - 1), kxj = slab_col<SC>(s, j), kxn = (SN - kxj) & (SN - 1);
                    for (int k = tg / SC; k < SN; k += SGT / SC)
                        cp_async4(wts + k * WS + j, wt + (k <= SH ? k * SN + kxj : (SN - k) * SN + kxn));
                    if (s == 0)  // line SC: the self-paired column 128
                        for (int k = tg; k < SN; k += SGT)
                            cp_async4(wts + k * WS + SC, wt + (k <= SH ? k : SN - k) * SN + SH);
                }
                float2 x[2][16];
                // pass A: 16-point DFTs over rows 16 n1 + n2 of the column, straight from L2
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int n2 = cq + 8 * i;
#pragma unroll
                    for (int n1 = 0; n1 < 16; ++n1) x[i][n1] = __ldcg(G + (16 * n1 + n2) * SN + kx);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int n2 = cq + 8 * i;
                    dft16_tw<false>(x[i], tw16, n2);
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) Lb[cl * CLS + 16 * k1 + n2] = x[i][k1];
                }
                group_sync(g, SGT);
                // pass B: bins ky = k1 + 16 k2 of the column
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int k1 = cq + 8 * i;
#pragma unroll
                    for (int n2 = 0; n2 < 16; ++n2) x[i][n2] = Lb[cl * CLS + 16 * k1 + n2];
                    dft_reg<16, false>(x[i]);
                }
                group_sync(g, SGT);
                // the spectrum in natural order, for the partner bins
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int k1 = cq + 8 * i;
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) Lb[cl * CLS + k1 + 16 * k2] = x[i][k2];
                }
                cp_wait_all();
                group_sync(g, SGT);
                // spectral step on the task's own bins (ky, kx), partner (-ky, -kx) from
                // shared memory; then the inverse pass A on the same registers
                float2 ey = make_float2(0.f, 0.f);
                if (fill) {
                    // Sy(0, kx) = (Z(0, kx) - conj Z(0, -kx)) / (2i), uncorrected values
                    const float2 e0 = Lb[cl * CLS], e1 = Lb[pl * CLS];
                    ey = make_float2(0.5f * (e0.y + e1.y), 0.5f * (e1.x - e0.x));
                }
                const float4 pu = *reinterpret_cast<const float4*>(pt + 4 * kx);
                const float2 Akx = A[kx], Tkx = Tt[kx];
                // weight column of this line and whether its rows are mirrored
                const bool first = cl < SC || (s == 0 && cl == SC);
                const int wcol = (s == 0 && cl == SC) ? SC : (cl & (SC - 1));
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int k1 = cq + 8 * i;
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) {
                        const int ky = k1 + 16 * k2, kyn = (SN - ky) & (SN - 1);
                        float2 z1 = x[i][k2], z2 = Lb[pl * CLS + kyn];
                        if (fill) {
                            // y part of Eq. PC: Z(k) -= i c, Z(-k) -= i conj(c),
                            // c = Sy(0, kx) e^{2 i pi ky / N}
                            const float2 c0 = cmul(ey, conjf2(tw[ky]));
                            z1 = make_float2(z1.x + c0.y, z1.y - c0.x);
                            z2 = make_float2(z2.x - c0.y, z2.y - c0.x);
                        }
                        const float w = wts[(first ? ky : kyn) * WS + wcol];
                        const float4 pv = *reinterpret_cast<const float4*>(pt + 4 * ky);
                        if (!final) {
                            // Algorithm 1 step 2: Z'(k) = w (a z1 + b conj z2) with, at the
                            // bin's own frequency, a = |G|^2/2 + Im P, b = (|Gx|^2 - |Gy|^2)/2
                            // + i Re P, P = Gx conj(Gy) = p(u) conj p(v)
                            const float Px = pu.x * pv.x + pu.y * pv.y, Py = pu.y * pv.x - pu.x * pv.y;
                            const float h1 = 0.5f * pu.z * pv.w, h2 = 0.5f * pu.w * pv.z;
                            const float a = h1 + h2 + Py, br = h1 - h2, bi = Px;
                            const float ox = a * z1.x + br * z2.x + bi * z2.y;
                            const float oy = a * z1.y + bi * z2.x - br * z2.y;
                            x[i][k2] = make_float2(w * ox, w * oy);
                        } else {
                            // Eq. 2 with the final filter: phi = w (conj(Gx) Sx + conj(Gy) Sy)
                            const float2 z2c = conjf2(z2);
                            const float2 sx = make_float2(0.5f * (z1.x + z2c.x), 0.5f * (z1.y + z2c.y));
                            const float2 sy = make_float2(0.5f * (z1.y - z2c.y), 0.5f * (z2c.x - z1.x));
                            const float2 gx = cmul(Akx, Tt[ky]);
                            const float2 gy = cmul(Tkx, A[ky]);
                            const float2 ph = cadd(cmulc(gx, sx), cmulc(gy, sy));
                            x[i][k2] = make_float2(ph.x * w, ph.y * w);
                        }
                    }
                    // inverse pass A: the bins ky = 16 n1 + n2 with n2 = k1
                    dft16_tw<true>(x[i], tw16, k1);
                }
                group_sync(g, SGT);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int n2 = cq + 8 * i;
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) Lb[cl * CLS + 16 * k1 + n2] = x[i][k1];
                }
                group_sync(g, SGT);
                // inverse pass B, rows k1 + 16 k2 of the column back to L2
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int k1 = cq + 8 * i;
#pragma unroll
                    for (int n2 = 0; n2 < 16; ++n2) x[i][n2] = Lb[cl * CLS + 16 * k1 + n2];
                    dft_reg<16, true>(x[i]);
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) __stcg(G + (k1 + 16 * k2) * SN + kx, x[i][k2]);
                }
                group_sync(g, SGT);
            }
            // both groups' columns are in L2 before any row is read
            __syncthreads();
        }
        // --------------------------------------------------------- row phase
        const bool fill_next = !final && (mode == PERIODIC_BEFORE_EACH_FFT ||
                                          (mode == PERIODIC_FINAL_ONLY && it + 1 == iters));
        for (int b = g; b < SN / SL; b += GROUPS) {
            const int m0 = SL * b;
            {
                // this slab's measured slopes into L2 while it is loaded and transformed
                const int p0 = max(0, m0 - off), p1 = min(n, m0 + SL - off);
                if (p1 > p0) {
                    prefetch_lines_l2(sl + p0 * n, size_t(p1 - p0) * n * sizeof(float), tg, SGT);
                    prefetch_lines_l2(sl + nn + p0 * n, size_t(p1 - p0) * n * sizeof(float), tg, SGT);
                }
            }
            // y[i][k2]: cell (row m0 + rl + SL/2 i, column rq + 16 k2)
            float2 y[2][16];
            if (it < 0) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int row = m0 + rl + (SL / 2) * i;
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) {
                        const int cc = rq + 16 * k2, gi = row * SN + cc;
                        float2 v = make_float2(0.f, 0.f);
                        if (ext) {
                            v = make_float2(ext[gi], ext[SN * SN + gi]);
                        } else if (hud) {
                            // Hudgin extension from the measured slopes of the pupil
                            // edges (the pupil cells are overwritten below)
                            const int ii = row - off, j = cc - off;
                            if (j >= 0 && j < n) {
                                const int t = __ldg(hud + j), b2 = __ldg(hud + n + j);
                                if (t >= 0 && (ii < t || ii > b2)) v.x = __ldg(sl + (ii < t ? t : b2) * n + j);
                            }
                            if (ii >= 0 && ii < n) {
                                const int le = __ldg(hud + 2 * n + ii), rt = __ldg(hud + 3 * n + ii);
                                if (le >= 0 && (j < le || j > rt)) v.y = __ldg(sl + nn + ii * n + (j < le ? le : rt));
                            }
                        }
                        y[i][k2] = v;
                    }
                }
            } else {
                // inverse pass A: 16-point DFTs over cells 16 n1 + n2 of the row (n2 = rq)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int row = m0 + rl + (SL / 2) * i;
#pragma unroll
                    for (int n1 = 0; n1 < 16; ++n1) y[i][n1] = __ldcg(G + row * SN + 16 * n1 + rq);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int line = rl + (SL / 2) * i;
                    dft16_tw<true>(y[i], tw16, rq);
#pragma unroll
                    for (int k1 = 0; k1 < 16; ++k1) Lb[line * RLS + RGS * k1 + rq] = y[i][k1];
                }
                group_sync(g, SGT);
                // inverse pass B: cells rq + 16 k2 of the row
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int line = rl + (SL / 2) * i;
#pragma unroll
                    for (int n2 = 0; n2 < 16; ++n2) y[i][n2] = Lb[line * RLS + RGS * rq + n2];
                    dft_reg<16, true>(y[i]);
                }
                if (final) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        float* ph = phase + (m0 + rl + (SL / 2) * i) * SN + rq;
#pragma unroll
                        for (int k2 = 0; k2 < 16; ++k2) __stcs(ph + 16 * k2, y[i][k2].x);
                    }
                    group_sync(g, SGT);
                    continue;
                }
            }
            // Algorithm 1 step 4 (and the embedding): the measurement in the pupil
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int ii = m0 + rl + (SL / 2) * i - off;
                if (ii >= 0 && ii < n) {
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) {
                        const int j = rq + 16 * k2 - off;
                        if (j >= 0 && j < n) {
                            const float vx = __ldg(sl + ii * n + j), vy = __ldg(sl + nn + ii * n + j);
                            if (mask[ii * n + j]) {
                                if (it < 0) finite &= isfinite(vx) && isfinite(vy);
                                y[i][k2] = make_float2(vx, vy);
                            }
                        }
                    }
                }
            }
            if (fill_next) {
                // x part of Eq. PC: the row's last cell takes minus the sum of the
                // other 255; the row's 16 tasks are 16 adjacent lanes
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    float t[16];
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) t[k2] = y[i][k2].x;
                    if (rq == 15) t[15] = 0.f;
#pragma unroll
                    for (int h = 8; h >= 1; h /= 2)
#pragma unroll
                        for (int k = 0; k < h; ++k) t[k] += t[k + h];
                    float sum = t[0];
                    sum += __shfl_xor_sync(half_mask, sum, 1);
                    sum += __shfl_xor_sync(half_mask, sum, 2);
                    sum += __shfl_xor_sync(half_mask, sum, 4);
                    sum += __shfl_xor_sync(half_mask, sum, 8);
                    if (rq == 15) y[i][15].x = -sum;
                }
            }
            // forward pass A on the same registers (cells 16 n1 + n2 with n2 = rq)
            if (it >= 0) group_sync(g, SGT);  // every inverse pass B has read its cells
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int line = rl + (SL / 2) * i;
                dft16_tw<false>(y[i], tw16, rq);
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) Lb[line * RLS + RGS * k1 + rq] = y[i][k1];
            }
            group_sync(g, SGT);
            // forward pass B: cells rq + 16 k2 of the row spectrum back to L2
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int line = rl + (SL / 2) * i;
#pragma unroll
                for (int n2 = 0; n2 < 16; ++n2) y[i][n2] = Lb[line * RLS + RGS * rq + n2];
                dft_reg<16, false>(y[i]);
                float2* const gp = G + (m0 + line) * SN + rq;
#pragma unroll
                for (int k2 = 0; k2 < 16; ++k2) __stcg(gp + 16 * k2, y[i][k2]);
            }
            group_sync(g, SGT);
        }
        // both groups' rows are in L2 before the next column phase (or the next frame)
        __syncthreads();
    }
    return finite;
}
