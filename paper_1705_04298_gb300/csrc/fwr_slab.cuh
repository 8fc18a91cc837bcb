// Device code of the 256^2 slab-streamed Gerchberg kernel (fwr_slab.cu),
// shared with the ragged-batch kernel (fwr_ragged.cu). Included inside
// namespace fwr after fwr_fft.cuh.
#pragma once

// Gerchberg kernel for 256^2 and 512^2 grids (sm_103a): slab-streamed through
// shared memory.
//
// An SN x SN complex grid (512 KB at SN = 256, 2 MB at 512) does not fit one
// SM's shared memory, so each persistent CTA keeps its frame's packed grid
// Z = sx + i sy in its own area of a global scratch buffer (L2 resident at
// 256^2; HBM at 512^2) and works it in slabs of lines:
//
//   row phase, slabs of rows:     inverse row FFTs, reinsertion of the
//                                 measured slopes (Algorithm 1 step 4),
//                                 x part of the periodic fill (Eq. PC),
//                                 forward row FFTs
//   column phase, slabs of cols:  forward column FFTs, y part of Eq. PC as a
//                                 spectral correction, the LSQ projection
//                                 (Sec. 3.3) or the final filter (Eqs. 2-3),
//                                 inverse column FFTs
//
// Column slab s holds SC first-half columns kx in [SC s, SC s + SC) and their
// partners -kx (slab 0 also holds the self-paired column SN/2), so every
// (k, -k) pair of the spectral step lies in one slab.
//
// The CTA's 16 warps form one group or two groups of 8 (the launch shape)
// that work different slabs of the same phase at the same time, each with its
// own shared-memory buffer and named barrier, so one group's memory loads
// overlap the other's arithmetic; a CTA barrier separates the phases.
//
// SN-point line FFTs, SN = 16 RB (RB = 16 or 32): two register passes
// (four-step). Forward: 16-point DFTs over elements RB apart with twiddles
// w_SN^(n2 k1), then RB-point DFTs (output k1 + 16 k2). Inverse, in the
// transposed order: RB-point DFTs over elements 16 apart with the conjugate
// twiddles, then 16-point DFTs (output k1 + RB k2). So the forward transform
// leaves each task exactly the elements the inverse one starts from, and the
// inverse transform each task the elements the forward one starts from. The
// slab data move between the scratch area and registers directly (coalesced
// 8-byte loads and stores: the lanes of a warp take adjacent columns in the
// column phase, 16 or 32 adjacent cells of a row in the row phase), and
// shared memory is used only for the exchanges between the passes:
//   column phase: memory -> pass A -> smem -> pass B -> smem (the partner
//     bins of the spectral step) -> spectral step and inverse pass A in
//     registers -> smem -> inverse pass B -> memory;
//   row phase: memory -> inverse pass A -> smem -> inverse pass B,
//     reinsertion, x fill (row sums by warp shuffles) and forward pass A in
//     registers -> smem -> pass B -> memory.
// That is six crossings of shared memory per column slab and four per row
// slab. Column-phase exchanges use lines SN + 1 cells apart, row-phase ones
// groups of 16 or RB cells padded by one: all bank-conflict free.

namespace {

constexpr int SNT = 512;       // threads per CTA
constexpr int SN = 256;        // the grid of the static-scratch entry point and of ragged batches

// Kernel shape of grid N: GROUPS warp groups (1 or 2) of 512 / GROUPS threads,
// each on its own slab of SL lines at a time.
template <int N, int GROUPS> struct SlabShape {
    static_assert(N == 256 || N == 512, "grid");
    static_assert(GROUPS == 1 || GROUPS == 2, "one or two groups");
    static constexpr int RB = N / 16;                       // size of the long pass
    static constexpr int H = N / 2;
    static constexpr int SL = (N == 256 ? 64 : 32) / GROUPS;  // lines per slab
    static constexpr int SGT = SNT / GROUPS;                // threads per group
    static constexpr int SC = SL / 2;                       // first-half columns of a column slab
    static constexpr int WS = SC + 1;                       // row stride of a group's spectral weights
    static constexpr int CLS = N + 1;                       // column phase: line stride (cells)
    static constexpr int RLS_I = RB * 17;                   // row phase, inverse: groups of 16, stride 17
    static constexpr int RLS_F = 16 * (RB + 1);             // row phase, forward: groups of RB, stride RB + 1
    static constexpr int M1 = SL * CLS > SL * RLS_I ? SL * CLS : SL * RLS_I;
    static constexpr int LB_CELLS = M1 > SL * RLS_F ? M1 : SL * RLS_F;  // one group's buffer
    static constexpr int NA = SL * RB / SGT;                // 16-point tasks per thread and pass
    static constexpr int NB = SL * 16 / SGT;                // RB-point tasks per thread and pass
    static_assert(NA * SGT == SL * RB && NB * SGT == SL * 16, "tasks divide evenly");
};

// Shared-memory layout of the slab path for grid N (the larger shape's
// buffers and weights): bytes, and where each table starts.
template <int N> struct SlabLayout {
    typedef SlabShape<N, 1> S1;
    typedef SlabShape<N, 2> S2;
    static constexpr int RB = N / 16;
    static constexpr size_t lb = 0;
    static constexpr size_t LB_BYTES =
        (size_t(S1::LB_CELLS) > 2 * size_t(S2::LB_CELLS) ? size_t(S1::LB_CELLS) : 2 * size_t(S2::LB_CELLS)) * 8;
    static constexpr size_t tw = lb + LB_BYTES;             // N cells: w_N^j
    static constexpr size_t a = tw + size_t(N) * 8;         // N cells: a(u)
    static constexpr size_t t = a + size_t(N) * 8;          // N cells: T(u)
    static constexpr size_t twa = t + size_t(N) * 8;        // 16 x RB cells: w_N^(n2 k1) at [k1][n2]
    static constexpr size_t twi = twa + size_t(16) * RB * 8;  // RB x 16 cells: w_N^(n2 k1) at [k1][n2]
    static constexpr size_t pt = twi + size_t(16) * RB * 8;   // 4 N floats
    static constexpr size_t WTS = 2 * size_t(S2::WS) * N > size_t(S1::WS) * N ? 2 * size_t(S2::WS) * N
                                                                               : size_t(S1::WS) * N;
    static constexpr size_t wts = pt + size_t(4) * N * 4;
    static constexpr size_t mask = wts + WTS * 4;           // n x n bytes (256^2 only; 512^2 reads global)
    __host__ __device__ static size_t bytes(int n) {
        return mask + (N == 256 ? ((size_t(n) * n + 15) & ~size_t(15)) : 0);
    }
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
// self-paired column N/2 in place of the duplicate 0 in slab 0
template <int N, int SC>
__device__ __forceinline__ int slab_col(int s, int j) {
    if (j < SC) return SC * s + j;
    const int jj = j - SC;
    return (s == 0 && jj == 0) ? N / 2 : (N - SC * s - jj) & (N - 1);
}
// the line holding the partner column -kx of line j (self-paired: columns 0
// and N/2, lines 0 and SC of slab 0)
template <int SC>
__device__ __forceinline__ int partner_line(int s, int j) { return (s == 0 && (j & (SC - 1)) == 0) ? j : (j ^ SC); }

// forward (INV = false) or inverse R-point DFT of x with the twiddle tws[k]
// (conjugated for the inverse) applied to output k; tws points at the
// task's column of a [k][n2] table with row stride `stride`
template <int R, bool INV>
__device__ __forceinline__ void dft_tw(float2 (&x)[R], const float2* tws, int stride) {
    dft_reg<R, INV>(x);
#pragma unroll
    for (int k = 1; k < R; ++k) {
        const float2 w = tws[stride * k];
        x[k] = INV ? cmulc(w, x[k]) : cmul(x[k], w);
    }
}

}  // namespace

// Shared-memory bytes of the slab path for grid N (256 or 512) and n lenslets.
__host__ __device__ __forceinline__ size_t slab_layout_bytes_n(int N, int n) {
    return N == 512 ? SlabLayout<512>::bytes(n) : SlabLayout<256>::bytes(n);
}
__host__ __device__ __forceinline__ size_t slab_layout_bytes(int n) { return SlabLayout<256>::bytes(n); }

// Per-CTA state of the slab path for one plan.
struct SlabCtx {
    float2* Lb;    // the groups' buffers
    float2* tw;    // w_N^j
    float2* A;
    float2* Tt;
    float2* twa;   // w_N^(n2 k1) at [k1][n2], k1 < 16, n2 < RB (forward pass A)
    float2* twi;   // w_N^(n2 k1) at [k1][n2], k1 < RB, n2 < 16 (inverse pass A)
    float* pt;
    float* wts;    // the groups' weight tables
    const uint8_t* mask;  // shared memory (256^2) or the plan's global copy (512^2)
    int n, off, nn, mode;
};

// Load a plan's 1-D tables (and at 256^2 the mask) into shared memory; ends
// with a barrier.
template <int N>
__device__ __forceinline__ void slab_setup(SlabCtx& c, unsigned char* smem, const Tables<float>& tab,
                                           const uint8_t* mask_g, int n, int off, int mode) {
    typedef SlabLayout<N> L;
    constexpr int RB = N / 16;
    c.Lb = reinterpret_cast<float2*>(smem + L::lb);
    c.tw = reinterpret_cast<float2*>(smem + L::tw);
    c.A = reinterpret_cast<float2*>(smem + L::a);
    c.Tt = reinterpret_cast<float2*>(smem + L::t);
    c.twa = reinterpret_cast<float2*>(smem + L::twa);
    c.twi = reinterpret_cast<float2*>(smem + L::twi);
    c.pt = reinterpret_cast<float*>(smem + L::pt);
    c.wts = reinterpret_cast<float*>(smem + L::wts);
    c.n = n;
    c.off = off;
    c.nn = n * n;
    c.mode = mode;
    const int tid = threadIdx.x;
    for (int i = tid; i < N; i += SNT) {
        c.tw[i] = tab.tw[i];
        c.A[i] = tab.A[i];
        c.Tt[i] = tab.Tt[i];
    }
    for (int i = tid; i < 4 * N; i += SNT) c.pt[i] = tab.pt[i];
    for (int i = tid; i < 16 * RB; i += SNT) {
        c.twa[i] = tab.tw[(i % RB) * (i / RB)];  // [k1][n2], k1 < 16
        c.twi[i] = tab.tw[(i % 16) * (i / 16)];  // [k1][n2], n2 < 16
    }
    if (N == 256) {
        uint8_t* m = smem + L::mask;
#pragma unroll 8
        for (int i = tid; i < c.nn; i += SNT) m[i] = mask_g[i];
        c.mask = m;
    } else {
        c.mask = mask_g;
    }
    __syncthreads();
}

// One frame through the whole path with the grid in G (this CTA's N^2
// scratch area). sl: [2][n][n] slopes; ext: [2][N][N] warm start or nullptr;
// phase: [N][N] output. Called by every thread; returns false in the threads
// that saw a non-finite measured slope.
//
// Tasks (t: the thread's index in its group, i: its task): column phase,
// line t mod SL and pass index q = t / SL + (SGT / SL) i; row phase, 16-cell
// tasks (inverse pass B, forward pass A) take index t mod RB and line
// t / RB + (SGT / RB) i, RB-cell tasks (inverse pass A, forward pass B) index
// t mod 16 and line t / 16 + (SGT / 16) i. Both shapes give bitwise the same
// result (each line transform and each bin's arithmetic is the same).
template <int N, int GROUPS>
__device__ __forceinline__ bool slab_frame(const SlabCtx& c, const Tables<float>& tab, const float* sl,
                                           const float* ext, float* phase, int iters, float2* G,
                                           const int16_t* hud = nullptr) {
    typedef SlabShape<N, GROUPS> Sh;
    constexpr int SL = Sh::SL, SGT = Sh::SGT, SC = Sh::SC, WS = Sh::WS, RB = Sh::RB, H = Sh::H;
    constexpr int CLS = Sh::CLS, RLS_I = Sh::RLS_I, RLS_F = Sh::RLS_F, NA = Sh::NA, NB = Sh::NB;
    const int g = threadIdx.x / SGT, tg = threadIdx.x % SGT;
    float2* const Lb = c.Lb + g * Sh::LB_CELLS;
    const float2* const tw = c.tw;
    const float2* const twa = c.twa;
    const float2* const twi = c.twi;
    const float2* const A = c.A;
    const float2* const Tt = c.Tt;
    const float* const pt = c.pt;
    float* const wts = c.wts + g * WS * N;
    const uint8_t* const mask = c.mask;
    const int n = c.n, off = c.off, nn = c.nn, mode = c.mode;
    bool finite = true;
    // column-phase roles: line cl, pass index cq + (SGT / SL) i
    const int cl = tg % SL, cq = tg / SL;
    constexpr int CQS = SGT / SL;
    // row-phase roles
    const int r16 = tg % 16, l16 = tg / 16;   // RB-cell tasks
    const int rrb = tg % RB, lrb = tg / RB;   // 16-cell tasks
    constexpr int L16S = SGT / 16, LRBS = SGT / RB;
    // the RB lanes of one row's 16-cell tasks (for the x-fill row sums)
    const unsigned row_mask = RB == 32 ? 0xFFFFFFFFu : (0xFFFFu << (threadIdx.x & 16));
    // it = -1: embed; it = 0 .. iters-1: Gerchberg; it = iters: final
    for (int it = -1; it <= iters; ++it) {
        const bool final = it == iters;
        if (it >= 0) {
            // ------------------------------------------------ column phase
            const bool fill = mode == PERIODIC_BEFORE_EACH_FFT || (mode == PERIODIC_FINAL_ONLY && final);
            for (int s = g; s < N / SL; s += GROUPS) {
                const int kx = slab_col<N, SC>(s, cl);
                const int pl = partner_line<SC>(s, cl);
                {
                    // spectral weights of the first-half columns: wts[ky][j] at
                    // (ky, kx) from the half-table (rows 0..N/2; (-ky, -kx) beyond)
                    const float* wt = final ? tab.wfin : tab.iota;
                    const int j = tg % SC, kxj = slab_col<N, SC>(s, j), kxn = (N - kxj) & (N - 1);
                    for (int k = tg / SC; k < N; k += SGT / SC)
                        cp_async4(wts + k * WS + j, wt + (k <= H ? k * N + kxj : (N - k) * N + kxn));
                    if (s == 0)  // line SC: the self-paired column N/2
                        for (int k = tg; k < N; k += SGT)
                            cp_async4(wts + k * WS + SC, wt + (k <= H ? k : N - k) * N + H);
                }
                // pass A: 16-point DFTs over rows RB n1 + n2 of the column, from memory
                {
                    float2 x[NA][16];
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        const int n2 = cq + CQS * i;
#pragma unroll
                        for (int n1 = 0; n1 < 16; ++n1) x[i][n1] = __ldcg(G + (RB * n1 + n2) * N + kx);
                    }
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        const int n2 = cq + CQS * i;
                        dft_tw<16, false>(x[i], twa + n2, RB);
#pragma unroll
                        for (int k1 = 0; k1 < 16; ++k1) Lb[cl * CLS + RB * k1 + n2] = x[i][k1];
                    }
                }
                group_sync(g, SGT);
                // pass B: bins ky = k1 + 16 k2 of the column
                float2 y[NB][RB];
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int k1 = cq + CQS * i;
#pragma unroll
                    for (int n2 = 0; n2 < RB; ++n2) y[i][n2] = Lb[cl * CLS + RB * k1 + n2];
                    dft_reg<RB, false>(y[i]);
                }
                group_sync(g, SGT);
                // the spectrum in natural order, for the partner bins
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int k1 = cq + CQS * i;
#pragma unroll
                    for (int k2 = 0; k2 < RB; ++k2) Lb[cl * CLS + k1 + 16 * k2] = y[i][k2];
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
                const int wcol = (s == 0 && cl == SC) ? SC : (cl % SC);
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int k1 = cq + CQS * i;
#pragma unroll
                    for (int k2 = 0; k2 < RB; ++k2) {
                        const int ky = k1 + 16 * k2, kyn = (N - ky) & (N - 1);
                        float2 z1 = y[i][k2], z2 = Lb[pl * CLS + kyn];
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
                            y[i][k2] = make_float2(w * ox, w * oy);
                        } else {
                            // Eq. 2 with the final filter: phi = w (conj(Gx) Sx + conj(Gy) Sy)
                            const float2 z2c = conjf2(z2);
                            const float2 sx = make_float2(0.5f * (z1.x + z2c.x), 0.5f * (z1.y + z2c.y));
                            const float2 sy = make_float2(0.5f * (z1.y - z2c.y), 0.5f * (z2c.x - z1.x));
                            const float2 gx = cmul(Akx, Tt[ky]);
                            const float2 gy = cmul(Tkx, A[ky]);
                            const float2 ph = cadd(cmulc(gx, sx), cmulc(gy, sy));
                            y[i][k2] = make_float2(ph.x * w, ph.y * w);
                        }
                    }
                    // inverse pass A: the bins ky = 16 n1 + n2 with n2 = k1
                    dft_tw<RB, true>(y[i], twi + k1, 16);
                }
                group_sync(g, SGT);
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int n2 = cq + CQS * i;
#pragma unroll
                    for (int k1 = 0; k1 < RB; ++k1) Lb[cl * CLS + 16 * k1 + n2] = y[i][k1];
                }
                group_sync(g, SGT);
                // inverse pass B, rows k1 + RB k2 of the column back to memory
                {
                    float2 x[NA][16];
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        const int k1 = cq + CQS * i;
#pragma unroll
                        for (int n2 = 0; n2 < 16; ++n2) x[i][n2] = Lb[cl * CLS + 16 * k1 + n2];
                        dft_reg<16, true>(x[i]);
#pragma unroll
                        for (int k2 = 0; k2 < 16; ++k2) __stcg(G + (k1 + RB * k2) * N + kx, x[i][k2]);
                    }
                }
                group_sync(g, SGT);
            }
            // both groups' columns are in memory before any row is read
            __syncthreads();
        }
        // --------------------------------------------------------- row phase
        const bool fill_next = !final && (mode == PERIODIC_BEFORE_EACH_FFT ||
                                          (mode == PERIODIC_FINAL_ONLY && it + 1 == iters));
        for (int b = g; b < N / SL; b += GROUPS) {
            const int m0 = SL * b;
            {
                // this slab's measured slopes into L2 while it is loaded and transformed
                const int p0 = max(0, m0 - off), p1 = min(n, m0 + SL - off);
                if (p1 > p0) {
                    prefetch_lines_l2(sl + p0 * n, size_t(p1 - p0) * n * sizeof(float), tg, SGT);
                    prefetch_lines_l2(sl + nn + p0 * n, size_t(p1 - p0) * n * sizeof(float), tg, SGT);
                }
            }
            // x[i][k2]: cell (row m0 + lrb + LRBS i, column rrb + RB k2)
            float2 x[NA][16];
            if (it < 0) {
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const int row = m0 + lrb + LRBS * i;
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) {
                        const int cc = rrb + RB * k2, gi = row * N + cc;
                        float2 v = make_float2(0.f, 0.f);
                        if (ext) {
                            v = make_float2(ext[gi], ext[N * N + gi]);
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
                        x[i][k2] = v;
                    }
                }
            } else {
                // inverse pass A: RB-point DFTs over cells 16 n1 + n2 of the row (n2 = r16)
                {
                    float2 y[NB][RB];
#pragma unroll
                    for (int i = 0; i < NB; ++i) {
                        const int row = m0 + l16 + L16S * i;
#pragma unroll
                        for (int n1 = 0; n1 < RB; ++n1) y[i][n1] = __ldcg(G + row * N + 16 * n1 + r16);
                    }
#pragma unroll
                    for (int i = 0; i < NB; ++i) {
                        const int line = l16 + L16S * i;
                        dft_tw<RB, true>(y[i], twi + r16, 16);
#pragma unroll
                        for (int k1 = 0; k1 < RB; ++k1) Lb[line * RLS_I + 17 * k1 + r16] = y[i][k1];
                    }
                }
                group_sync(g, SGT);
                // inverse pass B: cells rrb + RB k2 of the row
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const int line = lrb + LRBS * i;
#pragma unroll
                    for (int n2 = 0; n2 < 16; ++n2) x[i][n2] = Lb[line * RLS_I + 17 * rrb + n2];
                    dft_reg<16, true>(x[i]);
                }
                if (final) {
#pragma unroll
                    for (int i = 0; i < NA; ++i) {
                        float* ph = phase + (m0 + lrb + LRBS * i) * N + rrb;
#pragma unroll
                        for (int k2 = 0; k2 < 16; ++k2) __stcs(ph + RB * k2, x[i][k2].x);
                    }
                    group_sync(g, SGT);
                    continue;
                }
            }
            // Algorithm 1 step 4 (and the embedding): the measurement in the pupil
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                const int ii = m0 + lrb + LRBS * i - off;
                if (ii >= 0 && ii < n) {
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) {
                        const int j = rrb + RB * k2 - off;
                        if (j >= 0 && j < n) {
                            const float vx = __ldg(sl + ii * n + j), vy = __ldg(sl + nn + ii * n + j);
                            if (mask[ii * n + j]) {
                                if (it < 0) finite &= isfinite(vx) && isfinite(vy);
                                x[i][k2] = make_float2(vx, vy);
                            }
                        }
                    }
                }
            }
            if (fill_next) {
                // x part of Eq. PC: the row's last cell takes minus the sum of the
                // other N - 1; the row's RB tasks are RB adjacent lanes
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    float t[16];
#pragma unroll
                    for (int k2 = 0; k2 < 16; ++k2) t[k2] = x[i][k2].x;
                    if (rrb == RB - 1) t[15] = 0.f;
#pragma unroll
                    for (int h = 8; h >= 1; h /= 2)
#pragma unroll
                        for (int k = 0; k < h; ++k) t[k] += t[k + h];
                    float sum = t[0];
#pragma unroll
                    for (int o = 1; o < RB; o *= 2) sum += __shfl_xor_sync(row_mask, sum, o);
                    if (rrb == RB - 1) x[i][15].x = -sum;
                }
            }
            // forward pass A on the same registers (cells RB n1 + n2 with n2 = rrb)
            if (it >= 0) group_sync(g, SGT);  // every inverse pass B has read its cells
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                const int line = lrb + LRBS * i;
                dft_tw<16, false>(x[i], twa + rrb, RB);
#pragma unroll
                for (int k1 = 0; k1 < 16; ++k1) Lb[line * RLS_F + (RB + 1) * k1 + rrb] = x[i][k1];
            }
            group_sync(g, SGT);
            // forward pass B: cells r16 + 16 k2 of the row spectrum back to memory
            {
                float2 y[NB][RB];
#pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int line = l16 + L16S * i;
#pragma unroll
                    for (int n2 = 0; n2 < RB; ++n2) y[i][n2] = Lb[line * RLS_F + (RB + 1) * r16 + n2];
                    dft_reg<RB, false>(y[i]);
                    float2* const gp = G + (m0 + line) * N + r16;
#pragma unroll
                    for (int k2 = 0; k2 < RB; ++k2) __stcg(gp + 16 * k2, y[i][k2]);
                }
            }
            group_sync(g, SGT);
        }
        // both groups' rows are in memory before the next column phase (or the next frame)
        __syncthreads();
    }
    return finite;
}
