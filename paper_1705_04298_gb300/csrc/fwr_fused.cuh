// Device code of the main fused Gerchberg kernel (fwr_fused.cu), shared with
// the ragged-batch kernel (fwr_ragged.cu). Included inside namespace fwr after
// fwr_fft.cuh.
#pragma once

// Main fused persistent Gerchberg kernel for sm_103a.
//
// One CTA (4N threads) owns one frame at a time and keeps its N x N packed
// grid Z = sx + i sy in shared memory for every iteration of Algorithm 1
// (Sec. 3.3) and for the final reconstruction (Eqs. 2-3). HBM is read for the
// measured slopes and written for the phase only.
//
// 2-D FFT in three register passes (N = 4R):
//   P1  rows, R-point DFT over n1 of elements 4 n1 + n2
//   P2  row twiddle w_N^(n2 k1), rows 4-point DFT over n2  x  columns 4-point
//       DFT over m1 of rows R m1 + m2, column twiddle w_N^(m2 q1)
//   P3  columns, R-point DFT over m2
// Each pass writes back to the cells it read, so the spectrum ends in a
// digit-permuted layout: bin (ky, kx) sits at row R (ky mod 4) + ky / 4 and
// column 4 (kx mod R) + kx / R. The inverse transform runs the passes in
// reverse with conjugate twiddles, ending back in natural order.
//
// Shared-memory layout: cell (row, col) at row * (N + 2) + col; every pass
// addresses its cells as one base register plus compile-time offsets. The row
// stride is 2 mod 16 (in 8-byte cells) and 16-byte aligned, so
//   * the row stage (half-warp = 8 consecutive rows x 2 adjacent columns),
//   * P2 (8 consecutive rows per quarter-warp, 16-byte accesses),
//   * the column stage (32 consecutive columns of one row)
// are all bank-conflict free.
//
// Fusions:
//   * spectral step (Algorithm 1 step 2) sits between the forward and inverse
//     P3: each thread keeps its own bins in registers and reads the partner
//     bins (-k) of the other thread from shared memory;
//   * reinsertion (step 4) and the x part of the periodic fill (Eq. PC) sit
//     between the inverse and the next forward P1 (each row's sum comes from
//     the 4 threads that hold it, through a small shared partial-sum array);
//   * the y part of Eq. PC is applied in the frequency domain: setting the
//     last row of y slopes to minus the column sums adds
//     -Sy(0, kx) e^{2 i pi ky / N} to Sy(ky, kx), a rank-1 correction built
//     from the ky = 0 row of the spectrum. Along one column task's bins it is
//     the P3 DFT of a single input value, so it is added to that input before
//     P3 (the ky = 0 bins are summed from the q1 = 0 inputs first).

namespace {

// s0 staging row stride (elements): n rounded up to 2 mod 16, like the grid,
// so the row stage's reinsertion reads are bank-conflict free.
__host__ __device__ __forceinline__ int s0_stride(int n) { return n + ((18 - (n & 15)) & 15); }

// Row-stage role of a thread: row r, columns 4 n1 + n2. Each warp takes 16
// consecutive rows and 2 adjacent n2.
template <int N>
__device__ __forceinline__ void row_role(int tid, int& r, int& n2) {
    r = (tid >> 1) % N;
    n2 = (tid & 1) + 2 * ((tid >> 1) / N);
}

template <typename T, int N>
struct Layout {
    typedef typename cvec<T>::type V;
    static constexpr int R = N / 4, H = N / 2, S = N + 2;
    static constexpr size_t z = 0;
    static constexpr size_t xpart = z + size_t(N) * S * sizeof(V);
    static constexpr size_t tw = xpart + size_t(4 * N) * sizeof(T);
    static constexpr size_t tw2 = tw + size_t(N) * sizeof(V);
    static constexpr size_t a = tw2 + size_t(3 * R) * sizeof(V);
    static constexpr size_t t = a + size_t(N) * sizeof(V);
    static constexpr size_t pt = t + size_t(N) * sizeof(V);
    static constexpr size_t iota = pt + size_t(4 * N) * sizeof(T);
    static constexpr size_t s0 = (iota + size_t(H + 1) * N * sizeof(T) + 15) & ~size_t(15);
    __host__ __device__ static size_t bytes(int n) { return s0 + size_t(n) * s0_stride(n) * sizeof(V); }
    // optional resident copy of the final-filter half-table (same order as iota), after s0
    __host__ __device__ static size_t wf(int n) { return (bytes(n) + 15) & ~size_t(15); }
    __host__ __device__ static size_t bytes_wf(int n) { return wf(n) + size_t(H + 1) * N * sizeof(T); }
};

// Prefetch [p, p + bytes) into L2, one 128-byte line per thread and step.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const char* b = static_cast<const char*>(p);
    for (size_t o = size_t(threadIdx.x) * 128; o < bytes; o += size_t(blockDim.x) * 128)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(b + o));
}

__device__ __forceinline__ void store4(float* d, float a, float b, float c, float e) {
    *reinterpret_cast<float4*>(d) = make_float4(a, b, c, e);
}
__device__ __forceinline__ void store4(double* d, double a, double b, double c, double e) {
    reinterpret_cast<double2*>(d)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(d)[1] = make_double2(c, e);
}

// four adjacent values of a 16-byte-aligned row, read once (streaming)
__device__ __forceinline__ void load_row4(const float* p, float* v) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
__device__ __forceinline__ void load_row4(const double* p, double* v) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p)), b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

// four adjacent BF16 values (8-byte aligned; a BF16 value is the upper half
// of the FP32 with the same bits, so the widening is exact)
template <typename T>
__device__ __forceinline__ void load_row4(const uint16_t* p, T* v) {
    const uint2 a = __ldcs(reinterpret_cast<const uint2*>(p));
    v[0] = T(__uint_as_float(a.x << 16));
    v[1] = T(__uint_as_float(a.x & 0xFFFF0000u));
    v[2] = T(__uint_as_float(a.y << 16));
    v[3] = T(__uint_as_float(a.y & 0xFFFF0000u));
}

// four adjacent cells (16-byte aligned) in and out
__device__ __forceinline__ void load4(const float2* p, float2* x) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
    x[2] = make_float2(b.x, b.y);
    x[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2* x) {
#pragma unroll
    for (int b = 0; b < 4; ++b) x[b] = p[b];
}
__device__ __forceinline__ void store4c(float2* p, const float2* x) {
    reinterpret_cast<float4*>(p)[0] = make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
    reinterpret_cast<float4*>(p)[1] = make_float4(x[2].x, x[2].y, x[3].x, x[3].y);
}
__device__ __forceinline__ void store4c(double2* p, const double2* x) {
#pragma unroll
    for (int b = 0; b < 4; ++b) p[b] = x[b];
}
// the four separable factors of one frequency (16-byte aligned)
template <typename T> struct quad { T x, y, z, w; };
__device__ __forceinline__ quad<float> load_pt(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ quad<double> load_pt(const double* p) { return {p[0], p[1], p[2], p[3]}; }

__device__ __forceinline__ float mulrn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulrn(double a, double b) { return __dmul_rn(a, b); }

// LSQ projection of one bin pair (Algorithm 1 step 2, formula of Sec. 3.3)
// with the separable factors p(u) = a(u) conj T(u), |a(u)|^2, |T(u)|^2 of the
// bin's column (pux, puy, 2 ha2u = |a(u)|^2, 2 ht2u = |T(u)|^2) and row (pv),
// and w = 1/|G|^2 / N^2: the projected bin is
//   Z'(k) = al z(k) + (be + i ga) conj z(-k),
// al = w (|G|^2/2 + Im P), be = w (|Gx|^2 - |Gy|^2)/2, ga = w Re P, P = p(u)
// conj p(v). Every operation is written out (no contraction left to the
// compiler), so the coefficients come out bitwise the same wherever they are
// computed.
template <typename T>
__device__ __forceinline__ void lsq_coefs(T w, T pux, T puy, T ha2u, T ht2u, const quad<T>& pv, T& al, T& be,
                                          T& ga) {
    const T Py = fmadd(puy, pv.x, -mulrn(pux, pv.y));
    const T ca = fmadd(ha2u, pv.w, fmadd(ht2u, pv.z, Py));
    const T cb = fmadd(ha2u, pv.w, -mulrn(ht2u, pv.z));
    const T cc = fmadd(pux, pv.x, mulrn(puy, pv.y));
    al = mulrn(w, ca);
    be = mulrn(w, cb);
    ga = mulrn(w, cc);
}
template <typename T, typename V>
__device__ __forceinline__ V lsq_apply(T al, T be, T ga, V z1, V z2) {
    return mk(fmadd(al, z1.x, fmadd(be, z2.x, mulrn(ga, z2.y))), fmadd(al, z1.y, fmadd(ga, z2.x, -mulrn(be, z2.y))));
}

// Tensor memory as per-thread storage (32x32b shape: a thread reaches the
// lane of its warp quarter). Stores of 32 and loads of 8 consecutive columns.
__device__ __forceinline__ void tm_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
        "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]),
        "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]),
        "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
        : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t taddr, float (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// Columns of tensor memory the main kernel allocates (the per-thread LSQ
// coefficients: 3 x 32 per thread, four warps per lane quarter)
constexpr uint32_t FUSED_TMEM_COLS = 512;

template <bool INV, typename V>
__device__ __forceinline__ V twiddle(V x, V w) {
    return INV ? cmulc(w, x) : cmul(x, w);
}

// P2 in either direction over all R*R tasks (row radix-4 x column radix-4).
// Task (m2, k1) owns rows R a + m2 and columns 4 k1 + b, a, b = 0..3. The row
// twiddle w_N^(b k1) between P1 and the row radix-4 is applied here, on the
// way in (forward) or out (inverse): three twiddles per task, the same for a
// whole warp, instead of R - 1 per P1 row task.
template <bool INV, int N, typename V>
__device__ __forceinline__ void pass2(V* Z, const V* tw, const V* tw2) {
    constexpr int R = N / 4, S = N + 2, NT = 4 * N, TASKS = R * R, PER = (TASKS + NT - 1) / NT;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = threadIdx.x + i * NT;
        if (TASKS % NT != 0 && t >= TASKS) break;
        const int m2 = t % R, k1 = t / R;
        V* base = Z + m2 * S + 4 * k1;
        V x[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) load4(base + R * S * a, x[a]);
        V wr[3];
#pragma unroll
        for (int b = 1; b < 4; ++b) wr[b - 1] = tw[b * k1];
        if (!INV) {
            // rows: twiddle w_N^(b k1), then 4-point DFT over n2 (second index)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
#pragma unroll
                for (int b = 1; b < 4; ++b) x[a][b] = twiddle<false>(x[a][b], wr[b - 1]);
                dft_reg<4, false>(x[a]);
            }
            // columns: 4-point DFT over m1 (first index), then w_N^(m2 q1)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                V c[4] = {x[0][b], x[1][b], x[2][b], x[3][b]};
                dft_reg<4, false>(c);
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a][b] = c[a];
            }
#pragma unroll
            for (int a = 1; a < 4; ++a) {
                const V w = tw2[(a - 1) * R + m2];
#pragma unroll
                for (int b = 0; b < 4; ++b) x[a][b] = twiddle<false>(x[a][b], w);
            }
        } else {
#pragma unroll
            for (int a = 1; a < 4; ++a) {
                const V w = tw2[(a - 1) * R + m2];
#pragma unroll
                for (int b = 0; b < 4; ++b) x[a][b] = twiddle<true>(x[a][b], w);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                V c[4] = {x[0][b], x[1][b], x[2][b], x[3][b]};
                dft_reg<4, true>(c);
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a][b] = c[a];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                dft_reg<4, true>(x[a]);
#pragma unroll
                for (int b = 1; b < 4; ++b) x[a][b] = twiddle<true>(x[a][b], wr[b - 1]);
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) store4c(base + R * S * a, x[a]);
    }
}

}  // namespace

// Hudgin extension value of grid cell (row, col) outside the pupil, lenslet
// (i, j) = (row - off, col - off): the x slope of the nearer pupil edge of
// its column when above or below the pupil span, the y slope of the nearer
// pupil edge of its row when left or right of it, else 0 (see Params::hud).
// s0 holds the measured slopes of the pupil cells (row stride ns).
template <typename V>
__device__ __forceinline__ V hudgin_cell(const V* s0, int ns, const int16_t* hud, int n, int i, int j) {
    typedef decltype(V().x) T;
    T hx = T(0), hy = T(0);
    if (j >= 0 && j < n) {
        const int t = __ldg(hud + j), b = __ldg(hud + n + j);
        if (t >= 0 && (i < t || i > b)) hx = s0[(i < t ? t : b) * ns + j].x;
    }
    if (i >= 0 && i < n) {
        const int l = __ldg(hud + 2 * n + i), rt = __ldg(hud + 3 * n + i);
        if (l >= 0 && (j < l || j > rt)) hy = s0[i * ns + (j < l ? l : rt)].y;
    }
    return mk(hx, hy);
}

// Per-CTA state of the main kernel for one plan: shared-memory layout and
// the per-thread roles and constants.
template <typename T, int N>
struct FusedCtx {
    typedef typename cvec<T>::type V;
    V* Z;
    T* xpart;
    V* tw;
    V* tw2;
    V* A;
    V* Tt;
    T* pt;
    T* iota;
    V* s0;
    const uint8_t* mask;
    int n, off, nn, ns, mode;
    int r, n2, gam, q1, kx, kxn, gamp;
    V* rowp;
    V* colp;
    const V* partp;
    const V* s0row;
    unsigned pmask;
    V Ax, Tx;
    T pux, puy, a2u, t2u;
    const T* ptv;
    const V* twv;
    const T* iop;
    const T* ion;
    const T* wfp;
    const T* wfn;
    uint32_t tcoef;  // TMC: tensor-memory address of this thread's LSQ coefficients
};

// Load a plan's tables into shared memory and set the per-thread roles.
// Called by every thread of the CTA; ends with a barrier.
// TMC (FP32, one CTA per SM): the LSQ coefficients of the thread's 32 bins are
// computed here once and kept in tensor memory at tmem (the CTA's allocation).
template <typename T, int N, bool TMC = false>
__device__ __forceinline__ void fused_setup(FusedCtx<T, N>& c, unsigned char* smem, const Tables<T>& tab,
                                            const uint8_t* mask, int n, int off, int mode, bool wf_smem = false,
                                            uint32_t tmem = 0) {
    typedef typename cvec<T>::type V;
    typedef Layout<T, N> L;
    constexpr int R = N / 4, NT = 4 * N, H = N / 2, S = L::S;
    V* Z = c.Z = reinterpret_cast<V*>(smem + L::z);
    c.xpart = reinterpret_cast<T*>(smem + L::xpart);
    V* tw = c.tw = reinterpret_cast<V*>(smem + L::tw);
    V* tw2 = c.tw2 = reinterpret_cast<V*>(smem + L::tw2);
    V* A = c.A = reinterpret_cast<V*>(smem + L::a);
    V* Tt = c.Tt = reinterpret_cast<V*>(smem + L::t);
    T* pt = c.pt = reinterpret_cast<T*>(smem + L::pt);
    T* iota = c.iota = reinterpret_cast<T*>(smem + L::iota);
    V* s0 = c.s0 = reinterpret_cast<V*>(smem + L::s0);
    T* const wf = wf_smem ? reinterpret_cast<T*>(smem + L::wf(n)) : nullptr;
    c.mask = mask;
    c.n = n;
    c.off = off;
    c.nn = n * n;
    const int ns = c.ns = s0_stride(n);
    c.mode = mode;
    const int tid = threadIdx.x;

    for (int i = tid; i < N; i += NT) {
        tw[i] = tab.tw[i];
        A[i] = tab.A[i];
        Tt[i] = tab.Tt[i];
    }
    for (int i = tid; i < 4 * N; i += NT) pt[i] = tab.pt[i];
    // 1/|G|^2 weights in storage-column order (entry [ky][col] holds kx(col)),
    // so the lanes of a warp read consecutive words (unrolled: independent
    // loads in flight together)
#pragma unroll 8
    for (int i = tid; i < (H + 1) * N; i += NT) {
        const int col = i % N, src = (i / N) * N + (col >> 2) + R * (col & 3);
        iota[i] = tab.iota[src];
        if (wf) wf[i] = tab.wfin[src];
    }
    __syncthreads();
    for (int i = tid; i < 3 * R; i += NT) tw2[i] = tw[(i % R) * (1 + i / R)];

    // Row stage: row r, columns 4 n1 + n2 (row_role). Column stage: storage
    // column gam = tid mod N, row block q1 = tid / N.
    int r, n2;
    row_role<N>(tid, r, n2);
    const int gam = tid % N, q1 = tid / N;
    c.r = r;
    c.n2 = n2;
    c.gam = gam;
    c.q1 = q1;
    c.rowp = Z + r * S + n2;         // row-stage cells: rowp[4 k1]
    c.colp = Z + R * q1 * S + gam;   // column-stage cells: colp[S m2]
    unsigned pmask = 0;
    {
        const int i = r - off;
        if (i >= 0 && i < n) {
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) {
                const int j = 4 * n1 + n2 - off;
                if (j >= 0 && j < n && mask[i * n + j]) pmask |= 1u << n1;
            }
        }
    }
    c.pmask = pmask;
    c.s0row = s0 + (r - off) * ns + (n2 - off);  // dereferenced only under pmask
    // spectral roles: kx of the storage column and its partner -kx
    const int kx = (gam >> 2) + R * (gam & 3);
    const int kxn = (N - kx) & (N - 1);
    const int gamp = 4 * (kxn % R) + kxn / R;
    const int q1n = (4 - q1) & 3;
    c.kx = kx;
    c.kxn = kxn;
    c.gamp = gamp;
    c.partp = Z + R * q1n * S + gamp;  // partner cells: partp[S q2']
    c.Ax = A[kx];
    c.Tx = Tt[kx];
    // separable factors of the LSQ projection: with P = Gx conj(Gy) = p(u) conj(p(v)),
    // the projected bin is alpha z(k) + beta conj z(-k), alpha = iota (|G|^2/2 + Im P),
    // beta = iota ((|Gx|^2 - |Gy|^2)/2 + i Re P)
    c.pux = pt[4 * kx];
    c.puy = pt[4 * kx + 1];
    c.a2u = pt[4 * kx + 2];
    c.t2u = pt[4 * kx + 3];
    c.ptv = pt + 4 * q1;              // ptv[16 q2 + j] = pt[4 ky + j]
    c.twv = tw + q1;                  // twv[4 q2] = tw[ky]
    c.iop = iota + q1 * N + gam;       // iop[4 N q2] = 1/|G|^2 at (ky, kx)
    c.ion = iota + (N - q1) * N + gamp; // ion[-4 N q2] = 1/|G|^2 at (-ky, -kx)
    // final weights: the resident copy (storage-column order) or the table in global memory
    c.wfp = wf ? wf + q1 * N + gam : tab.wfin + q1 * N + kx;
    c.wfn = wf ? wf + (N - q1) * N + gamp : tab.wfin + (N - q1) * N + kxn;
    if constexpr (TMC) {
        static_assert(sizeof(T) == 4 && N / 4 == 32, "tensor-memory coefficients: FP32, 32 bins per thread");
        // columns: al at +0, be at +32, ga at +64 (bin q2 at + q2); lane quarter warp mod 4
        const int warp = tid >> 5;
        c.tcoef = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(96 * (warp >> 2));
        const T ha2u = T(0.5) * c.a2u, ht2u = T(0.5) * c.t2u;
        // one coefficient at a time (32 live values): al, be, ga
#pragma unroll 1
        for (int which = 0; which < 3; ++which) {
            float v[32];
#pragma unroll
            for (int q2 = 0; q2 < R; ++q2) {
                const bool lo = q2 < R / 2 || (q2 == R / 2 && q1 == 0);
                const T w = lo ? c.iop[4 * N * q2] : c.ion[-4 * N * q2];
                T al, be, ga;
                lsq_coefs(w, c.pux, c.puy, ha2u, ht2u, load_pt(c.ptv + 16 * q2), al, be, ga);
                v[q2] = which == 0 ? al : (which == 1 ? be : ga);
            }
            tm_st32(c.tcoef + uint32_t(32 * which), v);
            tm_wait_st();
        }
    }
    __syncthreads();
}

// One frame through the whole path (embed, iterations, final filter) with
// the state of fused_setup. sl: the frame's [2][n][n] slopes; ext: [2][N][N]
// warm start or nullptr; phase: [N][N] output or nullptr; ext_out: [2][N][N]
// extended slopes or nullptr. Called by every thread; returns false in the
// threads that saw a non-finite measured slope.
template <typename T, int N, bool TMC = false>
__device__ __forceinline__ bool fused_frame(const FusedCtx<T, N>& c, const T* sl, const T* ext,
                                            const uint16_t* exth, T* phase, T* ext_out, int iters,
                                            const int16_t* hud = nullptr) {
    typedef typename cvec<T>::type V;
    constexpr int R = N / 4, NT = 4 * N, S = Layout<T, N>::S;
    const int tid = threadIdx.x;
    V* const Z = c.Z;
    T* const xpart = c.xpart;
    const V* const tw2 = c.tw2;
    const V* const A = c.A;
    const V* const Tt = c.Tt;
    V* const s0 = c.s0;
    const uint8_t* const mask = c.mask;
    const int n = c.n, nn = c.nn, ns = c.ns, mode = c.mode;
    const int r = c.r, n2 = c.n2, gam = c.gam, q1 = c.q1, kx = c.kx, kxn = c.kxn, gamp = c.gamp;
    V* const rowp = c.rowp;
    V* const colp = c.colp;
    const V* const partp = c.partp;
    const V* const s0row = c.s0row;
    const unsigned pmask = c.pmask;
    const V Ax = c.Ax, Tx = c.Tx;
    const T pux = c.pux, puy = c.puy, ha2u = T(0.5) * c.a2u, ht2u = T(0.5) * c.t2u;
    const T* const ptv = c.ptv;
    const V* const twv = c.twv;
    const T* const iop = c.iop;
    const T* const ion = c.ion;
    const T* const wfp = c.wfp;
    const T* const wfn = c.wfn;
    const T half = T(0.5);
    bool finite = true;
    const bool warm = ext || exth;
    if (warm) {
        // warm start: coalesced 4-wide loads of both channels, staged in Z
        // (free between frames) as complex cells
        for (int q = tid; q < N * N / 4; q += NT) {
            const int rr = q / (N / 4), cc = 4 * (q - rr * (N / 4));
            T ex[4], ey[4];
            if (ext) {
                load_row4(ext + rr * N + cc, ex);
                load_row4(ext + N * N + rr * N + cc, ey);
            } else {
                load_row4(exth + rr * N + cc, ex);
                load_row4(exth + N * N + rr * N + cc, ey);
            }
            // two 16-byte stores per four cells (single cells at a 32-byte lane
            // stride would conflict eight ways)
            T* const zp = reinterpret_cast<T*>(Z + rr * S + cc);
            store4(zp, ex[0], ey[0], ex[1], ey[1]);
            store4(zp + 4, ex[2], ey[2], ex[3], ey[3]);
        }
    }
    // measured slopes of the pupil cells into s0: the mask and slope loads do
    // not depend on each other, so unrolled iterations keep them all in flight
#pragma unroll 4
    for (int c = tid; c < nn; c += NT) {
        const uint8_t m = __ldg(mask + c);
        const T vx = sl[c], vy = sl[nn + c];
        if (m) {
            const int i = c / n, j = c - i * n;
            finite &= isfinite(vx) && isfinite(vy);
            s0[i * ns + j] = mk(vx, vy);
        }
    }
    __syncthreads();

    if (hud && !warm) {
        // Hudgin extension staged in Z like a warm start (it needs s0)
        for (int q = tid; q < N * N; q += NT) {
            const int row = q / N, col = q % N;
            Z[row * S + col] = hudgin_cell(s0, ns, hud, n, row - c.off, col - c.off);
        }
        __syncthreads();
    }
    const bool staged = warm || hud;

    // embed: measurement in the pupil, the staged extension (or zero) outside
    V x[R];
#pragma unroll
    for (int n1 = 0; n1 < R; ++n1) {
        if (pmask & (1u << n1)) {
            x[n1] = s0row[4 * n1];
        } else if (staged) {
            x[n1] = rowp[4 * n1];
        } else {
            x[n1] = mk(T(0), T(0));
        }
    }
    // the passes below overwrite Z
    if (staged) __syncthreads();

    for (int it = 0; it <= iters; ++it) {
        const bool final = it == iters;
        // Eq. PC before this forward FFT?
        const bool fill = mode == PERIODIC_BEFORE_EACH_FFT || (mode == PERIODIC_FINAL_ONLY && final);
        if (fill) {
            // x part: last column of x slopes = -(sum of the other N-1 of its row)
            // pairwise sum of the thread's R values (the n2 = 3 thread leaves
            // out the last column)
            T t[R];
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) t[n1] = x[n1].x;
            if (n2 == 3) t[R - 1] = T(0);
#pragma unroll
            for (int h = R / 2; h >= 1; h /= 2)
#pragma unroll
                for (int i = 0; i < h; ++i) t[i] += t[i + h];
            xpart[n2 * N + r] = t[0];
            __syncthreads();
            if (n2 == 3) x[R - 1].x = -(((xpart[r] + xpart[N + r]) + xpart[2 * N + r]) + xpart[3 * N + r]);
        }
        if (final && ext_out) {
            // extended slopes out: finish the fill in direct space first
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) rowp[4 * n1] = x[n1];
            __syncthreads();
            if (fill) {
                for (int c = tid >> 5; c < N; c += NT / 32) {
                    T s = T(0);
                    for (int rr = tid & 31; rr < N - 1; rr += 32) s += Z[rr * S + c].y;
                    s = warp_sum(s);
                    if ((tid & 31) == 0) Z[(N - 1) * S + c].y = -s;
                }
                __syncthreads();
            }
            T* eo = ext_out;
            for (int c = tid; c < N * N; c += NT) {
                const V z = Z[(c / N) * S + c % N];
                eo[c] = z.x;
                eo[N * N + c] = z.y;
            }
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) x[n1] = rowp[4 * n1];
            __syncthreads();
            if (!phase) break;
        }

        // ---- P1 forward: rows, R-point DFT over n1 (its twiddle is applied in P2)
        dft_reg<R, false>(x);
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) rowp[4 * k1] = x[k1];
        __syncthreads();
        // ---- P2 forward
        pass2<false, N>(Z, c.tw, tw2);
        __syncthreads();
        // ---- P3 forward: columns, R-point DFT over m2; bins stay in registers
#pragma unroll
        for (int m2 = 0; m2 < R; ++m2) x[m2] = colp[S * m2];
        if (fill) {
            // y part of Eq. PC: the rank-1 correction -i Sy(0,kx) e^{2 i pi ky / N}
            // of every bin (ky = q1 + 4 q2) is the R-point DFT of one value,
            // d = -i Sy(0,kx) e^{2 i pi q1 / N}, added at m2 = R - 1. Sy(0,kx) =
            // (Z(0,kx) - conj Z(0,-kx)) / (2i) needs the ky = 0 bins, i.e. the
            // sums of the q1 = 0 inputs, published through xpart.
            V* const dc = reinterpret_cast<V*>(xpart);
            if (q1 == 0) {
                V t[R];
#pragma unroll
                for (int m2 = 0; m2 < R; ++m2) t[m2] = x[m2];
#pragma unroll
                for (int h = R / 2; h >= 1; h /= 2)
#pragma unroll
                    for (int i = 0; i < h; ++i) t[i] = cadd(t[i], t[i + h]);
                dc[gam] = t[0];
            }
            __syncthreads();
            const V z0 = dc[gam], z0p = dc[gamp];
            const V ey = mk(half * (z0.y + z0p.y), half * (z0p.x - z0.x));
            const V tq = twv[0];
            const V c0 = cmul(ey, mk(tq.x, -tq.y));
            x[R - 1] = mk(x[R - 1].x + c0.y, x[R - 1].y - c0.x);
        }
        dft_reg<R, false>(x);
#pragma unroll
        for (int q2 = 0; q2 < R; ++q2) colp[S * q2] = x[q2];
        __syncthreads();

        // ---- spectral step on bins ky = q1 + 4 q2, kx
        // partner row of -ky: R q1n + q2n, q2n = R - 1 - q2 (q1 > 0) or R - q2 (q1 = 0, q2 > 0)
        const V* const partq = q1 == 0 ? partp + S : partp;
        // the iterations' projection and the once-per-frame final filter in
        // loops of their own: interleaved per bin, the final filter's code sat
        // inside the iteration's path and overflowed the instruction cache
        // (10 % of the launch time at 128^2)
        if (!final) {
            float tal[8], tbe[8], tga[8];  // TMC: this chunk's coefficients
#pragma unroll
            for (int q2 = 0; q2 < R; ++q2) {
                if constexpr (TMC) {
                    if ((q2 & 7) == 0) {
                        tm_ld8(c.tcoef + q2, tal);
                        tm_ld8(c.tcoef + 32 + q2, tbe);
                        tm_ld8(c.tcoef + 64 + q2, tga);
                        tm_wait_ld();
                    }
                }
                const V z2 = q2 == 0 ? (q1 == 0 ? partp[0] : partp[S * (R - 1)]) : partq[S * (R - 1 - q2)];
                const V z1 = x[q2];
                const bool lo = q2 < R / 2 || (q2 == R / 2 && q1 == 0);
                // Algorithm 1 step 2: LSQ phase, slopes re-synthesised through G
                if constexpr (TMC) {
                    x[q2] = lsq_apply(T(tal[q2 & 7]), T(tbe[q2 & 7]), T(tga[q2 & 7]), z1, z2);
                } else {
                    const T w = lo ? iop[4 * N * q2] : ion[-4 * N * q2];
                    T al, be, ga;
                    lsq_coefs(w, pux, puy, ha2u, ht2u, load_pt(ptv + 16 * q2), al, be, ga);
                    x[q2] = lsq_apply(al, be, ga, z1, z2);
                }
            }
        } else {
#pragma unroll
            for (int q2 = 0; q2 < R; ++q2) {
                const V z2 = q2 == 0 ? (q1 == 0 ? partp[0] : partp[S * (R - 1)]) : partq[S * (R - 1 - q2)];
                const V z1 = x[q2];
                const V z2c = mk(z2.x, -z2.y);
                // ky = 4 q2 + q1 <= N/2: weight stored at (ky, kx); known at
                // compile time except for q2 = N/8
                const bool lo = q2 < R / 2 || (q2 == R / 2 && q1 == 0);
                // Eq. 2: phi = Rx Sx + Ry Sy with 2 Sx = z1 + conj z2, 2 Sy = (z1 - conj z2) / i
                const int ky = q1 + 4 * q2;
                const V sx = cadd(z1, z2c);
                const V dd = csub(z1, z2c);
                const V sy = mk(dd.y, -dd.x);
                const V gx = cmul(Ax, Tt[ky]);
                const V gy = cmul(Tx, A[ky]);
                const T w = half * (lo ? wfp[4 * N * q2] : wfn[-4 * N * q2]);
                const V ph = cadd(cmulc(gx, sx), cmulc(gy, sy));
                x[q2] = mk(ph.x * w, ph.y * w);
            }
        }
        // ---- P3 inverse
        dft_reg<R, true>(x);
        __syncthreads();
#pragma unroll
        for (int m2 = 0; m2 < R; ++m2) colp[S * m2] = x[m2];
        __syncthreads();
        // ---- P2 inverse
        pass2<true, N>(Z, c.tw, tw2);
        __syncthreads();
        // ---- P1 inverse
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) x[k1] = rowp[4 * k1];
        dft_reg<R, true>(x);

        if (!final) {
            // Algorithm 1 step 4: measured slopes back in the pupil (rows
            // without pupil cells skip the loop, whole warps at a time)
            if (pmask) {
#pragma unroll
                for (int n1 = 0; n1 < R; ++n1)
                    if (pmask & (1u << n1)) x[n1] = s0row[4 * n1];
            }
        } else {
            // real phase out through shared memory: every thread has read its
            // row cells, the real parts go to compact rows (stride S values,
            // bank-conflict free for the row roles) in the space of Z, and
            // pairs of values leave with coalesced 8- or 16-byte stores
            __syncthreads();
            T* const Zf = reinterpret_cast<T*>(Z);
            T* const rowf = Zf + r * S + n2;
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) rowf[4 * n1] = x[n1].x;
            __syncthreads();
            V* const ph2 = reinterpret_cast<V*>(phase);
            for (int c = tid; c < N * N / 2; c += NT) {
                const int row = (2 * c) / N, col = (2 * c) % N;
                ph2[c] = *reinterpret_cast<const V*>(Zf + row * S + col);
            }
        }
    }
    return finite;
}

