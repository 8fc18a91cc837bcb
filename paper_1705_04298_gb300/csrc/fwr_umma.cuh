// BF16 GEMM on the 5th-generation tensor cores (sm_103a): D = A B^T with
// A [M][K] and B [N][K] both K-major BF16, D [M][N] row-major (FP32 or BF16),
// FP32 accumulation in tensor memory (TMEM).
//
// Persistent and warp-specialised: one CTA per SM walks the 128 x BN output
// tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (M-tile fastest, so CTAs
// running at the same time share the B tile in L2). Six warps:
//   warp 0, lane 0   producer: TMA loads of the A (BK x 128) and B (BK x BN)
//                    k-blocks (BK = 64 or 32 K elements: one 128- or 64-byte
//                    swizzle row) into a ring of shared-memory stages, across tile
//                    boundaries; completion counted on the stage's "full"
//                    mbarrier
//   warp 1, lane 0   issuer: four tcgen05.mma (M 128, N BN, K 16) per k-block
//                    into one of two TMEM accumulators (2 BN columns in all),
//                    tcgen05.commit to the stage's "empty" mbarrier and, after
//                    a tile's last k-block, to the accumulator's "full" barrier
//   warps 2-5        epilogue (or, with a SplitDst, BF16 terms of each value
//                    written straight into the next product's B operand):
//                    tcgen05.ld of their 32 accumulator lanes
//                    (rows; warp w reads lanes 32 (w mod 4) ..), conversion,
//                    a pass through a swizzled shared tile so that each store
//                    instruction writes four whole 128-byte rows, then an
//                    arrive on the accumulator's "empty" barrier, so the next
//                    tile's MMAs run meanwhile
// With every tile of a CTA on the same A rows and K within four k-blocks, A
// is loaded once per CTA and the stages carry B only (ARES).
// Every mbarrier wait gives up after about two seconds (clock64), sets the
// CTA's abort flag and the caller's status word; the roles then skip their
// work, the producer waits (bounded) for its loads in flight, the issuer for
// its MMAs, and the TMEM is freed before the CTA returns.
//
// Shared-memory operand layout: the canonical K-major swizzled layout that TMA
// writes with CU_TENSOR_MAP_SWIZZLE_128B (64 x rows boxes, rows of 128 bytes,
// 16-byte chunk c of row r at chunk position c ^ (r mod 8)) or _64B (32 x rows
// boxes, rows of 64 bytes, chunk c at c ^ ((r / 2) mod 4)); stage bases are
// 1024-byte aligned. The matrix descriptor carries the start address, the
// 8-row stride (1024 or 512 bytes) and the swizzle mode; the k-th 16-element
// slice of a row is the start address plus 32 k bytes (the swizzle is applied
// to the final address).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fwr {
namespace umma {

constexpr int BM = 128, THREADS = 192;
constexpr long long WAIT_LIMIT = 4000000000LL;  // cycles (about 2 s at 2 GHz)

// Per-(BN, BK) configuration: BN = 128 or 256 output columns per tile, BK =
// 64 K elements per stage (128-byte rows, 128-byte swizzle) or 32 (64-byte
// rows, 64-byte swizzle: half the bytes per stage, twice the stages in the
// same 192 KB, so more TMA latency is covered).
template <int BN, int BK>
struct Cfg {
    static_assert(BN == 128 || BN == 256, "tile width");
    static_assert(BK == 32 || BK == 64, "k-block");
    static constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int STAGES = int(196608u / STAGE_BYTES);
    static constexpr uint32_t TMEM_COLS = 2 * BN;
    // kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
    // K-major, N = BN, M = BM
    static constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(BN >> 3) << 17) | (uint32_t(BM >> 4) << 24);
    // matrix descriptor: 8-row groups 8 x (2 BK) bytes apart; swizzle mode
    // 2 = 128-byte, 4 = 64-byte
    static constexpr uint32_t SBO = 8 * 2 * BK;
    static constexpr uint64_t SWIZZLE = BK == 64 ? 2 : 4;
    // epilogue staging: 32 rows x 128 bytes per epilogue warp
    static constexpr uint32_t EPI_BYTES = 4 * 32 * 128;
    // stages + epilogue staging + 1 KB alignment slack + barriers and flags
    static constexpr size_t SMEM = size_t(STAGES) * STAGE_BYTES + EPI_BYTES + 1024 + 512;
    // resident-A variant (K <= ARES_KB * BK): the CTA's A rows loaded once,
    // the same 192 KB holding them and a ring of B-only stages
    static constexpr int ARES_KB = 4;
    static constexpr int ARES_STAGES = int((uint32_t(STAGES) * STAGE_BYTES - ARES_KB * A_BYTES) / B_BYTES);
    static_assert(ARES_KB * A_BYTES + ARES_STAGES * B_BYTES <= uint32_t(STAGES) * STAGE_BYTES, "resident A fits");
};

__device__ __forceinline__ uint32_t su32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `parity`; false when the CTA aborted or `limit`
// cycles ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort,
                                          long long limit = WAIT_LIMIT) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > limit) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// K-major shared-memory matrix descriptor: start address, 8-row stride sbo,
// swizzle mode
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo, uint64_t swizzle) {
    uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t(1) << 16;            // leading-dimension offset (16 B; not used by swizzled K-major)
    d |= uint64_t(sbo >> 4) << 32;     // stride-dimension offset
    d |= uint64_t(1) << 46;            // descriptor version
    d |= swizzle << 61;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Output values per 128-byte row segment: 32 FP32 or 64 BF16
template <typename OutT>
struct Epi {
    static constexpr int COLS = 128 / int(sizeof(OutT));
};

// Pack 32 FP32 accumulator values as 8 16-byte chunks (FP32) or 4 (BF16).
__device__ __forceinline__ void pack_chunks(const uint32_t (&v)[32], uint4* out, float*) {
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = make_uint4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void pack_chunks(const uint32_t (&v)[32], uint4* out, __nv_bfloat16*) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h =
                __floats2bfloat162_rn(__uint_as_float(v[8 * i + 2 * j]), __uint_as_float(v[8 * i + 2 * j + 1]));
            w[j] = *reinterpret_cast<const uint32_t*>(&h);
        }
        out[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// One 128-byte-wide column segment of a warp's 32 accumulator rows to global
// memory: TMEM -> registers (the lane's row) -> shared tile (16-byte chunk c
// of row r at chunk position c ^ (r mod 8): conflict free both ways) -> rows
// written whole, 8 lanes per 128-byte row, 4 rows per store instruction.
// tw: TMEM address of the warp's lanes at the segment's first column; dst:
// the segment's first column in row m0w (the warp's first row); rows at or
// beyond M are not stored.
template <typename OutT>
__device__ __forceinline__ void epilogue_segment(uint32_t tw, uint4* tile, OutT* dst, long long ldd, int m0w, int M,
                                                 int lane) {
    uint4 ch[8];
    {
        uint32_t v[32];
        tmem_ld32(tw, v);
        pack_chunks(v, ch, static_cast<OutT*>(nullptr));
    }
    if (sizeof(OutT) == 2) {
        uint32_t v[32];
        tmem_ld32(tw + 32u, v);
        pack_chunks(v, ch + 4, static_cast<OutT*>(nullptr));
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) tile[lane * 8 + (c ^ (lane & 7))] = ch[c];
    __syncwarp();
    const int c = lane & 7;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = 4 * i + (lane >> 3);
        if (m0w + r < M) {
            const uint4 val = tile[r * 8 + (c ^ (r & 7))];
            *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(dst + (m0w + r) * ldd) + 16 * c) = val;
        }
    }
    __syncwarp();
}

// Destination of the split epilogue: instead of D[M][ldd] (FP32), each output
// (row i < M = 2n, column (f, x) with f = column / n, x = column mod n) goes
// to the next product's B operand as BF16 terms: row f n + (i mod n) of
// B [.][k], column x + n (i >= n), in each term region of the row (regions of
// 2n entries): 3 terms [hi | lo | hi], 6 terms [h | m | h | l | m | h]. With
// n a multiple of 64, M = 2n is a whole number of 128-row tiles, so every
// accumulator row of a tile is an output row.
struct SplitDst {
    __nv_bfloat16* B = nullptr;
    int n = 0, k = 0, terms = 0;
};

// term t (0: h, 1: m, 2: l) of x: h = bf16(x), m = bf16(x - h), l = bf16(x - h - m)
__device__ __forceinline__ uint32_t split_term_bits(float x, int t) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    if (t == 0) return __bfloat16_as_ushort(h);
    const float r = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r);
    if (t == 1) return __bfloat16_as_ushort(m);
    return __bfloat16_as_ushort(__float2bfloat16_rn(r - __bfloat162float(m)));
}

// One 64-column segment of a warp's 32 accumulator rows to the split
// destination. Per term: the lanes' rows (64 BF16 values, 128 bytes each)
// pass through the warp's swizzled shared tile (16-byte chunk c of row r at
// c ^ (r mod 8)), then each store instruction writes four whole 128-byte rows
// to every term region that holds the term. col0: the segment's first output
// column (a multiple of 64, within one frame since n is a multiple of 64).
__device__ __forceinline__ void epilogue_split_segment(uint32_t tw, uint4* tile, const SplitDst& sd, int m0w,
                                                       int col0, int lane) {
    uint32_t v[64];
    {
        uint32_t (&v0)[32] = *reinterpret_cast<uint32_t(*)[32]>(v);
        uint32_t (&v1)[32] = *reinterpret_cast<uint32_t(*)[32]>(v + 32);
        tmem_ld32(tw, v0);
        tmem_ld32(tw + 32u, v1);
    }
    const int f = col0 / sd.n, x = col0 % sd.n;
    const size_t region = size_t(2 * sd.n);
    const int c = lane & 7;
    const int nterms = sd.terms == 6 ? 3 : 2;
#pragma unroll 1
    for (int t = 0; t < nterms; ++t) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                w[j] = split_term_bits(__uint_as_float(v[8 * q + 2 * j]), t) |
                       (split_term_bits(__uint_as_float(v[8 * q + 2 * j + 1]), t) << 16);
            tile[lane * 8 + (q ^ (lane & 7))] = make_uint4(w[0], w[1], w[2], w[3]);
        }
        __syncwarp();
        // regions of term t: 3 terms [h | m | h]; 6 terms [h | m | h | l | m | h]
        int reg[3], nreg;
        if (sd.terms == 3) {
            nreg = t == 0 ? 2 : 1;
            reg[0] = t == 0 ? 0 : 1;
            reg[1] = 2;
        } else {
            nreg = t == 0 ? 3 : (t == 1 ? 2 : 1);
            reg[0] = t == 0 ? 0 : (t == 1 ? 1 : 3);
            reg[1] = t == 0 ? 2 : 4;
            reg[2] = 5;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = 4 * i + (lane >> 3);
            const uint4 val = tile[r * 8 + (c ^ (r & 7))];
            const int row = m0w + r;
            __nv_bfloat16* const b =
                sd.B + (size_t(f) * sd.n + (row % sd.n)) * sd.k + (row >= sd.n ? sd.n : 0) + x + 8 * c;
            for (int g = 0; g < nreg; ++g) *reinterpret_cast<uint4*>(b + reg[g] * region) = val;
        }
        __syncwarp();
    }
}

// bounded wait without an abort check (draining work already issued)
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, volatile int* abort) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > WAIT_LIMIT) {
            *abort = 1;
            return;
        }
}

// D[M][ldd] = A B^T over K, N a multiple of BN. The maps describe A as {K, M}
// with box {64, 128} and B as {K, N} with box {64, BN}; K beyond the tensors'
// extent and rows beyond M read as zeros (TMA fill) and are not stored.
// wait_limit bounds the MMA issuer's and the epilogue's waits (WAIT_LIMIT in
// normal use; a test passes a few cycles to make them run out); the
// producer's waits and every drain of work in flight keep WAIT_LIMIT.
// SPLIT: the epilogue writes split BF16 terms to sd instead of D (a separate
// instantiation, so the plain products keep their register budget).
// ARES: every tile of the CTA has the same A rows (the launcher guarantees it:
// the grid is a multiple of the M tiles, or one tile per CTA) and K fits
// Cfg::ARES_KB k-blocks: A is loaded once per CTA and the stages carry B only.
template <int BN, int BK, typename OutT, bool SPLIT = false, bool ARES = false>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                int K, OutT* __restrict__ D, long long ldd, int* status, long long wait_limit, SplitDst sd) {
    typedef Cfg<BN, BK> C;
    constexpr int S = ARES ? C::ARES_STAGES : C::STAGES;
    constexpr uint32_t SB = ARES ? C::B_BYTES : C::STAGE_BYTES;       // bytes per stage
    constexpr uint32_t RES = ARES ? C::ARES_KB * C::A_BYTES : 0u;     // resident A ahead of the stages
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* const gbase = smem_raw + (base - raw);
    const uint32_t sbase = base + RES;
    // barriers: full[S], empty[S], acc_full[2], acc_empty[2], mma_done,
    // a_full; then the TMEM address and the abort flag
    uint4* const epi = reinterpret_cast<uint4*>(gbase + C::STAGES * C::STAGE_BYTES);
    uint64_t* const bars = reinterpret_cast<uint64_t*>(gbase + C::STAGES * C::STAGE_BYTES + C::EPI_BYTES);
    uint32_t* const tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);
    volatile int* const abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t full0 = su32(bars), empty0 = full0 + 8 * S, accf0 = empty0 + 8 * S, acce0 = accf0 + 16,
                   mma_done = acce0 + 16, a_full = mma_done + 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + BM - 1) / BM, tiles = tiles_m * (N / BN), kblocks = (K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);  // one arrive per epilogue warp
        }
        mbar_init(mma_done, 1);
        mbar_init(a_full, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    // programmatic dependent launch: the next grid may start its own set-up
    // once every CTA of this one is resident; this grid's inputs are read only
    // after the grid it depends on (if any) has completed
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            // producer
            int it = 0;
            bool ok = true;
            if constexpr (ARES) {
                if (blockIdx.x < tiles) {
                    const int m0 = (blockIdx.x % tiles_m) * BM;
                    mbar_expect_tx(a_full, uint32_t(kblocks) * C::A_BYTES);
                    for (int kb = 0; kb < kblocks; ++kb) tma_load_2d(base + kb * C::A_BYTES, &mapA, kb * BK, m0, a_full);
                }
            }
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int m0 = (t % tiles_m) * BM, n0 = (t / tiles_m) * BN;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % S, use = it / S;
                    if (use > 0 && !mbar_wait(empty0 + 8 * s, uint32_t(use - 1) & 1u, abort)) {
                        ok = false;
                        break;
                    }
                    if constexpr (ARES) {
                        const uint32_t sb = sbase + s * SB;
                        mbar_expect_tx(full0 + 8 * s, C::B_BYTES);
                        tma_load_2d(sb, &mapB, kb * BK, n0, full0 + 8 * s);
                    } else {
                        const uint32_t sa = sbase + s * SB, sb = sa + C::A_BYTES;
                        mbar_expect_tx(full0 + 8 * s, C::STAGE_BYTES);
                        tma_load_2d(sa, &mapA, kb * BK, m0, full0 + 8 * s);
                        tma_load_2d(sb, &mapB, kb * BK, n0, full0 + 8 * s);
                    }
                }
            }
            // every load issued must land before the CTA may exit
            for (int j = it > S ? it - S : 0; j < it; ++j) mbar_drain(full0 + 8 * (j % S), uint32_t(j / S) & 1u, abort);
            if (ARES && blockIdx.x < tiles) mbar_drain(a_full, 0u, abort);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer
            int it = 0, jt = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++jt) {
                const int b = jt & 1, ub = jt >> 1;
                if (ub > 0 && !mbar_wait(acce0 + 8 * b, uint32_t(ub - 1) & 1u, abort, wait_limit)) break;
                fence_after();
                const uint32_t d = tmem + uint32_t(b * BN);
                if (ARES && jt == 0 && !mbar_wait(a_full, 0u, abort, wait_limit)) break;
                for (int kb = 0; kb < kblocks; ++kb, ++it) {
                    const int s = it % S, use = it / S;
                    if (!mbar_wait(full0 + 8 * s, uint32_t(use) & 1u, abort, wait_limit)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t sa = ARES ? base + kb * C::A_BYTES : sbase + s * SB;
                    const uint32_t sb = ARES ? sbase + s * SB : sa + C::A_BYTES;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        mma_bf16(d, sdesc(sa + 32u * k, C::SBO, C::SWIZZLE), sdesc(sb + 32u * k, C::SBO, C::SWIZZLE),
                                 C::IDESC, (kb > 0 || k > 0) ? 1u : 0u);
                    mma_commit(empty0 + 8 * s);
                }
                if (ok) mma_commit(accf0 + 8 * b);
            }
            // the TMEM may be freed only after every MMA issued has completed
            mma_commit(mma_done);
            mbar_drain(mma_done, 0u, abort);
        }
        __syncwarp();
    } else {
        // epilogue
        const int q = warp & 3;
        int jt = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++jt) {
            const int b = jt & 1, ub = jt >> 1;
            const bool ok =
                __all_sync(0xffffffffu, mbar_wait(accf0 + 8 * b, uint32_t(ub) & 1u, abort, wait_limit) && !*abort);
            if (!ok) break;
            fence_after();
            const int m0 = (t % tiles_m) * BM, n0 = (t / tiles_m) * BN;
            const uint32_t tw = tmem + uint32_t(b * BN) + (uint32_t(q * 32) << 16);
            uint4* const tile = epi + (warp - 2) * 256;
            if constexpr (SPLIT) {
#pragma unroll 1
                for (int c = 0; c < BN; c += 64)
                    epilogue_split_segment(tw + uint32_t(c), tile, sd, m0 + q * 32, n0 + c, lane);
            } else {
#pragma unroll 1
                for (int c = 0; c < BN; c += Epi<OutT>::COLS)
                    epilogue_segment<OutT>(tw + uint32_t(c), tile, D + n0 + c, ldd, m0 + q * 32, M, lane);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
    }
    fence_before();
    __syncthreads();
    if (*abort && threadIdx.x == 0) atomicOr(status, 2);
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::TMEM_COLS)
                     : "memory");
    }
}

}  // namespace umma
}  // namespace fwr
