// Warm-start network for the Gerchberg loop (sm_103a): a small U-Net that
// predicts the slopes outside the pupil from the measured ones, so that one
// or two iterations of Algorithm 1 (Sec. 3.3) start close to the converged
// extension. The paper has no learned component; this is the project's
// addition.
//
// Definition (input 3 x 32 x 32, output 2 x 32 x 32):
//   input    sx P, sy P (times IN_SCALE) and P on the 128^2 grid, averaged
//            over 4 x 4 blocks
//   levels   widths (w, 2w, 4w, 4w); two 3 x 3 convolutions (zero padding,
//            bias, ReLU) per level; 2 x 2 average pooling down; decoder
//            convolutions read [nearest-upsampled previous, skip] as one
//            concatenated input
//   output   1 x 1 convolution to 2 channels; divided by IN_SCALE and repeated
//            over 4 x 4 blocks it is the warm start outside the pupil
// Storage: activations NHWC in BF16, weights W[cout][dy][dx][cin] in BF16
// (FP32 master copy for Adam), every sum accumulated in FP32, gradients of
// activations in FP32. The forward 3 x 3 convolutions whose input channel
// groups are multiples of 16 (and output channels of 8) run on the tensor
// cores as implicit GEMMs (mma.sync m16n8k16, BF16 in, FP32 accumulate); the
// first and last layers, the backward pass and the small elementwise kernels
// are SIMT.

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/fwr.h"
#include "fwr_internal.h"
#include "fwr_plan.h"

namespace fwr {
namespace net {

constexpr float IN_SCALE = 0.5f;
constexpr int GRID = 128, LOW = 32, POOL = 4;

typedef __nv_bfloat16 bf16;

// ----------------------------------------------------------------- kernels --

// slopes [F][2][n][n] -> X [F][32][32][3]
__global__ void k_input(const float* sl, const uint8_t* mask, int n, int off, int F, bf16* X) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * LOW * LOW) return;
    const int f = idx / (LOW * LOW), Y = (idx / LOW) % LOW, Xc = idx % LOW;
    const float* s = sl + size_t(f) * 2 * n * n;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int i = 0; i < POOL; ++i)
        for (int j = 0; j < POOL; ++j) {
            const int bi = POOL * Y + i - off, bj = POOL * Xc + j - off;
            if (bi >= 0 && bi < n && bj >= 0 && bj < n && mask[bi * n + bj]) {
                a0 += s[bi * n + bj];
                a1 += s[n * n + bi * n + bj];
                a2 += 1.f;
            }
        }
    const float k = 1.f / (POOL * POOL);
    bf16* o = X + size_t(idx) * 3;
    o[0] = __float2bfloat16(a0 * IN_SCALE * k);
    o[1] = __float2bfloat16(a1 * IN_SCALE * k);
    o[2] = __float2bfloat16(a2 * k);
}

// extended slopes [F][2][128][128] -> target [F][32][32][2], loss mask [F][32][32]
__global__ void k_target(const float* ext, const uint8_t* mask, int n, int off, int F, float* T, float* LM) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * LOW * LOW) return;
    const int f = idx / (LOW * LOW), Y = (idx / LOW) % LOW, Xc = idx % LOW;
    const float* e = ext + size_t(f) * 2 * GRID * GRID;
    float a0 = 0.f, a1 = 0.f;
    bool pupil = false;
    for (int i = 0; i < POOL; ++i)
        for (int j = 0; j < POOL; ++j) {
            const int m = POOL * Y + i, c = POOL * Xc + j;
            a0 += e[m * GRID + c];
            a1 += e[GRID * GRID + m * GRID + c];
            const int bi = m - off, bj = c - off;
            pupil |= bi >= 0 && bi < n && bj >= 0 && bj < n && mask[bi * n + bj];
        }
    const float k = IN_SCALE / (POOL * POOL);
    T[2 * idx] = a0 * k;
    T[2 * idx + 1] = a1 * k;
    LM[idx] = (!pupil && Y != LOW - 1 && Xc != LOW - 1) ? 1.f : 0.f;
}

// 3 x 3 (K = 3) or 1 x 1 (K = 1) convolution. The input is the channel
// concatenation of A (ca channels; at half resolution when upA, read with
// nearest upsampling) and B (cb channels, may be null). Output: BF16 (relu'd
// when relu) or FP32. One block per (image, output row); each thread computes
// XG adjacent pixels of one output channel.
template <int K>
__global__ void k_conv_fwd(const bf16* A, int ca, bool upA, const bf16* Bt, int cb, int H, int W,
                           const bf16* Wt, const float* bias, int cout, bool relu, bf16* out_bf, float* out_f) {
    extern __shared__ float rows[];  // [K][W + 2][cin]
    const int cin = ca + cb;
    const int b = blockIdx.x / H, y = blockIdx.x % H;
    const int pad = K / 2, RW = W + 2 * pad;
    for (int i = threadIdx.x; i < K * RW * cin; i += blockDim.x) {
        const int r = i / (RW * cin), xx = (i / cin) % RW, c = i % cin;
        const int yy = y + r - pad, xc = xx - pad;
        float v = 0.f;
        if (yy >= 0 && yy < H && xc >= 0 && xc < W) {
            if (c < ca) {
                v = upA ? __bfloat162float(A[((size_t(b) * (H / 2) + yy / 2) * (W / 2) + xc / 2) * ca + c])
                        : __bfloat162float(A[((size_t(b) * H + yy) * W + xc) * ca + c]);
            } else {
                v = __bfloat162float(Bt[((size_t(b) * H + yy) * W + xc) * cb + (c - ca)]);
            }
        }
        rows[i] = v;
    }
    __syncthreads();
    constexpr int XG = 4;
    const int groups = (W + XG - 1) / XG;
    for (int t = threadIdx.x; t < cout * groups; t += blockDim.x) {
        const int co = t / groups, x0 = (t % groups) * XG;
        float acc[XG];
        for (int g = 0; g < XG; ++g) acc[g] = bias[co];
        for (int dy = 0; dy < K; ++dy)
            for (int dx = 0; dx < K; ++dx) {
                const bf16* w = Wt + ((size_t(co) * K + dy) * K + dx) * cin;
                for (int c = 0; c < cin; ++c) {
                    const float wv = __bfloat162float(w[c]);
#pragma unroll
                    for (int g = 0; g < XG; ++g)
                        if (x0 + g < W) acc[g] += wv * rows[(dy * RW + x0 + g + dx) * cin + c];
                }
            }
        for (int g = 0; g < XG; ++g) {
            if (x0 + g >= W) break;
            const size_t o = ((size_t(b) * H + y) * W + x0 + g) * cout + co;
            const float v = relu ? fmaxf(acc[g], 0.f) : acc[g];
            if (out_bf) out_bf[o] = __float2bfloat16(v);
            else out_f[o] = v;
        }
    }
}

// ---------------------------------------------- tensor-core convolution --
//
// Implicit GEMM: rows = output pixels, columns = output channels, reduction
// K = 9 cin ordered (tap, channel). A CTA of 4 warps owns TC_TM consecutive
// output pixels in (image, row, column) order, i.e. TC_TM / W whole rows; it
// stages those rows with one halo row above and below and one zero column on
// each side, channels [A (upsampled when upA) | B] with 8 padding channels per
// pixel (an odd number of 16-byte units per pixel keeps the 8 row reads of an
// ldmatrix on distinct banks). Each warp computes 32 pixels (two m16 tiles) by
// 8 NT channels; A fragments come from the halo with ldmatrix, B fragments
// from the packed weights (one 8-byte load per lane per n8 tile). A tap that
// falls above the first or below the last row of its image reads a zero
// block instead; the zero columns cover the left and right edges.

constexpr int TC_TM = 128, TC_THREADS = 128;

__device__ __forceinline__ void ldsm_x4(uint32_t (&a)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory bytes of k_conv_tc for a layer (W = H)
inline size_t tc_smem_bytes(int H, int cin) {
    return size_t(TC_TM / H + 2) * (H + 2) * (cin + 8) * sizeof(bf16) + 32;
}

// Packed weights of one 3 x 3 layer: Wp[(kc * cout / 8 + nt) * 32 + lane] holds
// the two B-fragment registers of lane (g, t) = (lane / 4, lane % 4) for the
// reduction chunk kc = tap * cin / 16 + c0 / 16 and the n8 tile nt:
// {W[co][tap][c0 + 2t, c0 + 2t + 1], W[co][tap][c0 + 8 + 2t, c0 + 9 + 2t]},
// co = 8 nt + g.
__global__ void k_pack_tc(const bf16* Wb, int cin, int cout, uint2* Wp) {
    const int ntt = cout / 8, kcs = cin / 16;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * kcs * ntt * 32) return;
    const int lane = i & 31, nt = (i >> 5) % ntt, kc = (i >> 5) / ntt;
    const int tap = kc / kcs, c0 = (kc % kcs) * 16;
    const int co = nt * 8 + (lane >> 2), t = lane & 3;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(Wb + (size_t(co) * 9 + tap) * cin + c0 + 2 * t);
    Wp[i] = make_uint2(src[0], src[4]);
}

template <int NT>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const bf16* __restrict__ A, int ca, int upA,
                                                        const bf16* __restrict__ Bs, int cb, int H,
                                                        const uint2* __restrict__ Wp, const float* __restrict__ bias,
                                                        int cout, int relu, int npix, bf16* __restrict__ out) {
    extern __shared__ __align__(16) bf16 halo[];
    const int W = H, cin = ca + cb, PS = cin + 8, RW = W + 2, rows = TC_TM / W + 2;
    const int P0 = blockIdx.x * TC_TM, g0 = P0 / W, grows = npix / W;
    const int zoff = rows * RW * PS;
    const int cv = cin >> 3;
    for (int i = threadIdx.x; i < rows * RW * cv; i += TC_THREADS) {
        const int v = i % cv, c = (i / cv) % RW, r = i / (cv * RW);
        const int gr = g0 - 1 + r, x = c - 1, ch = v * 8;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (gr >= 0 && gr < grows && x >= 0 && x < W) {
            if (ch < ca) {
                size_t pix = size_t(gr) * W + x;
                if (upA) {
                    const int b = gr / H, y = gr - b * H;
                    pix = (size_t(b) * (H / 2) + y / 2) * (W / 2) + x / 2;
                }
                val = __ldg(reinterpret_cast<const uint4*>(A + pix * ca + ch));
            } else {
                val = __ldg(reinterpret_cast<const uint4*>(Bs + (size_t(gr) * W + x) * cb + (ch - ca)));
            }
        }
        *reinterpret_cast<uint4*>(halo + (r * RW + c) * PS + ch) = val;
    }
    if (threadIdx.x < 4) reinterpret_cast<uint2*>(halo + zoff)[threadIdx.x] = make_uint2(0u, 0u);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kh = (lane >> 4) * 8;
    const uint32_t sbase = uint32_t(__cvta_generic_to_shared(halo));
    int hoff[2], yf[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int p = P0 + warp * 32 + j * 16 + (lane & 15);
        const int gr = p / W, x = p - gr * W, y = gr % H;
        hoff[j] = ((gr - g0) * RW + x) * PS + kh;
        yf[j] = (y == 0 ? 1 : 0) | (y == H - 1 ? 2 : 0);
    }
    float acc[2][NT][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[j][nt][0] = acc[j][nt][1] = acc[j][nt][2] = acc[j][nt][3] = 0.f;

    const int ntt = cout / 8;
    const uint2* wp = Wp + size_t(blockIdx.y) * NT * 32 + lane;
    int kc = 0;
    for (int dy = 0; dy < 3; ++dy) {
        bool ok[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) ok[j] = !((dy == 0 && (yf[j] & 1)) || (dy == 2 && (yf[j] & 2)));
        for (int dx = 0; dx < 3; ++dx) {
            uint32_t ad[2], inc[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                ad[j] = sbase + 2u * uint32_t(ok[j] ? hoff[j] + (dy * RW + dx) * PS : zoff + kh);
                inc[j] = ok[j] ? 32u : 0u;
            }
            for (int c0 = 0; c0 < cin; c0 += 16, ++kc) {
                uint32_t a[2][4];
                ldsm_x4(a[0], ad[0]);
                ldsm_x4(a[1], ad[1]);
                ad[0] += inc[0];
                ad[1] += inc[1];
                const uint2* wk = wp + size_t(kc) * ntt * 32;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const uint2 b = __ldg(wk + nt * 32);
                    mma_16816(acc[0][nt], a[0], b.x, b.y);
                    mma_16816(acc[1][nt], a[1], b.x, b.y);
                }
            }
        }
    }

    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int co = (blockIdx.y * NT + nt) * 8 + 2 * t;
        const float b0 = bias[co], b1 = bias[co + 1];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int p = P0 + warp * 32 + j * 16 + g + 8 * hh;
                if (p >= npix) continue;
                float v0 = acc[j][nt][2 * hh] + b0, v1 = acc[j][nt][2 * hh + 1] + b1;
                if (relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                *reinterpret_cast<__nv_bfloat162*>(out + size_t(p) * cout + co) = __floats2bfloat162_rn(v0, v1);
            }
    }
}

// g <- g * (a > 0)
__global__ void k_relu_mask(float* g, const bf16* a, size_t n) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n && !(__bfloat162float(a[i]) > 0.f)) g[i] = 0.f;
}

// dIn[b,y,x,ci] = sum_{co,dy,dx} dZ[b, y-dy+p, x-dx+p, co] W[co][dy][dx][ci]
template <int K>
__global__ void k_conv_dgrad(const float* dZ, int cout, int H, int W, const bf16* Wt, int cin, float* dIn) {
    extern __shared__ float rows[];  // [K][W + 2][cout]
    const int b = blockIdx.x / H, y = blockIdx.x % H;
    const int pad = K / 2, RW = W + 2 * pad;
    for (int i = threadIdx.x; i < K * RW * cout; i += blockDim.x) {
        const int r = i / (RW * cout), xx = (i / cout) % RW, c = i % cout;
        const int yy = y - r + pad, xc = xx - pad;  // row r holds dZ at y - r + pad
        rows[i] = (yy >= 0 && yy < H && xc >= 0 && xc < W) ? dZ[((size_t(b) * H + yy) * W + xc) * cout + c] : 0.f;
    }
    __syncthreads();
    constexpr int XG = 4;
    const int groups = (W + XG - 1) / XG;
    for (int t = threadIdx.x; t < cin * groups; t += blockDim.x) {
        const int ci = t / groups, x0 = (t % groups) * XG;
        float acc[XG] = {0.f, 0.f, 0.f, 0.f};
        for (int dy = 0; dy < K; ++dy)
            for (int dx = 0; dx < K; ++dx)
                for (int co = 0; co < cout; ++co) {
                    const float wv = __bfloat162float(Wt[((size_t(co) * K + dy) * K + dx) * cin + ci]);
#pragma unroll
                    for (int g = 0; g < XG; ++g) {
                        const int xc = x0 + g - dx + pad;  // dZ column, shifted by RW offset pad
                        if (x0 + g < W) acc[g] += wv * rows[(dy * RW + xc + pad) * cout + co];
                    }
                }
        for (int g = 0; g < XG; ++g)
            if (x0 + g < W) dIn[((size_t(b) * H + y) * W + x0 + g) * cin + ci] = acc[g];
    }
}

// dW[co][dy][dx][ci] = sum_{b,y,x} dZ[b,y,x,co] in[b, y+dy-p, x+dx-p, ci];
// db[co] = sum dZ. One block per (co, dy, dx); threads over (ci, pixel
// subsets), reduced in shared memory (fixed order).
template <int K>
__global__ void k_conv_wgrad(const float* dZ, int cout, const bf16* A, int ca, bool upA, const bf16* Bt, int cb,
                             int Bn, int H, int W, float* dW, float* db) {
    const int cin = ca + cb;
    const int co = blockIdx.x / (K * K), tap = blockIdx.x % (K * K), dy = tap / K, dx = tap % K;
    const int pad = K / 2;
    const int nthr = blockDim.x, lanes_c = cin < nthr ? cin : nthr, parts = nthr / lanes_c;
    const int ci = threadIdx.x % lanes_c, part = threadIdx.x / lanes_c;
    extern __shared__ float red[];
    const int P = Bn * H * W;
    for (int c0 = 0; c0 < cin; c0 += lanes_c) {
        const int c = c0 + ci;
        float acc = 0.f, accb = 0.f;
        if (part < parts && c < cin) {
            for (int p = part; p < P; p += parts) {
                const int b = p / (H * W), y = (p / W) % H, x = p % W;
                const float g = dZ[size_t(p) * cout + co];
                if (c0 == 0 && ci == 0 && tap == 0) accb += g;
                const int yy = y + dy - pad, xc = x + dx - pad;
                if (yy < 0 || yy >= H || xc < 0 || xc >= W) continue;
                float v;
                if (c < ca) {
                    v = upA ? __bfloat162float(A[((size_t(b) * (H / 2) + yy / 2) * (W / 2) + xc / 2) * ca + c])
                            : __bfloat162float(A[((size_t(b) * H + yy) * W + xc) * ca + c]);
                } else {
                    v = __bfloat162float(Bt[((size_t(b) * H + yy) * W + xc) * cb + (c - ca)]);
                }
                acc += g * v;
            }
        }
        red[threadIdx.x] = acc;
        red[nthr + threadIdx.x] = accb;
        __syncthreads();
        if (part == 0 && c < cin) {
            float s = 0.f, sb = 0.f;
            for (int q = 0; q < parts; ++q) {
                s += red[q * lanes_c + ci];
                sb += red[nthr + q * lanes_c + ci];
            }
            dW[((size_t(co) * K + dy) * K + dx) * cin + c] = s;
            if (c0 == 0 && ci == 0 && tap == 0) db[co] = sb;
        }
        __syncthreads();
    }
}

__global__ void k_avgpool(const bf16* in, int Bn, int H, int W, int C, bf16* out) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= size_t(Bn) * Ho * Wo * C) return;
    const int c = i % C, x = (i / C) % Wo, y = (i / (size_t(C) * Wo)) % Ho, b = i / (size_t(C) * Wo * Ho);
    float s = 0.f;
    for (int a = 0; a < 2; ++a)
        for (int d = 0; d < 2; ++d) s += __bfloat162float(in[((size_t(b) * H + 2 * y + a) * W + 2 * x + d) * C + c]);
    out[i] = __float2bfloat16(0.25f * s);
}

// dIn (H x W) += pool^T(dOut)
__global__ void k_avgpool_bwd_add(const float* dOut, int Bn, int H, int W, int C, float* dIn) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(Bn) * H * W * C) return;
    const int c = i % C, x = (i / C) % W, y = (i / (size_t(C) * W)) % H, b = i / (size_t(C) * W * H);
    dIn[i] += 0.25f * dOut[((size_t(b) * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
}

// dCat [B,H,W,ca+cb] -> dLow [B,H/2,W/2,ca] = up^T(dCat[..., :ca]); dSkip (+)= dCat[..., ca:]
__global__ void k_split_concat(const float* dCat, int Bn, int H, int W, int ca, int cb, float* dLow, float* dSkip) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int C = ca + cb;
    const int Hl = H / 2, Wl = W / 2;
    if (i < size_t(Bn) * Hl * Wl * ca) {
        const int c = i % ca, x = (i / ca) % Wl, y = (i / (size_t(ca) * Wl)) % Hl, b = i / (size_t(ca) * Wl * Hl);
        float s = 0.f;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 2; ++d) s += dCat[((size_t(b) * H + 2 * y + a) * W + 2 * x + d) * C + c];
        dLow[i] = s;
    }
    if (i < size_t(Bn) * H * W * cb) {
        const int c = i % cb;
        const size_t p = i / cb;
        dSkip[i] = dCat[p * C + ca + c];
    }
}

// masked MSE: loss += sum m (p - t)^2 / cnt ; dP = 2 m (p - t) / cnt
__global__ void k_loss(const float* pred, const float* T, const float* LM, int npix, float inv_cnt, float* dP,
                       float* loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < npix) {
        const float m = LM[i];
        const float d0 = (pred[2 * i] - T[2 * i]) * m, d1 = (pred[2 * i + 1] - T[2 * i + 1]) * m;
        dP[2 * i] = 2.f * d0 * inv_cnt;
        dP[2 * i + 1] = 2.f * d1 * inv_cnt;
        l = (d0 * d0 + d1 * d1) * inv_cnt;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

__global__ void k_sum(const float* v, int n, float* out) {
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int(blockDim.x) + 31) / 32; ++w) t += part[w];
        *out = t;
    }
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, bf16* wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float* w, int n, bf16* wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16(w[i]);
}

// prediction [F][32][32][2] -> warm start [F][2][128][128]
__global__ void k_warm_start(const float* pred, int F, float* ext) {
    const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= size_t(F) * 2 * GRID * GRID) return;
    const int c = i % GRID, m = (i / GRID) % GRID, ch = (i / (GRID * GRID)) % 2;
    const size_t f = i / (2 * GRID * GRID);
    ext[i] = pred[((f * LOW + m / POOL) * LOW + c / POOL) * 2 + ch] * (1.f / IN_SCALE);
}

// ----------------------------------------------------------------- runner --

struct Layer {
    int ca, cb, cout, k, H;   // inputs: A (ca), B (cb); output channels; kernel; resolution
    bool upA, relu;
    size_t woff, boff;        // offsets in the flat parameter vector
    bool tc;                  // forward on the tensor cores (k_conv_tc)
    size_t poff;              // offset of the packed weights (uint2 units)
};

inline unsigned blocks(size_t n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace net
}  // namespace fwr

using namespace fwr::net;

struct fwr_net {
    int w = 0, max_batch = 0, device = 0;
    std::vector<Layer> layers;
    size_t nparam = 0;
    float* W = nullptr;   // FP32 master weights (flat)
    bf16* Wb = nullptr;   // BF16 copy used by the kernels
    uint2* Wp = nullptr;  // BF16 weights of the tensor-core layers in fragment order
    size_t npacked = 0;   // uint2 count of Wp
    int conv = FWR_NET_CONV_AUTO;
    float *G = nullptr, *M = nullptr, *V = nullptr;
    int step = 0;
    // activations (BF16) and their gradients (FP32), one per layer output
    std::vector<bf16*> act;
    std::vector<float*> grad;
    bf16 *X = nullptr, *pool1 = nullptr, *pool2 = nullptr, *pool3 = nullptr;
    float *pred = nullptr, *dpred = nullptr, *T = nullptr, *LM = nullptr, *loss = nullptr, *cnt = nullptr;
    float *dcat = nullptr, *dtmp = nullptr, *dpool = nullptr;
};

namespace {

// layer order as in the definition: e1a e1b e2a e2b e3a e3b ba bb d3a d3b d2a d2b d1a d1b out
void build_layers(fwr_net* n) {
    const int w1 = n->w, w2 = 2 * n->w, w3 = 4 * n->w, w4 = 4 * n->w;
    struct S { int ca, cb, co, k, H; bool up, relu; };
    const S s[] = {{3, 0, w1, 3, 32, false, true},   {w1, 0, w1, 3, 32, false, true},
                   {w1, 0, w2, 3, 16, false, true},  {w2, 0, w2, 3, 16, false, true},
                   {w2, 0, w3, 3, 8, false, true},   {w3, 0, w3, 3, 8, false, true},
                   {w3, 0, w4, 3, 4, false, true},   {w4, 0, w4, 3, 4, false, true},
                   {w4, w3, w3, 3, 8, true, true},   {w3, 0, w3, 3, 8, false, true},
                   {w3, w2, w2, 3, 16, true, true},  {w2, 0, w2, 3, 16, false, true},
                   {w2, w1, w1, 3, 32, true, true},  {w1, 0, w1, 3, 32, false, true},
                   {w1, 0, 2, 1, 32, false, false}};
    size_t pos = 0;
    for (const S& x : s) {
        Layer L;
        L.ca = x.ca;
        L.cb = x.cb;
        L.cout = x.co;
        L.k = x.k;
        L.H = x.H;
        L.upA = x.up;
        L.relu = x.relu;
        L.woff = pos;
        pos += size_t(x.co) * x.k * x.k * (x.ca + x.cb);
        L.boff = pos;
        pos += x.co;
        // tensor-core forward: whole 16-channel reduction chunks from one
        // input, n8 output tiles, 32-bit aligned weight rows, whole rows per CTA
        L.tc = x.k == 3 && x.ca % 16 == 0 && x.cb % 16 == 0 && x.co % 8 == 0 && L.woff % 2 == 0 &&
               TC_TM % x.H == 0;
        L.poff = n->npacked;
        if (L.tc) n->npacked += size_t(9) * (x.ca + x.cb) * x.co / 4;
        n->layers.push_back(L);
    }
    n->nparam = pos;
}

int tc_nt(int cout) {
    const int ntt = cout / 8;
    return ntt % 8 == 0 ? 8 : ntt % 4 == 0 ? 4 : ntt % 2 == 0 ? 2 : 1;
}

// BF16 weights -> fragment order for every tensor-core layer
cudaError_t pack_weights(fwr_net* n, cudaStream_t s) {
    for (const Layer& L : n->layers) {
        if (!L.tc) continue;
        const int cin = L.ca + L.cb;
        const size_t cnt = size_t(9) * cin * L.cout / 4;
        k_pack_tc<<<blocks(cnt, 256), 256, 0, s>>>(n->Wb + L.woff, cin, L.cout, n->Wp + L.poff);
    }
    return cudaGetLastError();
}

cudaError_t conv_fwd(fwr_net* n, int li, const bf16* A, const bf16* B, int Bn, bf16* out_bf, float* out_f,
                     cudaStream_t s) {
    const Layer& L = n->layers[li];
    const int cin = L.ca + L.cb, RW = L.H + 2 * (L.k / 2);
    if (L.tc && out_bf && n->conv == FWR_NET_CONV_AUTO) {
        const int npix = Bn * L.H * L.H, nt = tc_nt(L.cout);
        const dim3 grid(unsigned((npix + TC_TM - 1) / TC_TM), unsigned(L.cout / (8 * nt)));
        const size_t sm = tc_smem_bytes(L.H, cin);
        const uint2* wp = n->Wp + L.poff;
        const float* bias = n->W + L.boff;
        const int up = L.upA ? 1 : 0, relu = L.relu ? 1 : 0;
        switch (nt) {
            case 8: k_conv_tc<8><<<grid, TC_THREADS, sm, s>>>(A, L.ca, up, B, L.cb, L.H, wp, bias, L.cout, relu, npix, out_bf); break;
            case 4: k_conv_tc<4><<<grid, TC_THREADS, sm, s>>>(A, L.ca, up, B, L.cb, L.H, wp, bias, L.cout, relu, npix, out_bf); break;
            case 2: k_conv_tc<2><<<grid, TC_THREADS, sm, s>>>(A, L.ca, up, B, L.cb, L.H, wp, bias, L.cout, relu, npix, out_bf); break;
            default: k_conv_tc<1><<<grid, TC_THREADS, sm, s>>>(A, L.ca, up, B, L.cb, L.H, wp, bias, L.cout, relu, npix, out_bf); break;
        }
        return cudaGetLastError();
    }
    const size_t smem = size_t(L.k) * RW * cin * sizeof(float);
    if (L.k == 3)
        k_conv_fwd<3><<<Bn * L.H, 256, smem, s>>>(A, L.ca, L.upA, B, L.cb, L.H, L.H, n->Wb + L.woff, n->W + L.boff,
                                                  L.cout, L.relu, out_bf, out_f);
    else
        k_conv_fwd<1><<<Bn * L.H, 256, smem, s>>>(A, L.ca, L.upA, B, L.cb, L.H, L.H, n->Wb + L.woff, n->W + L.boff,
                                                  L.cout, L.relu, out_bf, out_f);
    return cudaGetLastError();
}

// forward of the whole network on X (Bn images); prediction into n->pred
cudaError_t forward(fwr_net* n, int Bn, cudaStream_t s) {
    bf16** a = n->act.data();
    cudaError_t e;
    const int w1 = n->w, w3 = 4 * n->w;
    if ((e = conv_fwd(n, 0, n->X, nullptr, Bn, a[0], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 1, a[0], nullptr, Bn, a[1], nullptr, s)) != cudaSuccess) return e;
    k_avgpool<<<blocks(size_t(Bn) * 16 * 16 * w1, 256), 256, 0, s>>>(a[1], Bn, 32, 32, w1, n->pool1);
    if ((e = conv_fwd(n, 2, n->pool1, nullptr, Bn, a[2], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 3, a[2], nullptr, Bn, a[3], nullptr, s)) != cudaSuccess) return e;
    k_avgpool<<<blocks(size_t(Bn) * 8 * 8 * 2 * w1, 256), 256, 0, s>>>(a[3], Bn, 16, 16, 2 * w1, n->pool2);
    if ((e = conv_fwd(n, 4, n->pool2, nullptr, Bn, a[4], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 5, a[4], nullptr, Bn, a[5], nullptr, s)) != cudaSuccess) return e;
    k_avgpool<<<blocks(size_t(Bn) * 4 * 4 * w3, 256), 256, 0, s>>>(a[5], Bn, 8, 8, w3, n->pool3);
    if ((e = conv_fwd(n, 6, n->pool3, nullptr, Bn, a[6], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 7, a[6], nullptr, Bn, a[7], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 8, a[7], a[5], Bn, a[8], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 9, a[8], nullptr, Bn, a[9], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 10, a[9], a[3], Bn, a[10], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 11, a[10], nullptr, Bn, a[11], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 12, a[11], a[1], Bn, a[12], nullptr, s)) != cudaSuccess) return e;
    if ((e = conv_fwd(n, 13, a[12], nullptr, Bn, a[13], nullptr, s)) != cudaSuccess) return e;
    return conv_fwd(n, 14, a[13], nullptr, Bn, nullptr, n->pred, s);
}

// backward of one conv layer: dZ = g (relu-masked by the caller); writes dW,
// db into G and dIn (concatenated input gradient) into din
cudaError_t conv_bwd(fwr_net* n, int li, const float* dZ, const bf16* A, const bf16* B, int Bn, float* din,
                     cudaStream_t s) {
    const Layer& L = n->layers[li];
    const int cin = L.ca + L.cb, RW = L.H + 2 * (L.k / 2);
    const int thr = 256;
    if (L.k == 3) {
        k_conv_wgrad<3><<<L.cout * 9, thr, 2 * thr * sizeof(float), s>>>(dZ, L.cout, A, L.ca, L.upA, B, L.cb, Bn, L.H,
                                                                          L.H, n->G + L.woff, n->G + L.boff);
        if (din)
            k_conv_dgrad<3><<<Bn * L.H, 256, size_t(3) * RW * L.cout * sizeof(float), s>>>(
                dZ, L.cout, L.H, L.H, n->Wb + L.woff, cin, din);
    } else {
        k_conv_wgrad<1><<<L.cout, thr, 2 * thr * sizeof(float), s>>>(dZ, L.cout, A, L.ca, L.upA, B, L.cb, Bn, L.H,
                                                                      L.H, n->G + L.woff, n->G + L.boff);
        if (din)
            k_conv_dgrad<1><<<Bn * L.H, 256, size_t(1) * RW * L.cout * sizeof(float), s>>>(
                dZ, L.cout, L.H, L.H, n->Wb + L.woff, cin, din);
    }
    return cudaGetLastError();
}

void relu_mask(float* g, const bf16* a, size_t cnt, cudaStream_t s) {
    k_relu_mask<<<blocks(cnt, 256), 256, 0, s>>>(g, a, cnt);
}

// backward of the whole network from n->dpred; gradients into n->G
cudaError_t backward(fwr_net* n, int Bn, cudaStream_t s) {
    bf16** a = n->act.data();
    float** g = n->grad.data();
    const int w1 = n->w, w2 = 2 * n->w, w3 = 4 * n->w, w4 = 4 * n->w;
    auto px = [&](int H, int C) { return size_t(Bn) * H * H * C; };
    cudaError_t e;
    // out: 1x1, no ReLU
    if ((e = conv_bwd(n, 14, n->dpred, a[13], nullptr, Bn, g[13], s)) != cudaSuccess) return e;
    // d1b, d1a (input concat [up(d2b) w2 | s1 w1] at 32)
    relu_mask(g[13], a[13], px(32, w1), s);
    if ((e = conv_bwd(n, 13, g[13], a[12], nullptr, Bn, g[12], s)) != cudaSuccess) return e;
    relu_mask(g[12], a[12], px(32, w1), s);
    if ((e = conv_bwd(n, 12, g[12], a[11], a[1], Bn, n->dcat, s)) != cudaSuccess) return e;
    k_split_concat<<<blocks(px(32, w1 + w2), 256), 256, 0, s>>>(n->dcat, Bn, 32, 32, w2, w1, g[11], g[1]);
    // d2b, d2a (concat [up(d3b) w3 | s2 w2] at 16)
    relu_mask(g[11], a[11], px(16, w2), s);
    if ((e = conv_bwd(n, 11, g[11], a[10], nullptr, Bn, g[10], s)) != cudaSuccess) return e;
    relu_mask(g[10], a[10], px(16, w2), s);
    if ((e = conv_bwd(n, 10, g[10], a[9], a[3], Bn, n->dcat, s)) != cudaSuccess) return e;
    k_split_concat<<<blocks(px(16, w2 + w3), 256), 256, 0, s>>>(n->dcat, Bn, 16, 16, w3, w2, g[9], g[3]);
    // d3b, d3a (concat [up(bb) w4 | s3 w3] at 8)
    relu_mask(g[9], a[9], px(8, w3), s);
    if ((e = conv_bwd(n, 9, g[9], a[8], nullptr, Bn, g[8], s)) != cudaSuccess) return e;
    relu_mask(g[8], a[8], px(8, w3), s);
    if ((e = conv_bwd(n, 8, g[8], a[7], a[5], Bn, n->dcat, s)) != cudaSuccess) return e;
    k_split_concat<<<blocks(px(8, w3 + w4), 256), 256, 0, s>>>(n->dcat, Bn, 8, 8, w4, w3, g[7], g[5]);
    // bottleneck at 4
    relu_mask(g[7], a[7], px(4, w4), s);
    if ((e = conv_bwd(n, 7, g[7], a[6], nullptr, Bn, g[6], s)) != cudaSuccess) return e;
    relu_mask(g[6], a[6], px(4, w4), s);
    if ((e = conv_bwd(n, 6, g[6], n->pool3, nullptr, Bn, n->dpool, s)) != cudaSuccess) return e;
    k_avgpool_bwd_add<<<blocks(px(8, w3), 256), 256, 0, s>>>(n->dpool, Bn, 8, 8, w3, g[5]);
    // encoder level 3 (8)
    relu_mask(g[5], a[5], px(8, w3), s);
    if ((e = conv_bwd(n, 5, g[5], a[4], nullptr, Bn, g[4], s)) != cudaSuccess) return e;
    relu_mask(g[4], a[4], px(8, w3), s);
    if ((e = conv_bwd(n, 4, g[4], n->pool2, nullptr, Bn, n->dpool, s)) != cudaSuccess) return e;
    k_avgpool_bwd_add<<<blocks(px(16, w2), 256), 256, 0, s>>>(n->dpool, Bn, 16, 16, w2, g[3]);
    // level 2 (16)
    relu_mask(g[3], a[3], px(16, w2), s);
    if ((e = conv_bwd(n, 3, g[3], a[2], nullptr, Bn, g[2], s)) != cudaSuccess) return e;
    relu_mask(g[2], a[2], px(16, w2), s);
    if ((e = conv_bwd(n, 2, g[2], n->pool1, nullptr, Bn, n->dpool, s)) != cudaSuccess) return e;
    k_avgpool_bwd_add<<<blocks(px(32, w1), 256), 256, 0, s>>>(n->dpool, Bn, 32, 32, w1, g[1]);
    // level 1 (32)
    relu_mask(g[1], a[1], px(32, w1), s);
    if ((e = conv_bwd(n, 1, g[1], a[0], nullptr, Bn, g[0], s)) != cudaSuccess) return e;
    relu_mask(g[0], a[0], px(32, w1), s);
    return conv_bwd(n, 0, g[0], n->X, nullptr, Bn, nullptr, s);
}

void free_net(fwr_net* n) {
    cudaFree(n->W);
    cudaFree(n->Wb);
    cudaFree(n->Wp);
    cudaFree(n->G);
    cudaFree(n->M);
    cudaFree(n->V);
    for (auto p : n->act) cudaFree(p);
    for (auto p : n->grad) cudaFree(p);
    cudaFree(n->X);
    cudaFree(n->pool1);
    cudaFree(n->pool2);
    cudaFree(n->pool3);
    cudaFree(n->pred);
    cudaFree(n->dpred);
    cudaFree(n->T);
    cudaFree(n->LM);
    cudaFree(n->loss);
    cudaFree(n->cnt);
    cudaFree(n->dcat);
    cudaFree(n->dtmp);
    cudaFree(n->dpool);
    delete n;
}

bool geometry_ok(const fwr_plan* p) { return p && p->N == GRID; }

cudaError_t prepare(fwr_net* n, const fwr_plan* p, const float* slopes, int F, cudaStream_t s) {
    k_input<<<blocks(size_t(F) * LOW * LOW, 256), 256, 0, s>>>(slopes, p->d_mask, p->n, p->off, F, n->X);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

fwr_status fwr_net_create(fwr_net** out, int width, int max_batch, const float* init_weights, int count) {
    if (!out) return FWR_ERR_ARG;
    *out = nullptr;
    if (width < 1 || width > 32 || max_batch < 1 || max_batch > 65536) return FWR_ERR_ARG;
    fwr_net* n = new (std::nothrow) fwr_net();
    if (!n) return FWR_ERR_CUDA;
    n->w = width;
    n->max_batch = max_batch;
    build_layers(n);
    if (init_weights && size_t(count) != n->nparam) {
        delete n;
        return FWR_ERR_ARG;
    }
    cudaGetDevice(&n->device);
    cudaError_t e = cudaSuccess;
    auto falloc = [&](float** p, size_t cnt) {
        if (e == cudaSuccess) e = cudaMalloc(p, cnt * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(*p, 0, cnt * sizeof(float));
    };
    auto balloc = [&](bf16** p, size_t cnt) {
        if (e == cudaSuccess) e = cudaMalloc(p, cnt * sizeof(bf16));
    };
    falloc(&n->W, n->nparam);
    balloc(&n->Wb, n->nparam);
    if (e == cudaSuccess && n->npacked) e = cudaMalloc(&n->Wp, n->npacked * sizeof(uint2));
    falloc(&n->G, n->nparam);
    falloc(&n->M, n->nparam);
    falloc(&n->V, n->nparam);
    const size_t B = size_t(max_batch);
    for (const Layer& L : n->layers) {
        const size_t cnt = B * L.H * L.H * L.cout;
        bf16* a = nullptr;
        float* g = nullptr;
        balloc(&a, cnt);
        falloc(&g, cnt);
        n->act.push_back(a);
        n->grad.push_back(g);
    }
    const int w1 = width, w2 = 2 * width, w3 = 4 * width, w4 = 4 * width;
    balloc(&n->X, B * 32 * 32 * 3);
    balloc(&n->pool1, B * 16 * 16 * w1);
    balloc(&n->pool2, B * 8 * 8 * w2);
    balloc(&n->pool3, B * 4 * 4 * w3);
    falloc(&n->pred, B * 32 * 32 * 2);
    falloc(&n->dpred, B * 32 * 32 * 2);
    falloc(&n->T, B * 32 * 32 * 2);
    falloc(&n->LM, B * 32 * 32);
    falloc(&n->loss, 1);
    falloc(&n->cnt, 1);
    falloc(&n->dcat, B * 32 * 32 * size_t(w1 + w2 + w3 + w4));
    falloc(&n->dpool, B * 16 * 16 * w1 + B * 8 * 8 * w2 + B * 4 * 4 * w3);
    if (e == cudaSuccess) {
        std::vector<float> h(n->nparam, 0.f);
        if (init_weights) h.assign(init_weights, init_weights + n->nparam);
        e = cudaMemcpy(n->W, h.data(), n->nparam * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) k_to_bf16<<<blocks(n->nparam, 256), 256>>>(n->W, int(n->nparam), n->Wb);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = pack_weights(n, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    // the convolution kernels stage K rows of (H + 2) pixels x channels as floats
    size_t fwd_smem = 0, dgrad_smem = 0;
    for (const Layer& L : n->layers) {
        const size_t rw = size_t(L.H + 2 * (L.k / 2)) * L.k * sizeof(float);
        fwd_smem = std::max(fwd_smem, rw * (L.ca + L.cb));
        dgrad_smem = std::max(dgrad_smem, rw * L.cout);
    }
    size_t tc_smem = 0;
    for (const Layer& L : n->layers)
        if (L.tc) tc_smem = std::max(tc_smem, tc_smem_bytes(L.H, L.ca + L.cb));
    if (fwd_smem > 227 * 1024 || dgrad_smem > 227 * 1024) e = cudaErrorInvalidValue;
    if (tc_smem > 227 * 1024) {
        for (Layer& L : n->layers) L.tc = false;
        tc_smem = 0;
    }
    if (e == cudaSuccess && tc_smem) {
        const int v = int(tc_smem);
        e = cudaFuncSetAttribute(k_conv_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_fwd<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(fwd_smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_dgrad<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dgrad_smem));
    if (e != cudaSuccess) {
        free_net(n);
        return fwr::cuda_fail(e, "fwr_net_create");
    }
    *out = n;
    return FWR_OK;
}

void fwr_net_destroy(fwr_net* n) {
    if (n) free_net(n);
}

int fwr_net_param_count(const fwr_net* n) { return n ? int(n->nparam) : -1; }

fwr_status fwr_net_get_weights(fwr_net* n, float* host, int count) {
    if (!n || !host || size_t(count) != n->nparam) return FWR_ERR_ARG;
    cudaError_t e = cudaMemcpy(host, n->W, n->nparam * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_net_get_weights");
}

fwr_status fwr_net_set_weights(fwr_net* n, const float* host, int count) {
    if (!n || !host || size_t(count) != n->nparam) return FWR_ERR_ARG;
    cudaError_t e = cudaMemcpy(n->W, host, n->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_to_bf16<<<blocks(n->nparam, 256), 256>>>(n->W, int(n->nparam), n->Wb);
        e = pack_weights(n, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_net_set_weights");
}

fwr_status fwr_net_set_option(fwr_net* n, int option, int value) {
    if (!n) return FWR_ERR_ARG;
    if (option == FWR_NET_OPT_CONV) {
        if (value != FWR_NET_CONV_AUTO && value != FWR_NET_CONV_SIMT) return FWR_ERR_ARG;
        n->conv = value;
        return FWR_OK;
    }
    return FWR_ERR_ARG;
}

int fwr_net_tc_layers(const fwr_net* n) {
    if (!n) return -1;
    int c = 0;
    for (const Layer& L : n->layers) c += L.tc ? 1 : 0;
    return c;
}

fwr_status fwr_net_forward(fwr_net* n, const fwr_plan* p, const float* slopes, int F, float* ext_init, void* stream) {
    if (!n || !geometry_ok(p) || F < 0 || F > n->max_batch || (F > 0 && (!slopes || !ext_init))) return FWR_ERR_ARG;
    if (F == 0) return FWR_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = prepare(n, p, slopes, F, s);
    if (e == cudaSuccess) e = forward(n, F, s);
    if (e == cudaSuccess) {
        k_warm_start<<<blocks(size_t(F) * 2 * GRID * GRID, 256), 256, 0, s>>>(n->pred, F, ext_init);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_net_forward");
}

// forward + loss + backward; gradients left in the net (and copied to
// grad_host when given); loss written to *loss_host (synchronises)
fwr_status fwr_net_gradients(fwr_net* n, const fwr_plan* p, const float* slopes, const float* target_ext, int F,
                             float* grad_host, float* loss_host, void* stream) {
    if (!n || !geometry_ok(p) || F < 1 || F > n->max_batch || !slopes || !target_ext) return FWR_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = prepare(n, p, slopes, F, s);
    if (e == cudaSuccess) {
        k_target<<<blocks(size_t(F) * LOW * LOW, 256), 256, 0, s>>>(target_ext, p->d_mask, p->n, p->off, F, n->T,
                                                                     n->LM);
        k_sum<<<1, 1024, 0, s>>>(n->LM, F * LOW * LOW, n->cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = forward(n, F, s);
    float cnt = 0.f;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, n->cnt, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        cudaMemsetAsync(n->loss, 0, sizeof(float), s);
        const int npix = F * LOW * LOW;
        k_loss<<<blocks(npix, 256), 256, 0, s>>>(n->pred, n->T, n->LM, npix, 1.f / fmaxf(1.f, 2.f * cnt), n->dpred,
                                                  n->loss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(n, F, s);
    if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grad_host)
        e = cudaMemcpyAsync(grad_host, n->G, n->nparam * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_net_gradients");
}

fwr_status fwr_net_train_step(fwr_net* n, const fwr_plan* p, const float* slopes, const float* target_ext, int F,
                              float lr, float* loss_host, void* stream) {
    fwr_status st = fwr_net_gradients(n, p, slopes, target_ext, F, nullptr, loss_host, stream);
    if (st != FWR_OK) return st;
    if (!(lr > 0.f)) return FWR_ERR_ARG;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, float(n->step)), c2 = 1.f - std::pow(b2, float(n->step));
    k_adam<<<blocks(n->nparam, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n->W, n->G, n->M, n->V, int(n->nparam), lr, b1, b2, 1e-8f, c1, c2, n->Wb);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = pack_weights(n, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FWR_OK : fwr::cuda_fail(e, "fwr_net_train_step");
}

}  // extern "C"
