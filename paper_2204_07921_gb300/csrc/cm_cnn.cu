// cm_cnn.cu -- the learned warm start: a small CNN maps f to an initial u.
//
// Network: six 3x3 convolutions with zero padding, channels 1 -> 32 -> 32 ->
// 32 -> 32 -> 32 -> 1, ReLU after the first five, residual output
// u0 = f + conv6(...).  Activations are BF16, 64 bytes per pixel per layer,
// stored plane-major within each image row: [n][y][plane q][x][8 channels],
// plane q holding channels 8q .. 8q + 7 (act_off), so a run of pixels of
// one plane is contiguous and a TMA box of 4-pixel groups of one plane reads
// whole 32-byte sectors.  Weights are kept in FP32 (master copy, Adam) and
// used in BF16; every product is accumulated in FP32.
//
//  conv_in_kernel     1 -> 32 on CUDA cores (9 MACs per output), two pixels
//                     and 16 channels per thread, persistent CTAs.
//  conv_tc_kernel     32 -> 32 (and the output layer 32 -> 1 with the
//                     residual, and dX of the backward pass with the ReLU
//                     mask of the layer's input) on the 5th-generation
//                     tensor cores: TMA-loaded strip halos, tcgen05.mma into
//                     TMEM accumulators, warp-specialised and persistent
//                     (details at the kernel).
//  conv_mid_kernel    the same three roles as an implicit GEMM with
//                     ldmatrix + mma.sync m16n8k16 BF16 -> FP32: M = pixels
//                     (8 x 16 tiles), N = 32, K = 9 x 32; persistent CTAs
//                     (weights staged once) with cp.async double-buffered
//                     halo tiles.  Built with CM_CNN_TC=0, for comparison.
//  dw_mid_kernel      dW = sum_p X[p + tap]^T dZ[p] on the tensor cores, per
//                     CTA partial sums over a grid-stride set of tiles,
//                     reduced in a fixed order (deterministic).
//  out_grad_kernel    dL/dout of the MSE loss, dX of conv6, ReLU mask.
//  dw_small kernels   dW of conv1 and conv6 (CUDA cores).
//  adam_kernel        Adam (Kingma and Ba) on the FP32 master weights, then
//                     the BF16 copies are repacked.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <stdint.h>

#include "../../include/cm.h"
#include "cm_cnn.h"

namespace cm {
namespace cnn {

using bf16 = __nv_bfloat16;

constexpr int C = 32;
constexpr int TH = 8, TW = 16;                 // output tile: 8 rows x 16 columns
constexpr int HH = TH + 2, HW = TW + 2;        // with a one-pixel halo
constexpr int CS = 40;                         // smem pixel stride (32 channels + 8 pad)
constexpr int MIDW = 9 * C * C;                // weights of one 32 -> 32 layer
constexpr int OFF_W1 = 0, OFF_B1 = 9 * C;
__host__ __device__ constexpr int off_w(int l) { return 9 * C + C + (l - 2) * (MIDW + C); }
__host__ __device__ constexpr int off_b(int l) { return off_w(l) + MIDW; }
constexpr int OFF_W6 = 9 * C + C + 4 * (MIDW + C);
constexpr int OFF_B6 = OFF_W6 + 9 * C;
constexpr int NPAR = OFF_B6 + 1;
static_assert(NPAR == 37601, "parameter count");
static_assert(OFF_B1 + C == off_w(2) && OFF_W1 + 9 * C == OFF_B1, "layer 1: weights, bias");
constexpr int DW_STRIDE = MIDW + C;            // one CTA partial of a 32 -> 32 layer
constexpr int DW_GRID = 2 * 152;               // CTAs of the weight-gradient kernels

// ---------------------------------------------------------------------------
// PTX helpers.

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_addr(p)));
}

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte asynchronous copy global -> shared; zero-filled when !valid (the
// source address is then not read).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)),
                 "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ float bf(bf16 x) { return __bfloat162float(x); }

// Activation layout (BF16, 32 channels), plane-major per image row: element
// (pixel (n, y, x), channel c) sits at ((row 4 + c / 8) Wp + x) 8 + c mod 8,
// row = n H + y, Wp = W rounded up to a multiple of 4.  In each row the four
// planes of 8 channels (16 bytes per pixel) are contiguous along x, and the
// tensor-core convolution's TMA boxes read them in groups of 4 pixels
// (64 bytes, two whole 32-byte sectors): a box whose innermost extent is one
// 16-byte pixel costs a sector per pixel, twice the bytes.  The Wp - W pad
// pixels of a row are never written; readers skip them or zero them.
__host__ __device__ __forceinline__ int act_wp(int W) { return (W + 3) & ~3; }
__host__ __device__ __forceinline__ size_t act_off(size_t row, int x, int q, int W) {
    return ((row * 4 + (size_t)q) * (size_t)act_wp(W) + (size_t)x) * 8;
}
__device__ __forceinline__ float round_bf(float x) { return __bfloat162float(__float2bfloat16(x)); }

// Tile geometry shared by the tiled kernels: tile t of image n.
struct Tile {
    int n, y0, x0;
};
__device__ __forceinline__ Tile tile_of(int t, int H, int W) {
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH;
    Tile r;
    r.n = t / (tx * ty);
    const int rem = t - r.n * tx * ty;
    r.y0 = (rem / tx) * TH;
    r.x0 = (rem % tx) * TW;
    return r;
}

// Stage the (TH+2) x (TW+2) x 32 BF16 halo tile of X (zero outside the image).
__device__ __forceinline__ void load_halo(bf16 (*s)[CS], const bf16* __restrict__ X, const Tile& t,
                                          int H, int W) {
    for (int i = threadIdx.x; i < HH * HW * 4; i += blockDim.x) {
        const int pix = i >> 2, q = i & 3;
        const int gy = t.y0 - 1 + pix / HW, gx = t.x0 - 1 + pix % HW;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            v = *reinterpret_cast<const uint4*>(X + act_off((size_t)t.n * H + gy, gx, q, W));
        *reinterpret_cast<uint4*>(&s[pix][q * 8]) = v;
    }
}

// Stage the TH x TW x 32 tile of X (zero outside the image).
__device__ __forceinline__ void load_tile(bf16 (*s)[CS], const bf16* __restrict__ X, const Tile& t,
                                          int H, int W) {
    for (int i = threadIdx.x; i < TH * TW * 4; i += blockDim.x) {
        const int pix = i >> 2, q = i & 3;
        const int gy = t.y0 + pix / TW, gx = t.x0 + pix % TW;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gy < H && gx < W)
            v = *reinterpret_cast<const uint4*>(X + act_off((size_t)t.n * H + gy, gx, q, W));
        *reinterpret_cast<uint4*>(&s[pix][q * 8]) = v;
    }
}

// The halo tile of load_halo, staged with asynchronous copies.
__device__ __forceinline__ void load_halo_async(bf16 (*s)[CS], const bf16* __restrict__ X,
                                                const Tile& t, int H, int W) {
    for (int i = threadIdx.x; i < HH * HW * 4; i += blockDim.x) {
        const int pix = i >> 2, q = i & 3;
        const int gy = t.y0 - 1 + pix / HW, gx = t.x0 - 1 + pix % HW;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const bf16* src = in ? X + act_off((size_t)t.n * H + gy, gx, q, W) : X;
        cp_async16(&s[pix][q * 8], src, in);
    }
}

// ---------------------------------------------------------------------------
// Forward kernels.

// Persistent: a CTA stages the weights once and walks the work items
// (image row `row` = n H + y, chunk of CI_PX columns) it = blockIdx.x,
// + gridDim.x, ...  Warp w of the CTA takes the pixel pairs x, x + 1 with
// x = 64 (w / 2) + 2 lane of the chunk and the 16 output channels 16 (w mod
// 2) ..: a thread's two pixels share their 3 x 4 input neighbourhood and
// every 16-byte weight load (8 MACs per load), and 16 channels keep the
// registers low enough for eight resident CTAs.  ReLU and the BF16 rounding
// are one conversion.
constexpr int CI_THREADS = 128, CI_PX = 128;   // pixels of a row per work item
constexpr int CI_PER_SM = 8;                   // resident CTAs
__global__ void __launch_bounds__(CI_THREADS, CI_PER_SM) conv_in_kernel(
    const float* __restrict__ f, const float* __restrict__ P, bf16* __restrict__ Y, int H, int W,
    int nitems) {
    __shared__ __align__(16) float sw[9 * C + C];
    for (int i = threadIdx.x; i < 9 * C + C; i += blockDim.x) sw[i] = round_bf(P[OFF_W1 + i]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = 16 * (warp & 1), q0 = c0 / 8;
    const int nchunk = (W + CI_PX - 1) / CI_PX;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int row = it / nchunk, y = row % H;
        const int x = (it - row * nchunk) * CI_PX + 64 * (warp >> 1) + 2 * lane;
        if (x >= W) continue;
        const bool two = x + 1 < W;
        // v[r][c]: f at image row y + r - 1, column x + c - 1 (zero outside)
        float v[3][4];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int yy = y + r - 1;
            const bool rin = yy >= 0 && yy < H;
            const float* fr = f + (size_t)(rin ? row + r - 1 : row) * (size_t)W;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int xx = x + c - 1;
                v[r][c] = (rin && xx >= 0 && xx < W) ? fr[xx] : 0.0f;
            }
        }
        // weights and bias four output channels per 16-byte shared load
        float a[2][16];
#pragma unroll
        for (int o = 0; o < 16; o += 4) {
            const float4 b4 = *reinterpret_cast<const float4*>(&sw[9 * C + c0 + o]);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                a[k][o] = b4.x;
                a[k][o + 1] = b4.y;
                a[k][o + 2] = b4.z;
                a[k][o + 3] = b4.w;
            }
        }
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
            for (int o = 0; o < 16; o += 4) {
                const float4 w4 = *reinterpret_cast<const float4*>(&sw[t * C + c0 + o]);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float vt = v[t / 3][t % 3 + k];
                    a[k][o] = fmaf(vt, w4.x, a[k][o]);
                    a[k][o + 1] = fmaf(vt, w4.y, a[k][o + 1]);
                    a[k][o + 2] = fmaf(vt, w4.z, a[k][o + 2]);
                    a[k][o + 3] = fmaf(vt, w4.w, a[k][o + 3]);
                }
            }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (k == 1 && !two) break;
            __align__(16) unsigned out[8];   // channels c0 + 2 j (low half), c0 + 2 j + 1
#pragma unroll
            for (int j = 0; j < 8; ++j)
                asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;"
                    : "=r"(out[j])
                    : "f"(a[k][2 * j + 1]), "f"(a[k][2 * j]));
#pragma unroll
            for (int q = 0; q < 2; ++q)
                *reinterpret_cast<uint4*>(Y + act_off((size_t)row, x + k, q0 + q, W)) =
                    reinterpret_cast<const uint4*>(out)[q];
        }
    }
}

// MODE 0: Y = ReLU(conv(X) + bias).  MODE 1: Y = conv(X) * [mask_src > 0]
// (the backward dX of a 32 -> 32 layer, X = dZ, weights flipped and
// transposed).  MODE 2: the output layer, u0 = f + conv(X) + bias[0] with
// one output channel (weights padded to 16 columns, column 0 real).
// Wt: [9][NO out][32 in] BF16.  Persistent: every CTA stages the weights once
// and walks the tiles t = blockIdx.x, + gridDim.x, ..., the halo of the next
// tile loading (cp.async) while the current one is multiplied.
template <int MODE>
constexpr size_t conv_smem_bytes() {
    return (size_t)(2 * HH * HW + 9 * (MODE == 2 ? 16 : C)) * CS * sizeof(bf16);
}

template <int MODE>
__global__ void __launch_bounds__(128, 4) conv_mid_kernel(const bf16* __restrict__ X,
                                                          const bf16* __restrict__ Wt,
                                                          const float* __restrict__ bias,
                                                          const bf16* __restrict__ mask_src,
                                                          bf16* __restrict__ Y,
                                                          const float* __restrict__ f,
                                                          float* __restrict__ u0, int H, int W,
                                                          int ntiles) {
    constexpr int NO = MODE == 2 ? 16 : C;   // MMA output columns
    constexpr int NP = NO / 16;               // ldmatrix x4 loads of B per k-chunk
    extern __shared__ __align__(16) unsigned char conv_smem[];
    bf16(*s_in)[HH * HW][CS] = reinterpret_cast<bf16(*)[HH * HW][CS]>(conv_smem);
    bf16(*s_w)[CS] = reinterpret_cast<bf16(*)[CS]>(conv_smem + 2 * HH * HW * CS * sizeof(bf16));
    for (int i = threadIdx.x; i < 9 * NO * 4; i += blockDim.x) {
        const int row = i >> 2, q = i & 3;
        *reinterpret_cast<uint4*>(&s_w[row][q * 8]) = reinterpret_cast<const uint4*>(Wt)[i];
    }
    int tcur = blockIdx.x;
    if (tcur < ntiles) load_halo_async(s_in[0], X, tile_of(tcur, H, W), H, W);
    cp_async_commit();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lrow = lane & 7, lmat = lane >> 3;
    const int g = lane >> 2, q = lane & 3;
    for (int it = 0; tcur < ntiles; ++it, tcur += gridDim.x) {
        const int buf = it & 1;
        const int tnext = tcur + gridDim.x;
        if (tnext < ntiles) load_halo_async(s_in[buf ^ 1], X, tile_of(tnext, H, W), H, W);
        cp_async_commit();
        cp_async_wait<1>();   // this tile's copies (all but the newest group) have landed
        __syncthreads();
        float acc[2][NO / 8][4];
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
            for (int y = 0; y < NO / 8; ++y)
#pragma unroll
                for (int z = 0; z < 4; ++z) acc[x][y][z] = 0.0f;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int rr = 2 * warp + mt;
                    const int col = lrow + 8 * (lmat & 1);
                    const int pix = (rr + 1 + dy) * HW + (col + 1 + dx);
                    ldsm_x4(a[mt], &s_in[buf][pix][8 * (lmat >> 1) + 16 * kc]);
                }
#pragma unroll
                for (int pr = 0; pr < NP; ++pr) {
                    unsigned bb[4];
                    const int o = 16 * pr + 8 * (lmat >> 1) + lrow;
                    ldsm_x4(bb, &s_w[tap * NO + o][16 * kc + 8 * (lmat & 1)]);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma16816(acc[mt][2 * pr], a[mt], bb[0], bb[1]);
                        mma16816(acc[mt][2 * pr + 1], a[mt], bb[2], bb[3]);
                    }
                }
            }
        }
        const Tile t = tile_of(tcur, H, W);
        const size_t img = (size_t)t.n * H * W;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int gy = t.y0 + 2 * warp + mt;
            if (MODE == 2) {
                if (q == 0) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int gx = t.x0 + g + 8 * h;
                        if (gy >= H || gx >= W) continue;
                        const size_t pp = img + (size_t)gy * W + gx;
                        u0[pp] = f[pp] + (acc[mt][0][2 * h] + bias[0]);
                    }
                }
                continue;
            }
#pragma unroll
            for (int nt = 0; nt < NO / 8; ++nt) {
                const int co = 8 * nt + 2 * q;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int gx = t.x0 + g + 8 * h;
                    if (gy >= H || gx >= W) continue;
                    const size_t pi = act_off((size_t)t.n * H + gy, gx, co >> 3, W) + (co & 7);
                    float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                    if (MODE == 0) {
                        v0 = fmaxf(v0 + bias[co], 0.0f);
                        v1 = fmaxf(v1 + bias[co + 1], 0.0f);
                    } else {
                        const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(mask_src + pi);
                        v0 = bf(m.x) > 0.0f ? v0 : 0.0f;
                        v1 = bf(m.y) > 0.0f ? v1 : 0.0f;
                    }
                    *reinterpret_cast<__nv_bfloat162*>(Y + pi) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncthreads();   // the buffer is refilled two tiles on
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Backward kernels.

// dL/dout = 2 (u0 - u*) / P_total; dZ5 = (sum_tap W6[tap] dL/dout[p - tap]) *
// [X5 > 0]; per-CTA FP64 partial of sum (u0 - u*)^2.
__global__ void __launch_bounds__(256) out_grad_kernel(const float* __restrict__ u0,
                                                       const float* __restrict__ us,
                                                       const float* __restrict__ P,
                                                       const bf16* __restrict__ X5,
                                                       bf16* __restrict__ dZ,
                                                       double* __restrict__ loss_part, int N,
                                                       int H, int W, float scale) {
    __shared__ float sw[9 * C];
    __shared__ double red[8];
    for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) sw[i] = round_bf(P[OFF_W6 + i]);
    __syncthreads();
    const size_t total = (size_t)N * H * W;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (p < total) {
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const size_t img = p - ((size_t)y * W + x);
        const float e = u0[p] - us[p];
        sq = (double)e * (double)e;
        float d[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
            d[t] = 0.0f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const size_t q = img + (size_t)yy * W + xx;
                d[t] = scale * (u0[q] - us[q]);
            }
        }
        const size_t row = p / W;
        __align__(16) bf16 out[C];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = *reinterpret_cast<const uint4*>(X5 + act_off(row, x, q, W));
            const bf16* e8 = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = 8 * q + j;
                float a = 0.0f;
#pragma unroll
                for (int t = 0; t < 9; ++t) a = fmaf(sw[t * C + c], d[t], a);
                out[c] = __float2bfloat16(bf(e8[j]) > 0.0f ? a : 0.0f);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(dZ + act_off(row, x, q, W)) =
                reinterpret_cast<const uint4*>(out)[q];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += red[i];
        loss_part[blockIdx.x] = s;
    }
}

// dW of a 32 -> 32 layer: dW[tap][ci][co] = sum_p X[p + tap][ci] dZ[p][co],
// db[co] = sum_p dZ[p][co].  Warp w owns taps w, w + 4, w + 8.  Partials of
// CTA b go to part + b * DW_STRIDE ([tap][ci][co] then db).
__global__ void __launch_bounds__(128) dw_mid_kernel(const bf16* __restrict__ X,
                                                     const bf16* __restrict__ dZ,
                                                     float* __restrict__ part, int N, int H,
                                                     int W) {
    __shared__ __align__(16) bf16 s_x[HH * HW][CS];
    __shared__ __align__(16) bf16 s_dz[TH * TW][CS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lrow = lane & 7, lmat = lane >> 3;
    float acc[3][2][4][4];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[s][a][b][c] = 0.0f;
    float dbacc = 0.0f;
    const int ntiles = N * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tile_of(ti, H, W);
        __syncthreads();   // the previous tile's readers are done
        load_halo(s_x, X, t, H, W);
        load_tile(s_dz, dZ, t, H, W);
        __syncthreads();
        if (threadIdx.x < C)
            for (int p = 0; p < TH * TW; ++p) dbacc += bf(s_dz[p][threadIdx.x]);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int tap = warp + 4 * s;
            if (tap >= 9) continue;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
#pragma unroll 1
            for (int ry = 0; ry < TH; ++ry) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int px = lrow + 8 * (lmat >> 1);
                    ldsm_x4_t(a[mt], &s_x[(ry + 1 + dy) * HW + (px + 1 + dx)][16 * mt + 8 * (lmat & 1)]);
                }
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    unsigned b[4];
                    const int px = lrow + 8 * (lmat & 1);
                    ldsm_x4_t(b, &s_dz[ry * TW + px][16 * pr + 8 * (lmat >> 1)]);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma16816(acc[s][mt][2 * pr], a[mt], b[0], b[1]);
                        mma16816(acc[s][mt][2 * pr + 1], a[mt], b[2], b[3]);
                    }
                }
            }
        }
    }
    float* out = part + (size_t)blockIdx.x * DW_STRIDE;
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int tap = warp + 4 * s;
        if (tap >= 9) continue;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int ci = 16 * mt + g, co = 8 * nt + 2 * q;
                float* o = out + tap * C * C;
                o[ci * C + co] = acc[s][mt][nt][0];
                o[ci * C + co + 1] = acc[s][mt][nt][1];
                o[(ci + 8) * C + co] = acc[s][mt][nt][2];
                o[(ci + 8) * C + co + 1] = acc[s][mt][nt][3];
            }
    }
    if (threadIdx.x < C) out[MIDW + threadIdx.x] = dbacc;
}

// dW of conv6: dW6[tap][ci] = sum_p X5[p + tap][ci] d[p], db6 = sum_p d[p],
// d = 2 (u0 - u*) / P_total.  Thread (tap, ci).  Partial stride 9 C + 1.
__global__ void __launch_bounds__(288) dw_out_kernel(const bf16* __restrict__ X5,
                                                     const float* __restrict__ u0,
                                                     const float* __restrict__ us,
                                                     float* __restrict__ part, int N, int H,
                                                     int W, float scale) {
    __shared__ __align__(16) bf16 s_x[HH * HW][CS];
    __shared__ float s_d[TH * TW];
    const int tap = threadIdx.x / C, ci = threadIdx.x % C;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    float acc = 0.0f, dacc = 0.0f;
    const int ntiles = N * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tile_of(ti, H, W);
        __syncthreads();
        load_halo(s_x, X5, t, H, W);
        const size_t img = (size_t)t.n * H * W;
        for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
            const int gy = t.y0 + i / TW, gx = t.x0 + i % TW;
            float v = 0.0f;
            if (gy < H && gx < W) {
                const size_t p = img + (size_t)gy * W + gx;
                v = scale * (u0[p] - us[p]);
            }
            s_d[i] = v;
        }
        __syncthreads();
        for (int p = 0; p < TH * TW; ++p) {
            const int py = p / TW, px = p % TW;
            acc = fmaf(bf(s_x[(py + 1 + dy) * HW + (px + 1 + dx)][ci]), s_d[p], acc);
        }
        if (threadIdx.x == 0)
            for (int p = 0; p < TH * TW; ++p) dacc += s_d[p];
    }
    float* out = part + (size_t)blockIdx.x * (9 * C + 1);
    out[tap * C + ci] = acc;
    if (threadIdx.x == 0) out[9 * C] = dacc;
}

// dW of conv1: dW1[tap][co] = sum_p f[p + tap] dZ1[p][co], db1 = sum_p dZ1.
// Thread (tap, co).  Partial stride 9 C + C.
__global__ void __launch_bounds__(288) dw_in_kernel(const float* __restrict__ f,
                                                    const bf16* __restrict__ dZ,
                                                    float* __restrict__ part, int N, int H,
                                                    int W) {
    __shared__ float s_f[HH * HW];
    __shared__ __align__(16) bf16 s_dz[TH * TW][CS];
    const int tap = threadIdx.x / C, co = threadIdx.x % C;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    float acc = 0.0f, bacc = 0.0f;
    const int ntiles = N * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const Tile t = tile_of(ti, H, W);
        __syncthreads();
        const size_t img = (size_t)t.n * H * W;
        for (int i = threadIdx.x; i < HH * HW; i += blockDim.x) {
            const int gy = t.y0 - 1 + i / HW, gx = t.x0 - 1 + i % HW;
            s_f[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? f[img + (size_t)gy * W + gx] : 0.0f;
        }
        load_tile(s_dz, dZ, t, H, W);
        __syncthreads();
        for (int p = 0; p < TH * TW; ++p) {
            const int py = p / TW, px = p % TW;
            const float g = bf(s_dz[p][co]);
            acc = fmaf(s_f[(py + 1 + dy) * HW + (px + 1 + dx)], g, acc);
            if (tap == 0) bacc += g;
        }
    }
    float* out = part + (size_t)blockIdx.x * (9 * C + C);
    out[tap * C + co] = acc;
    if (tap == 0) out[9 * C + co] = bacc;
}

// out[i] = sum_{b < nb} part[b * stride + i], fixed order.
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nb, int stride, int count,
                                    float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * stride + i];
    out[i] = s;
}

__global__ void reduce_loss_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of the 32 -> 32 weights: forward [tap][co][ci] (transpose of
// the master [tap][ci][co]) and backward [tap][ci][co] with the tap flipped
// (dX = conv(dZ, W'), W'[tap][ci][co] = W[8 - tap][ci][co]).
__global__ void pack_kernel(const float* __restrict__ P, bf16* __restrict__ wf,
                            bf16* __restrict__ wb, bf16* __restrict__ w6p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 9 * 16 * C) {   // output layer: [tap][16 out][32 in], column 0 real
        const int tap = i / (16 * C), o = (i / C) % 16, ci = i % C;
        w6p[i] = __float2bfloat16(o == 0 ? P[OFF_W6 + tap * C + ci] : 0.0f);
    }
    if (i >= 4 * MIDW) return;
    const int l = i / MIDW, r = i % MIDW;
    const int tap = r / (C * C), ci = (r / C) % C, co = r % C;
    const float w = P[off_w(l + 2) + r];
    wf[l * MIDW + tap * C * C + co * C + ci] = __float2bfloat16(w);
    wb[l * MIDW + (8 - tap) * C * C + ci * C + co] = __float2bfloat16(w);
}

// ---------------------------------------------------------------------------
// 5th-generation tensor cores (tcgen05): the same convolutions with the
// accumulators in tensor memory.  A work unit is a strip of TR = 4 output
// rows x 128 columns.  Output row o of the strip is one M = 128 (pixels) x NO
// (channels) accumulator slot in TMEM, the TR slots side by side.  The three
// vertical taps of one input row share their A operand, so one tcgen05.mma
// with the weights of several taps side by side along N adds that input
// row's contribution to several output rows at once: input row hr of the
// halo (image row r0 - 1 + hr) feeds output row o = hr - 2 + jj through the
// tap dy = 1 - jj, jj = 0, 1, 2, and the jj with 0 <= o < TR form one
// contiguous range of slots.  So per input row, horizontal tap and K-step of
// 16 input channels one MMA of N = NO, 2 NO or 3 NO (rows 0 and TR + 1: one
// output row; rows 1 and TR: two; the rest: three): per strip 36 MMAs doing
// exactly the strip's TR x 9 x 32 products, after one MMA with zero operands
// (no accumulate) that clears the set.  The halo of the strip (6 rows x 136
// pixels, the 130 it needs widened to whole groups of 4) is loaded by TMA
// (four tile copies, one per plane of 8 channels, zero outside the tensor;
// the row pad is zeroed after the copy), so plane j holds channels 8j ..
// 8j + 7 of every pixel, 16 bytes each: 8 consecutive pixels are one
// 128-byte core matrix of the no-swizzle K-major layout, and the operand of
// input row hr and horizontal tap dx is that layout started hr rows and dx
// pixels further on (descriptor start = plane + pixel x 16 B, K-direction
// byte offset = the plane stride, M-direction byte offset = 128 B).  The
// weights are staged the same way, [dx][plane][jj NO + n] x 16 B, so the
// taps of a range of jj are one operand too.
//
// Pipeline (one CTA per SM, persistent over strips): one thread waits for a
// strip's halo, issues its 37 MMAs into one of NSET TMEM accumulator sets
// and commits them to an mbarrier; meanwhile the drain warps empty the sets
// of earlier strips (tcgen05.ld; a warp reads the TMEM lanes of its lane
// quarter), and as soon as a strip's MMAs are known complete its halo buffer
// is refilled by TMA with a strip NSTAGE further on.  Every wait is bounded.

constexpr int TR = 4, TXC = 128;                         // strip: 4 rows x 128 columns
constexpr int NSTAGE = 4;                                // halo buffers in flight
constexpr int NSET = 4;                                  // TMEM accumulator sets
constexpr unsigned TSET = 128;                           // TMEM columns per set (TR x NO)
// The halo of a strip at columns x0 .. x0 + 127 is loaded as 34 groups of 4
// pixels, x0 - 4 .. x0 + 131 (halo pixel i is column x0 - 4 + i), so
// column x0 - 1 is halo pixel HOFF.
constexpr int HRW = TR + 2, HCL = TXC + 8, HOFF = 3;     // halo rows / columns
constexpr unsigned PLANE_DATA = HRW * HCL * 16;          // bytes of one plane
constexpr unsigned PLANE = (PLANE_DATA + 127) & ~127u;   // plane stride (TMA: 128-byte aligned)
constexpr unsigned HALO_BYTES = 4 * PLANE;
// Zero operands of the clearing MMA: A = 128 pixels x 2 planes, B = TR NO
// <= 128 rows x 2 planes, both read from one zero-filled region.
constexpr unsigned ZERO_BYTES = 2 * 128 * 16;
static_assert(NSET * TSET <= 512 && TR * C <= (int)TSET, "TMEM accumulator sets");

template <int MODE>
constexpr int tc_no() { return MODE == 2 ? 16 : C; }

template <int MODE>
constexpr size_t tc_smem_bytes() {
    return 128 + NSTAGE * (size_t)HALO_BYTES + 9 * 4 * (size_t)tc_no<MODE>() * 16 +
           ZERO_BYTES + 128;
}
static_assert(tc_smem_bytes<0>() <= 227 * 1024, "conv_tc shared memory");

__device__ __forceinline__ uint64_t umma_sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version; base offset 0, no swizzle
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr unsigned umma_idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem, uint64_t a, uint64_t b, unsigned idesc,
                                       unsigned accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Wait for phase `parity` of an mbarrier, giving up after `limit` tries
// (false: timed out; the caller sets its error status and returns).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned mbar, unsigned parity,
                                                  int limit = 1 << 22) {
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
            "selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Failure-detection self-test of the bounded wait: phase 0 of a fresh
// mbarrier (arrival count 1) that nothing arrives on must time out; after
// one arrival the same wait must see the phase complete.  out[0] = 1 on the
// timeout, out[1] = 1 on the completion.
__global__ void wait_selftest_kernel(int limit, int* out) {
    __shared__ alignas(8) unsigned long long bar;
    const unsigned mbar = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    out[0] = mbar_wait_bounded(mbar, 0u, limit) ? 0 : 1;
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
    out[1] = mbar_wait_bounded(mbar, 0u, limit) ? 1 : 0;
}

__device__ __forceinline__ void tmem_ld32(unsigned taddr, unsigned (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld1(unsigned taddr, unsigned& r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
}

// Strip u of the batch: image n, rows y0 .., columns x0 ..
struct Strip {
    int n, y0, x0;
};
__device__ __forceinline__ Strip strip_of(int u, int H, int W) {
    const int sx = (W + TXC - 1) / TXC, sy = (H + TR - 1) / TR;
    Strip s;
    s.n = u / (sx * sy);
    const int rem = u - s.n * sx * sy;
    s.y0 = (rem / sx) * TR;
    s.x0 = (rem % sx) * TXC;
    return s;
}

// TMA: the halo of strip s into `halo` (four planes), completing on lbar.
__device__ __forceinline__ void tma_strip(unsigned halo, unsigned lbar, const CUtensorMap* tmap,
                                          const Strip& s) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lbar),
                 "r"(4 * PLANE_DATA)
                 : "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j)
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(halo + j * PLANE),
            "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(s.x0 / 4 - 1), "r"(j), "r"(s.y0 - 1),
            "r"(s.n), "r"(lbar)
            : "memory");
}

// MODE 0: Y = ReLU(conv(X) + bias).  MODE 1: Y = conv(X) * [mask_src > 0].
// MODE 2: u0 = f + conv(X) + bias[0] (one output channel of 16 MMA columns).
// tmap: X as (4 pixels x 8 channels, Wp / 4, 4 planes, H, N) BF16, box (32, 34, 1, TR + 2,
// 1).  status:
// set to 1 if a wait timed out (the kernel then stops; results are invalid).
// Warp-specialised: warp TC_DRAIN = 8 (one lane) is the producer (TMA, MMA
// issue); warps 0..7 drain the accumulators: a warp reads the TMEM lanes of
// its quarter, 32 (w mod 4) .., and warps w and w + 4 take the even and odd
// rows of a strip, so two TMEM loads per lane quarter are in flight.  Strip
// k uses halo buffer k % NSTAGE and TMEM set k % NSET: lbar[k % NSTAGE] =
// halo landed, mbar[k % NSET] = MMAs done, tfree[k % NSET] = accumulators
// drained (one arrival per drain warp), so the MMAs of strip k wait only for
// the drain of strip k - NSET.  The halo of strip k + NSTAGE - 1 is
// requested as soon as strip k - 1's MMAs are done, NSTAGE - 1 strips ahead
// of its use.
constexpr int TC_DRAIN = 8;                      // drain warps (two per TMEM lane quarter)
constexpr int TC_THREADS = 32 * (TC_DRAIN + 1);

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) conv_tc_kernel(
    const __grid_constant__ CUtensorMap tmap, const bf16* __restrict__ Wt,
    const float* __restrict__ bias, const bf16* __restrict__ mask_src, bf16* __restrict__ Y,
    const float* __restrict__ f, float* __restrict__ u0, int H, int W, int nunits,
    int* __restrict__ status) {
    constexpr int NO = tc_no<MODE>();
    constexpr int N3 = 3 * NO;                               // weight rows per (dx, plane)
    constexpr unsigned IDESC_ZERO = umma_idesc_bf16(TR * NO);
    static_assert((NO % 16) == 0 && TR * NO <= 128, "MMA N of M = 128; zero operand rows");
    extern __shared__ unsigned char tc_raw[];
    unsigned char* tc_smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(tc_raw) + 127) & ~(uintptr_t)127);   // TMA: 128-byte aligned
    unsigned char* halo = tc_smem;                                // NSTAGE buffers
    unsigned char* wsm = tc_smem + NSTAGE * HALO_BYTES;           // [dx][plane][N3] x 16 B
    unsigned char* zsm = wsm + 9 * 4 * NO * 16;                   // zero operands
    uint64_t* bars = reinterpret_cast<uint64_t*>(zsm + ZERO_BYTES);
    unsigned* tslot = reinterpret_cast<unsigned*>(bars + NSTAGE + 2 * NSET);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned lbar0 = smem_addr(bars), mbar0 = lbar0 + 8 * NSTAGE, tfree0 = mbar0 + 8 * NSET;
    const unsigned hbase0 = smem_addr(halo), wbase = smem_addr(wsm), zbase = smem_addr(zsm);

    // Wt: [tap][n][plane] x 16 B, tap = (dy + 1) 3 + (dx + 1); staged as
    // [dx][plane][jj NO + n] with jj = 2 - (dy + 1)
    for (int i = tid; i < 9 * NO * 4; i += blockDim.x) {
        const int j = i & 3, n = (i >> 2) % NO, tap = (i >> 2) / NO;
        const int ty = tap / 3, tx = tap - 3 * ty;
        *reinterpret_cast<uint4*>(wsm + ((tx * 4 + j) * N3 + (2 - ty) * NO + n) * 16) =
            reinterpret_cast<const uint4*>(Wt)[i];
    }
    for (int i = tid; i < (int)(ZERO_BYTES / 16); i += blockDim.x)
        reinterpret_cast<uint4*>(zsm)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int i = 0; i < NSTAGE + NSET; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(lbar0 + 8 * i));
        for (int i = 0; i < NSET; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tfree0 + 8 * i),
                         "r"(TC_DRAIN));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == TC_DRAIN) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
            smem_addr(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tslot;
    const int G = gridDim.x;
    const int nmine = (int)blockIdx.x < nunits ? (nunits - 1 - (int)blockIdx.x) / G + 1 : 0;

    if (warp == TC_DRAIN) {
        if (lane == 0) {
            // producer: halo loads and MMAs.  issued / landed count the strips
            // whose halo load was requested / seen complete; committed the
            // strips whose MMAs were committed (for the drain on abort).
            int issued = 0, landed = 0, committed = 0;
            for (int k = 0; k < NSTAGE && k < nmine; ++k, ++issued)
                tma_strip(hbase0 + k * HALO_BYTES, lbar0 + 8 * k, &tmap,
                          strip_of(blockIdx.x + k * G, H, W));
            const uint64_t bdesc0 = umma_sdesc(wbase, N3 * 16, 128);
            // clearing MMA: A = 128 zero pixels (plane stride 2 KB), B = TR NO
            // zero rows (plane stride TR NO x 16 B)
            const uint64_t azero = umma_sdesc(zbase, 128 * 16, 128);
            const uint64_t bzero = umma_sdesc(zbase, TR * NO * 16, 128);
            for (int k = 0; k < nmine; ++k) {
                const int hb = k % NSTAGE, b = k % NSET;
                bool ok = mbar_wait_bounded(lbar0 + 8 * hb, (unsigned)((k / NSTAGE) & 1));
                if (ok) landed = k + 1;
                if (ok && k >= NSET)
                    ok = mbar_wait_bounded(tfree0 + 8 * b, (unsigned)((k / NSET - 1) & 1));
                if (!ok || *abort_flag) {
                    *abort_flag = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if ((W & 3) != 0) {
                    // the row pad W .. Wp - 1 lies inside the padded tensor, so
                    // the TMA copied it (never written): zero it in the halo
                    // before the MMAs read it as the image's right border
                    const Strip s = strip_of(blockIdx.x + k * G, H, W);
                    const int i0 = W - s.x0 + 4, i1 = min(act_wp(W) - s.x0 + 4, HCL);
                    if (i0 < HCL) {
                        unsigned char* hp = halo + hb * HALO_BYTES;
                        for (int j = 0; j < 4; ++j)
                            for (int hr = 0; hr < HRW; ++hr)
                                for (int i = i0; i < i1; ++i)
                                    *reinterpret_cast<uint4*>(hp + j * PLANE + (hr * HCL + i) * 16) =
                                        make_uint4(0u, 0u, 0u, 0u);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    }
                }
                const uint64_t adesc0 = umma_sdesc(hbase0 + hb * HALO_BYTES, PLANE, 128);
                const unsigned dset = tmem + b * TSET;
                tc_mma(dset, azero, bzero, IDESC_ZERO, 0u);
#pragma unroll
                for (int hr = 0; hr < HRW; ++hr) {
                    // output rows hr - 2 + jj for jj = jlo .. jhi, the ones inside
                    // the strip: slots hr - 2 + jlo .., weight rows jlo NO ..
                    const int jlo = hr < 2 ? 2 - hr : 0, jhi = hr > TR - 1 ? TR + 1 - hr : 2;
                    const unsigned idesc = umma_idesc_bf16((jhi - jlo + 1) * NO);
                    const unsigned d = dset + (unsigned)((hr - 2 + jlo) * NO);
#pragma unroll
                    for (int tx = 0; tx < 3; ++tx) {
                        const unsigned pix = (unsigned)(hr * HCL + HOFF + tx);
#pragma unroll
                        for (int kc = 0; kc < 2; ++kc)
                            tc_mma(d, adesc0 + ((2 * kc * PLANE + pix * 16) >> 4),
                                   bdesc0 + ((((tx * 4 + 2 * kc) * N3 + jlo * NO) * 16) >> 4),
                                   idesc, 1u);
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        mbar0 + 8 * b)
                    : "memory");
                committed = k + 1;
                // strip k - 1's MMAs done: its halo buffer takes strip k - 1 + NSTAGE
                if (k >= 1 && k - 1 + NSTAGE < nmine) {
                    if (!mbar_wait_bounded(mbar0 + 8 * ((k - 1) % NSET),
                                           (unsigned)(((k - 1) / NSET) & 1))) {
                        *abort_flag = 1;
                        break;
                    }
                    const int hbo = (k - 1) % NSTAGE;
                    tma_strip(hbase0 + hbo * HALO_BYTES, lbar0 + 8 * hbo, &tmap,
                              strip_of(blockIdx.x + (k - 1 + NSTAGE) * G, H, W));
                    ++issued;
                }
            }
            // Drain before the CTA frees its TMEM and exits: wait (bounded) for
            // every halo load still in flight into shared memory (at most one
            // per buffer, so each has its own phase; none on the normal path)
            // and for the last commit, which covers every MMA issued before it
            // (on the normal path the drain warps wait for it as well).
            for (int k = landed; k < issued; ++k)
                mbar_wait_bounded(lbar0 + 8 * (k % NSTAGE), (unsigned)((k / NSTAGE) & 1));
            if (committed > 0) {
                const int kc = committed - 1;
                mbar_wait_bounded(mbar0 + 8 * (kc % NSET), (unsigned)((kc / NSET) & 1));
            }
        }
    } else {
        // drain warps
        float bias_r[MODE == 0 ? C : 1];
        if (MODE == 0) {
#pragma unroll
            for (int o = 0; o < C; ++o) bias_r[o] = bias[o];
        }
        for (int k = 0; k < nmine; ++k) {
            const int b = k % NSET;
            if (!mbar_wait_bounded(mbar0 + 8 * b, (unsigned)((k / NSET) & 1)) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const Strip s = strip_of(blockIdx.x + k * G, H, W);
            const int quarter = warp & 3;
            const int gx = s.x0 + 32 * quarter + lane;
            const size_t img = (size_t)s.n * H * W;
            const unsigned lanebase = tmem + b * TSET + ((unsigned)(32 * quarter) << 16);
            for (int r = warp >> 2; r < TR; r += 2) {
                const int gy = s.y0 + r;
                if (MODE == 2) {
                    unsigned v;
                    tmem_ld1(lanebase + (unsigned)(r * NO), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (gy < H && gx < W) {
                        const size_t pp = img + (size_t)gy * W + gx;
                        u0[pp] = f[pp] + (__uint_as_float(v) + bias[0]);
                    }
                    continue;
                }
                unsigned v[32];
                tmem_ld32(lanebase + (unsigned)(r * NO), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (gy >= H || gx >= W) continue;
                const size_t row = (size_t)s.n * H + gy;
                __align__(16) bf16 out[C];
                if (MODE == 0) {
#pragma unroll
                    for (int o = 0; o < C; ++o)
                        out[o] = __float2bfloat16(fmaxf(__uint_as_float(v[o]) + bias_r[o], 0.0f));
                } else {
                    __align__(16) bf16 m[C];
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4)
                        reinterpret_cast<uint4*>(m)[q4] =
                            *reinterpret_cast<const uint4*>(mask_src + act_off(row, gx, q4, W));
#pragma unroll
                    for (int o = 0; o < C; ++o)
                        out[o] = __float2bfloat16(bf(m[o]) > 0.0f ? __uint_as_float(v[o]) : 0.0f);
                }
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4)
                    *reinterpret_cast<uint4*>(Y + act_off(row, gx, q4, W)) =
                        reinterpret_cast<const uint4*>(out)[q4];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tfree0 + 8 * b) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag && tid == 0) atomicExch(status, 1);
    if (warp == TC_DRAIN) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
}

// ---------------------------------------------------------------------------
// Host side.

#ifndef CM_CNN_TC
#define CM_CNN_TC 1
#endif

// Dynamic shared memory above 48 KB must be allowed per kernel.
cudaError_t conv_setup() {
    if (CM_CNN_TC) {
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_smem_bytes<0>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_smem_bytes<1>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_smem_bytes<2>());
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(conv_mid_kernel<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)conv_smem_bytes<0>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(conv_mid_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)conv_smem_bytes<1>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(conv_mid_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)conv_smem_bytes<2>());
    return e;
}

// The driver's tensor-map encoder, fetched once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// TMA map of an activation tensor X (the plane-major layout of act_off:
// groups of 4 pixels x 8 channels, Wp / 4 groups, 4 planes, H rows, N
// images) with the halo box of the tcgen05 convolution: 34 groups (136
// columns) of one plane x HRW rows of one image, zero outside the tensor.
cudaError_t act_tensor_map(CUtensorMap* m, const bf16* X, int N, int H, int W) {
    auto fn = tensor_map_encoder();
    if (!fn) return cudaErrorNotSupported;
    // (32 = 4 pixels x 8 channels, Wp / 4 pixel groups, 4 planes, H, N)
    const int Wp = act_wp(W);
    const cuuint64_t dims[5] = {32, (cuuint64_t)(Wp / 4), 4, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[4] = {(cuuint64_t)32 * sizeof(bf16), (cuuint64_t)Wp * 8 * sizeof(bf16),
                                   (cuuint64_t)Wp * C * sizeof(bf16),
                                   (cuuint64_t)H * Wp * C * sizeof(bf16)};
    const cuuint32_t box[5] = {32, (cuuint32_t)(HCL / 4), 1, (cuuint32_t)HRW, 1};
    const cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(X), dims, strides,
                          box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

struct Net {
    int device = 0;
    std::string err;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    bf16 *wf = nullptr, *wb = nullptr, *w6p = nullptr;
    int step = 0;
    int conv_grid = 0;      // persistent CTAs of the mma.sync convolutions
    int tc_grid = 0;        // persistent CTAs of the tcgen05 convolutions (one per SM)
    int ci_grid = 0;        // persistent CTAs of the first layer
    int* status = nullptr;  // device: set when a tensor-core wait timed out
    // activations (capacity in pixels)
    size_t cap = 0;
    bf16* act[6] = {};      // act[1..5] = X1..X5
    bf16* dz[2] = {};
    float* u0 = nullptr;
    float* part = nullptr;  // weight-gradient partials
    double* lpart = nullptr;
    size_t lpart_cap = 0;
    double* loss = nullptr;
};

namespace {

#define NET_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) {                                    \
            net->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
            return e_ == cudaErrorMemoryAllocation ? CM_ERR_OOM : CM_ERR_CUDA; \
        }                                                           \
    } while (0)

// npx: pixels of the padded activation rows, N H act_wp(W).
int ensure_acts(Net* net, size_t npx) {
    if (npx <= net->cap) return CM_OK;
    for (int i = 1; i <= 5; ++i)
        if (net->act[i]) cudaFree(net->act[i]);
    for (int i = 0; i < 2; ++i)
        if (net->dz[i]) cudaFree(net->dz[i]);
    if (net->u0) cudaFree(net->u0);
    if (net->lpart) cudaFree(net->lpart);
    net->cap = 0;
    for (int i = 1; i <= 5; ++i) NET_CUDA(cudaMalloc(&net->act[i], npx * C * sizeof(bf16)));
    for (int i = 0; i < 2; ++i) NET_CUDA(cudaMalloc(&net->dz[i], npx * C * sizeof(bf16)));
    NET_CUDA(cudaMalloc(&net->u0, npx * sizeof(float)));
    NET_CUDA(cudaMalloc(&net->lpart, ((npx + 255) / 256) * sizeof(double)));
    net->cap = npx;
    return CM_OK;
}

int pack(Net* net, cudaStream_t st) {
    pack_kernel<<<(4 * MIDW + 255) / 256, 256, 0, st>>>(net->P, net->wf, net->wb, net->w6p);
    NET_CUDA(cudaGetLastError());
    return CM_OK;
}

int forward(Net* net, const float* f, int N, int H, int W, float* u0, cudaStream_t st) {
    const size_t npx = (size_t)N * H * W;
    const int ci_items = N * H * ((W + CI_PX - 1) / CI_PX);
    conv_in_kernel<<<std::min(ci_items, net->ci_grid), CI_THREADS, 0, st>>>(f, net->P, net->act[1],
                                                                           H, W, ci_items);
    if (CM_CNN_TC) {
        const int nunits = N * ((H + TR - 1) / TR) * ((W + TXC - 1) / TXC);
        const int grid = std::min(nunits, net->tc_grid);
        CUtensorMap m;
        for (int l = 2; l <= 5; ++l) {
            NET_CUDA(act_tensor_map(&m, net->act[l - 1], N, H, W));
            conv_tc_kernel<0><<<grid, TC_THREADS, tc_smem_bytes<0>(), st>>>(
                m, net->wf + (l - 2) * MIDW, net->P + off_b(l), nullptr, net->act[l], nullptr,
                nullptr, H, W, nunits, net->status);
        }
        NET_CUDA(act_tensor_map(&m, net->act[5], N, H, W));
        conv_tc_kernel<2><<<grid, TC_THREADS, tc_smem_bytes<2>(), st>>>(
            m, net->w6p, net->P + OFF_B6, nullptr, nullptr, f, u0, H, W, nunits, net->status);
    } else {
        const int ntiles = N * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
        const int grid = std::min(ntiles, net->conv_grid);
        for (int l = 2; l <= 5; ++l)
            conv_mid_kernel<0><<<grid, 128, conv_smem_bytes<0>(), st>>>(
                net->act[l - 1], net->wf + (l - 2) * MIDW, net->P + off_b(l), nullptr, net->act[l],
                nullptr, nullptr, H, W, ntiles);
        conv_mid_kernel<2><<<grid, 128, conv_smem_bytes<2>(), st>>>(
            net->act[5], net->w6p, net->P + OFF_B6, nullptr, nullptr, f, u0, H, W, ntiles);
    }
    NET_CUDA(cudaGetLastError());
    return CM_OK;
}

// Gradients of the mean squared error into net->G; loss sum into net->loss.
int backward(Net* net, const float* f, const float* us, int N, int H, int W, cudaStream_t st) {
    const size_t npx = (size_t)N * H * W;
    const int ntiles = N * ((H + TH - 1) / TH) * ((W + TW - 1) / TW);
    const int nb = (int)((npx + 255) / 256);
    const float scale = 2.0f / (float)npx;
    out_grad_kernel<<<nb, 256, 0, st>>>(net->u0, us, net->P, net->act[5], net->dz[0], net->lpart,
                                        N, H, W, scale);
    reduce_loss_kernel<<<1, 256, 0, st>>>(net->lpart, nb, net->loss);
    const int g6 = std::min(ntiles, DW_GRID);
    dw_out_kernel<<<g6, 288, 0, st>>>(net->act[5], net->u0, us, net->part, N, H, W, scale);
    reduce_parts_kernel<<<(9 * C + 1 + 255) / 256, 256, 0, st>>>(net->part, g6, 9 * C + 1, 9 * C + 1,
                                                                 net->G + OFF_W6);
    int cur = 0;   // dz[cur] holds dZ of layer l's output
    for (int l = 5; l >= 2; --l) {
        const int gm = std::min(ntiles, DW_GRID);
        dw_mid_kernel<<<gm, 128, 0, st>>>(net->act[l - 1], net->dz[cur], net->part, N, H, W);
        reduce_parts_kernel<<<(DW_STRIDE + 255) / 256, 256, 0, st>>>(net->part, gm, DW_STRIDE,
                                                                     DW_STRIDE, net->G + off_w(l));
        if (CM_CNN_TC) {
            const int nunits = N * ((H + TR - 1) / TR) * ((W + TXC - 1) / TXC);
            CUtensorMap m;
            NET_CUDA(act_tensor_map(&m, net->dz[cur], N, H, W));
            conv_tc_kernel<1><<<std::min(nunits, net->tc_grid), TC_THREADS, tc_smem_bytes<1>(), st>>>(
                m, net->wb + (l - 2) * MIDW, nullptr, net->act[l - 1], net->dz[cur ^ 1], nullptr,
                nullptr, H, W, nunits, net->status);
        } else {
            conv_mid_kernel<1><<<std::min(ntiles, net->conv_grid), 128, conv_smem_bytes<1>(), st>>>(
                net->dz[cur], net->wb + (l - 2) * MIDW, nullptr, net->act[l - 1], net->dz[cur ^ 1],
                nullptr, nullptr, H, W, ntiles);
        }
        cur ^= 1;
    }
    const int g1 = std::min(ntiles, DW_GRID);
    dw_in_kernel<<<g1, 288, 0, st>>>(f, net->dz[cur], net->part, N, H, W);
    reduce_parts_kernel<<<(9 * C + C + 255) / 256, 256, 0, st>>>(net->part, g1, 9 * C + C, 9 * C + C,
                                                                 net->G + OFF_W1);
    NET_CUDA(cudaGetLastError());
    return CM_OK;
}

int check_images(Net* net, const float* f, int N, int H, int W) {
    // (pixels of the batch < 2^31: the kernels index rows and strips in int)
    if (!f || N < 1 || H < 1 || W < 1 || H > CM_MAX_SIDE || W > CM_MAX_SIDE ||
        (long long)H * W > CM_MAX_PIXELS || (long long)N * H * W > 0x7fffffffLL) {
        net->err = "invalid image arguments";
        return CM_ERR_INVALID;
    }
    return CM_OK;
}

}  // namespace

// Exposed to the runtime (cm_warmstart).
int net_forward(Net* net, const float* f, int N, int H, int W, float* u0, cudaStream_t st) {
    int rc = check_images(net, f, N, H, W);
    if (rc || !u0) return rc ? rc : CM_ERR_INVALID;
    NET_CUDA(cudaSetDevice(net->device));
    rc = ensure_acts(net, (size_t)N * H * act_wp(W));
    if (rc) return rc;
    return forward(net, f, N, H, W, u0, st);
}

// Forward into the net's own u0 buffer (the training paths).
int net_forward_own(Net* net, const float* f, int N, int H, int W, cudaStream_t st) {
    int rc = check_images(net, f, N, H, W);
    if (rc) return rc;
    NET_CUDA(cudaSetDevice(net->device));
    rc = ensure_acts(net, (size_t)N * H * act_wp(W));
    if (rc) return rc;
    return forward(net, f, N, H, W, net->u0, st);
}

const char* net_error(const Net* net) { return net->err.c_str(); }

// After a synchronisation: CM_ERR_TIMEOUT if a tensor-core wait timed out.
int net_status(Net* net) {
    int h = 0;
    NET_CUDA(cudaMemcpy(&h, net->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        net->err = "tensor-core convolution: a wait for the MMAs timed out";
        return CM_ERR_TIMEOUT;
    }
    return CM_OK;
}

}  // namespace cnn
}  // namespace cm

using cm::cnn::Net;

struct cm_net : public Net {};

extern "C" {

int cm_net_num_params(void) { return cm::cnn::NPAR; }

int cm_net_create(cm_ctx* ctx, cm_net** out) {
    if (!ctx || !out) return CM_ERR_INVALID;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CM_ERR_CUDA;
    cm_net* net = new cm_net();
    net->device = dev;
    const size_t np = cm::cnn::NPAR * sizeof(float);
    cudaError_t e = cudaMalloc(&net->P, np);
    if (e == cudaSuccess) e = cudaMalloc(&net->G, np);
    if (e == cudaSuccess) e = cudaMalloc(&net->M, np);
    if (e == cudaSuccess) e = cudaMalloc(&net->V, np);
    if (e == cudaSuccess) e = cudaMalloc(&net->wf, 4 * cm::cnn::MIDW * sizeof(cm::cnn::bf16));
    if (e == cudaSuccess) e = cudaMalloc(&net->wb, 4 * cm::cnn::MIDW * sizeof(cm::cnn::bf16));
    if (e == cudaSuccess) e = cudaMalloc(&net->w6p, 9 * 16 * cm::cnn::C * sizeof(cm::cnn::bf16));
    if (e == cudaSuccess) {
        int nsm = 0;
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, net->device);
        net->conv_grid = 4 * nsm;   // four resident CTAs per SM (shared memory, registers)
        net->tc_grid = nsm;         // one CTA per SM (shared memory; one TMEM allocation)
        net->ci_grid = cm::cnn::CI_PER_SM * nsm;
    }
    if (e == cudaSuccess) e = cudaMalloc(&net->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(net->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cm::cnn::conv_setup();
    if (e == cudaSuccess)
        e = cudaMalloc(&net->part, (size_t)cm::cnn::DW_GRID * cm::cnn::DW_STRIDE * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&net->loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(net->P, 0, np);
    if (e == cudaSuccess) e = cudaMemset(net->M, 0, np);
    if (e == cudaSuccess) e = cudaMemset(net->V, 0, np);
    if (e == cudaSuccess) e = cudaMemset(net->G, 0, np);
    if (e != cudaSuccess) {
        cm_net_destroy(net);
        return e == cudaErrorMemoryAllocation ? CM_ERR_OOM : CM_ERR_CUDA;
    }
    if (cm::cnn::pack(net, 0) != CM_OK || cudaDeviceSynchronize() != cudaSuccess) {
        cm_net_destroy(net);
        return CM_ERR_CUDA;
    }
    *out = net;
    return CM_OK;
}

void cm_net_destroy(cm_net* net) {
    if (!net) return;
    cudaSetDevice(net->device);
    for (float* p : {net->P, net->G, net->M, net->V, net->u0, net->part})
        if (p) cudaFree(p);
    if (net->wf) cudaFree(net->wf);
    if (net->w6p) cudaFree(net->w6p);
    if (net->status) cudaFree(net->status);
    if (net->wb) cudaFree(net->wb);
    for (int i = 1; i <= 5; ++i)
        if (net->act[i]) cudaFree(net->act[i]);
    for (int i = 0; i < 2; ++i)
        if (net->dz[i]) cudaFree(net->dz[i]);
    if (net->lpart) cudaFree(net->lpart);
    if (net->loss) cudaFree(net->loss);
    delete net;
}

const char* cm_net_last_error(const cm_net* net) { return net ? net->err.c_str() : "null net"; }

int cm_net_set_params(cm_net* net, const float* host) {
    if (!net || !host) return CM_ERR_INVALID;
    NET_CUDA(cudaSetDevice(net->device));
    const size_t np = cm::cnn::NPAR * sizeof(float);
    NET_CUDA(cudaMemcpy(net->P, host, np, cudaMemcpyHostToDevice));
    NET_CUDA(cudaMemset(net->M, 0, np));
    NET_CUDA(cudaMemset(net->V, 0, np));
    net->step = 0;
    int rc = cm::cnn::pack(net, 0);
    if (rc) return rc;
    NET_CUDA(cudaDeviceSynchronize());
    return CM_OK;
}

int cm_net_get_params(cm_net* net, float* host) {
    if (!net || !host) return CM_ERR_INVALID;
    NET_CUDA(cudaSetDevice(net->device));
    NET_CUDA(cudaMemcpy(host, net->P, cm::cnn::NPAR * sizeof(float), cudaMemcpyDeviceToHost));
    return CM_OK;
}

int cm_net_forward(cm_net* net, const float* f, int N, int H, int W, float* u0_out, void* stream) {
    if (!net) return CM_ERR_INVALID;
    return cm::cnn::net_forward(net, f, N, H, W, u0_out, (cudaStream_t)stream);
}

int cm_net_gradients(cm_net* net, const float* f, const float* ustar, int N, int H, int W,
                     float* grad_host, double* loss_host, void* stream) {
    if (!net || !ustar) return CM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cm::cnn::net_forward_own(net, f, N, H, W, st);
    if (rc) return rc;
    rc = cm::cnn::backward(net, f, ustar, N, H, W, st);
    if (rc) return rc;
    NET_CUDA(cudaStreamSynchronize(st));
    rc = cm::cnn::net_status(net);
    if (rc) return rc;
    if (grad_host)
        NET_CUDA(cudaMemcpy(grad_host, net->G, cm::cnn::NPAR * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss_host) {
        double s = 0.0;
        NET_CUDA(cudaMemcpy(&s, net->loss, sizeof(double), cudaMemcpyDeviceToHost));
        *loss_host = s / ((double)N * H * W);
    }
    return CM_OK;
}

int cm_net_train_step(cm_net* net, const float* f, const float* ustar, int N, int H, int W,
                      float lr, double* loss_host, void* stream) {
    if (!net || !ustar || !(lr > 0.0f)) return CM_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cm::cnn::net_forward_own(net, f, N, H, W, st);
    if (rc) return rc;
    rc = cm::cnn::backward(net, f, ustar, N, H, W, st);
    if (rc) return rc;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)net->step), c2 = 1.0f - powf(b2, (float)net->step);
    cm::cnn::adam_kernel<<<(cm::cnn::NPAR + 255) / 256, 256, 0, st>>>(net->P, net->G, net->M, net->V,
                                                                      cm::cnn::NPAR, lr, b1, b2, eps,
                                                                      c1, c2);
    NET_CUDA(cudaGetLastError());
    rc = cm::cnn::pack(net, st);
    if (rc) return rc;
    if (loss_host) {
        double s = 0.0;
        NET_CUDA(cudaMemcpyAsync(&s, net->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        NET_CUDA(cudaStreamSynchronize(st));
        *loss_host = s / ((double)N * H * W);
        rc = cm::cnn::net_status(net);
        if (rc) return rc;
    }
    return CM_OK;
}

// ---------------------------------------------------------------------------
// Checkpoints: "CMNETCK1", version, parameter count, Adam step (24-byte
// little-endian header), then the FP32 parameters, the Adam moments m and v,
// and a CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320) of everything
// before it.

static uint32_t ckpt_crc32(uint32_t crc, const unsigned char* p, size_t n) {
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t nparams;
    uint64_t step;
};
static_assert(sizeof(CkptHeader) == 24, "checkpoint header layout");
static const char CKPT_MAGIC[8] = {'C', 'M', 'N', 'E', 'T', 'C', 'K', '1'};

int cm_net_save(cm_net* net, const char* path) {
    if (!net || !path) return CM_ERR_INVALID;
    NET_CUDA(cudaSetDevice(net->device));
    const size_t n = cm::cnn::NPAR;
    std::vector<unsigned char> buf(sizeof(CkptHeader) + 3 * n * sizeof(float) + 4);
    CkptHeader h;
    memcpy(h.magic, CKPT_MAGIC, 8);
    h.version = 1;
    h.nparams = (uint32_t)n;
    h.step = (uint64_t)net->step;
    memcpy(buf.data(), &h, sizeof h);
    float* body = (float*)(buf.data() + sizeof h);
    NET_CUDA(cudaDeviceSynchronize());
    NET_CUDA(cudaMemcpy(body, net->P, n * sizeof(float), cudaMemcpyDeviceToHost));
    NET_CUDA(cudaMemcpy(body + n, net->M, n * sizeof(float), cudaMemcpyDeviceToHost));
    NET_CUDA(cudaMemcpy(body + 2 * n, net->V, n * sizeof(float), cudaMemcpyDeviceToHost));
    const uint32_t crc = ckpt_crc32(0u, buf.data(), buf.size() - 4);
    memcpy(buf.data() + buf.size() - 4, &crc, 4);
    FILE* fp = fopen(path, "wb");
    if (!fp) {
        net->err = std::string("cm_net_save: cannot open ") + path;
        return CM_ERR_INVALID;
    }
    const size_t wrote = fwrite(buf.data(), 1, buf.size(), fp);
    const int closed = fclose(fp);
    if (wrote != buf.size() || closed != 0) {
        net->err = std::string("cm_net_save: short write to ") + path;
        return CM_ERR_INVALID;
    }
    return CM_OK;
}

int cm_net_load(cm_net* net, const char* path) {
    if (!net || !path) return CM_ERR_INVALID;
    const size_t n = cm::cnn::NPAR;
    const size_t want = sizeof(CkptHeader) + 3 * n * sizeof(float) + 4;
    FILE* fp = fopen(path, "rb");
    if (!fp) {
        net->err = std::string("cm_net_load: cannot open ") + path;
        return CM_ERR_INVALID;
    }
    std::vector<unsigned char> buf(want + 1);
    const size_t got = fread(buf.data(), 1, buf.size(), fp);
    fclose(fp);
    CkptHeader h;
    if (got != want) {
        net->err = "cm_net_load: not a checkpoint of this network (size)";
        return CM_ERR_INVALID;
    }
    memcpy(&h, buf.data(), sizeof h);
    uint32_t crc = 0;
    memcpy(&crc, buf.data() + want - 4, 4);
    if (memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != 1 || h.nparams != (uint32_t)n) {
        net->err = "cm_net_load: not a checkpoint of this network (header)";
        return CM_ERR_INVALID;
    }
    if (ckpt_crc32(0u, buf.data(), want - 4) != crc) {
        net->err = "cm_net_load: checksum mismatch";
        return CM_ERR_INVALID;
    }
    const float* body = (const float*)(buf.data() + sizeof h);
    NET_CUDA(cudaSetDevice(net->device));
    NET_CUDA(cudaMemcpy(net->P, body, n * sizeof(float), cudaMemcpyHostToDevice));
    NET_CUDA(cudaMemcpy(net->M, body + n, n * sizeof(float), cudaMemcpyHostToDevice));
    NET_CUDA(cudaMemcpy(net->V, body + 2 * n, n * sizeof(float), cudaMemcpyHostToDevice));
    net->step = (int)h.step;
    int rc = cm::cnn::pack(net, 0);
    if (rc) return rc;
    NET_CUDA(cudaDeviceSynchronize());
    return CM_OK;
}

// ---------------------------------------------------------------------------
// Training loop.  Mini-batch of global step t: `batch` distinct pair indices
// from a partial Fisher-Yates shuffle of 0 .. N-1 driven by SplitMix64
// (Steele, Lea and Flood, OOPSLA 2014): the stream's state for step t is its
// (t + 1)-th output from `seed`, and draw j is the (j + 1)-th output from that
// state; r = j + draw mod (N - j) is swapped into place j.

static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void batch_indices(uint64_t seed, long long t, int N, int batch, std::vector<int>& perm,
                          std::vector<int>& idx) {
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    const uint64_t state = sm64_mix(seed + gamma * (uint64_t)(t + 1));
    for (int i = 0; i < N; ++i) perm[i] = i;
    for (int j = 0; j < batch; ++j) {
        const uint64_t x = sm64_mix(state + gamma * (uint64_t)(j + 1));
        const int r = j + (int)(x % (uint64_t)(N - j));
        std::swap(perm[j], perm[r]);
        idx[j] = perm[j];
    }
}

int cm_net_train(cm_ctx* ctx, cm_net* net, const float* f, const float* ustar, int N, int H,
                 int W, const cm_train_opts* o, cm_train_log* log, void* stream) {
    if (!ctx || !net || !f || !ustar || !o || N < 1 || H < 1 || W < 1 || H > CM_MAX_SIDE ||
        W > CM_MAX_SIDE || (long long)H * W > CM_MAX_PIXELS || o->steps < 1 ||
        o->batch < 1 || o->batch > N || !(o->lr > 0.0f) || !(o->lr_final > 0.0f) ||
        o->start_step < 0 || o->log_every < 1 || o->total_steps < 0 ||
        (o->total_steps > 0 && o->start_step + o->steps > o->total_steps))
        return CM_ERR_INVALID;
    if (log && log->losses_cap > 0 && !log->losses) return CM_ERR_INVALID;
    NET_CUDA(cudaSetDevice(net->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t hw = (size_t)H * W;
    float *fb = nullptr, *ub = nullptr;
    cudaError_t e = cudaMalloc(&fb, (size_t)o->batch * hw * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ub, (size_t)o->batch * hw * sizeof(float));
    if (e != cudaSuccess) {
        cudaFree(fb);
        net->err = "cm_net_train: out of device memory for the mini-batch";
        return e == cudaErrorMemoryAllocation ? CM_ERR_OOM : CM_ERR_CUDA;
    }
    const long long T = o->total_steps > 0 ? o->total_steps : (long long)o->start_step + o->steps;
    std::vector<int> perm(N), idx(o->batch);
    int rc = CM_OK;
    if (log) log->n_logged = 0;
    for (int s = 0; s < o->steps && rc == CM_OK; ++s) {
        const long long t = (long long)o->start_step + s;
        batch_indices(o->seed, t, N, o->batch, perm, idx);
        for (int j = 0; j < o->batch && e == cudaSuccess; ++j) {
            e = cudaMemcpyAsync(fb + j * hw, f + (size_t)idx[j] * hw, hw * sizeof(float),
                                cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ub + j * hw, ustar + (size_t)idx[j] * hw, hw * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st);
        }
        if (e != cudaSuccess) {
            rc = CM_ERR_CUDA;
            net->err = std::string("cm_net_train: ") + cudaGetErrorString(e);
            break;
        }
        // cosine decay lr -> lr_final over the schedule's T steps
        const double lr = (double)o->lr_final + 0.5 * ((double)o->lr - (double)o->lr_final) *
                                                    (1.0 + cos(3.14159265358979323846 * (double)t /
                                                               (double)std::max(1LL, T - 1)));
        const bool want = log && ((s % o->log_every) == 0 || s == o->steps - 1 || s == 0);
        double loss = 0.0;
        rc = cm_net_train_step(net, fb, ub, o->batch, H, W, (float)lr, want ? &loss : nullptr,
                               stream);
        if (rc == CM_OK && want) {
            if (s == 0) log->loss_first = loss;
            log->loss_last = loss;
            if (log->n_logged < log->losses_cap) {
                log->losses[log->n_logged] = loss;
                if (log->logged_steps) log->logged_steps[log->n_logged] = (int)t;
                log->n_logged += 1;
            }
        }
    }
    if (rc == CM_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = CM_ERR_CUDA;
            net->err = std::string("cm_net_train: ") + cudaGetErrorString(e);
        } else {
            rc = cm::cnn::net_status(net);
        }
    }
    cudaFree(fb);
    cudaFree(ub);
    return rc;
}

}  // extern "C"

extern "C" int cm_selftest_wait(int device, int limit, int* timed_out, int* completed) {
    if (!timed_out || !completed || device < 0 || limit < 1 || limit > (1 << 22))
        return CM_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return CM_ERR_CUDA;
    int* d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return CM_ERR_OOM;
    int h[2] = {-1, -1};
    cudaError_t e = cudaMemset(d, 0xff, 2 * sizeof(int));
    if (e == cudaSuccess) {
        cm::cnn::wait_selftest_kernel<<<1, 32>>>(limit, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return CM_ERR_CUDA;
    *timed_out = h[0];
    *completed = h[1];
    return CM_OK;
}
