// cm_energy.cu -- discrete energy and curvature map kernels.
//
//  energy_kernel     F(u) = sum |kappa| + alpha/2 (u - f)^2 (Eq. MCM / Eq. GCM;
//                    kappa of any of the four kinds of kappa_signed):
//                    smem halo tile, FP32 per pixel, warp and CTA, a
//                    fixed-order FP64 sum of the CTA partials in the last
//                    CTA (deterministic).
//  curvature_kernel  signed kappa per pixel (diagnostics and tests).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cm_device.cuh"
#include "cm_kernels.h"

namespace cm {

// ---------------------------------------------------------------------------
// Energy.

constexpr int E_TW = 32;   // tile columns
constexpr int E_TH = 32;   // tile rows (each thread 4 rows)

// Reduction: FP32 per pixel, per thread (4 pixels), per warp (a fixed
// shuffle tree) and per CTA (the 8 warp sums in order): a sum of 1024
// non-negative terms with relative error <= 11 eps32 ~ 7e-7; then FP64 for
// the grid: the CTA sums, in a fixed order, by the last CTA.  FP64 stays out
// of the per-CTA code: the GB300's FP64 pipe runs at a small fraction of its
// FP32 rate, and FP64 conversions and shuffles in every warp kept it about
// half busy (one FP64 sum per CTA still took a fifth of it).
template <int KIND>
__global__ void __launch_bounds__(256) energy_kernel(const float* __restrict__ u,
                                                     const float* __restrict__ f, int H, int W,
                                                     float alpha, double* __restrict__ partials,
                                                     unsigned int* __restrict__ ticket,
                                                     double* __restrict__ E_out,
                                                     const int* __restrict__ active) {
    if (active && *active == 0) return;
    __shared__ float tile[E_TH + 2][E_TW + 3];
    __shared__ float wsum[8];
    __shared__ double dsum[8];
    __shared__ bool is_last;
    const int r0 = blockIdx.y * E_TH, c0 = blockIdx.x * E_TW;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // the f values of this thread's pixels, requested before the tile barrier
    float fv[E_TH / 8];
#pragma unroll
    for (int i = 0; i < E_TH / 8; ++i) {
        const int r = r0 + ty + 8 * i, c = c0 + tx;
        fv[i] = (r < H && c < W) ? f[(size_t)r * W + c] : 0.0f;
    }
    // Tiles away from the left and right edges of an image whose rows are
    // 16-byte aligned read the halo columns c0 - 1 .. c0 + 32 as the float4
    // words of the aligned span c0 - 4 .. c0 + 35; rows clamp as below.
    const bool vec = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(u) & 15) == 0 && c0 >= 4 &&
                     c0 + E_TW + 4 <= W;
    if (vec) {
        constexpr int NV = (E_TW + 8) / 4;   // float4 words per tile row
        for (int i = threadIdx.x; i < (E_TH + 2) * NV; i += 256) {
            const int lr = i / NV, v = i - lr * NV;
            const int r = clampi(r0 - 1 + lr, 0, H - 1);
            const float4 q4 = *reinterpret_cast<const float4*>(u + (size_t)r * W + (c0 - 4 + 4 * v));
            const float e[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int lc = 4 * v - 3 + q;   // column c0 - 4 + 4v + q, tile column + 1
                if (lc >= 0 && lc < E_TW + 2) tile[lr][lc] = e[q];
            }
        }
    } else {
        for (int i = threadIdx.x; i < (E_TH + 2) * (E_TW + 2); i += 256) {
            int lr = i / (E_TW + 2), lc = i - lr * (E_TW + 2);
            int r = clampi(r0 - 1 + lr, 0, H - 1), c = clampi(c0 - 1 + lc, 0, W - 1);
            tile[lr][lc] = u[(size_t)r * W + c];
        }
    }
    __syncthreads();
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < E_TH / 8; ++i) {
        int lr = ty + 8 * i;
        int r = r0 + lr, c = c0 + tx;
        if (r < H && c < W) {
            float w[9];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) w[3 * a + b] = tile[lr + a][tx + b];
            float e = w[4] - fv[i];
            acc += abs_curvature<KIND>(w) + 0.5f * alpha * e * e;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (tx == 0) wsum[ty] = acc;
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += wsum[i];
        partials[bid] = (double)s;
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        is_last = (t == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // Fixed-order finish: thread t sums partials t, t+256, ...; then a tree.
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += 256) s += ((volatile double*)partials)[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __syncthreads();
    if (tx == 0) dsum[ty] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += dsum[i];
        *E_out = t;
        *ticket = 0u;   // ready for the next launch
    }
}

template <int KIND>
__global__ void curvature_kernel(const float* __restrict__ u, int H, int W,
                                 float* __restrict__ out) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (r >= H || c >= W) return;
    float w[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            w[3 * a + b] = u[(size_t)clampi(r + a - 1, 0, H - 1) * W + clampi(c + b - 1, 0, W - 1)];
    const KBar4 k = direction_curvatures(w);
    out[(size_t)r * W + c] = kappa_signed<KIND>(k.k[0], k.k[1], k.k[2], k.k[3]);
}

cudaError_t launch_energy(const float* u, const float* f, int H, int W, float alpha, int kind,
                          double* partials, unsigned int* ticket, double* E_out,
                          cudaStream_t st, const int* active) {
    dim3 grid((W + E_TW - 1) / E_TW, (H + E_TH - 1) / E_TH);
    decltype(&energy_kernel<KIND_MEAN>) k;
    switch (kind) {
        case KIND_MEAN: k = energy_kernel<KIND_MEAN>; break;
        case KIND_GAUSS: k = energy_kernel<KIND_GAUSS>; break;
        case KIND_MEAN_EULER: k = energy_kernel<KIND_MEAN_EULER>; break;
        case KIND_GAUSS_EULER: k = energy_kernel<KIND_GAUSS_EULER>; break;
        default: return cudaErrorInvalidValue;
    }
    return launch_k(k, grid, dim3(256), st, 1, u, f, H, W, alpha, partials, ticket, E_out, active);
}

size_t energy_partials_needed(int H, int W) {
    return (size_t)((W + E_TW - 1) / E_TW) * (size_t)((H + E_TH - 1) / E_TH);
}

cudaError_t launch_curvature(const float* u, int H, int W, int kind, float* out,
                             cudaStream_t st) {
    dim3 blk(32, 8), grid((W + 31) / 32, (H + 7) / 8);
    switch (kind) {
        case KIND_MEAN: curvature_kernel<KIND_MEAN><<<grid, blk, 0, st>>>(u, H, W, out); break;
        case KIND_GAUSS: curvature_kernel<KIND_GAUSS><<<grid, blk, 0, st>>>(u, H, W, out); break;
        case KIND_MEAN_EULER:
            curvature_kernel<KIND_MEAN_EULER><<<grid, blk, 0, st>>>(u, H, W, out);
            break;
        case KIND_GAUSS_EULER:
            curvature_kernel<KIND_GAUSS_EULER><<<grid, blk, 0, st>>>(u, H, W, out);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace cm
