// cm_phase_blocks.cu -- levels with block side b >= 2: the coarse path's
// block-sum and apply kernels, and dispatch to the per-kind kernels
// (cm_phase_blocks.cuh, instantiated in cm_blocks_<kind>.cu).
#include <cuda_runtime.h>

#include "cm_device.cuh"
#include "cm_kernels.h"
#include "cm_phase_kinds.h"

namespace cm {


// Coarse levels (b >= 64): few blocks, so every step is made short.
//  * S1 comes from 32 x 32 tile sums of S - f computed by one wide kernel per
//    level (a block of side >= 64 is a union of whole tiles);
//  * the search kernel writes only the block's c; pixels of blocks of earlier
//    colours of the level are read as S + c (the value R would hold);
//  * one wide kernel writes R = S + c after the last colour.
// The result is the same as the direct phases up to the FP32 order of the
// S1 sum.

__global__ void __launch_bounds__(256) tile_sums_kernel(const float* __restrict__ S,
                                                        const float* __restrict__ f, int H, int W,
                                                        float* __restrict__ partials,
                                                        const int* __restrict__ active) {
    if (active && *active == 0) return;
    __shared__ float red[8];
    const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * TILE;
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < TILE * TILE / 256; ++i) {
        const int idx = threadIdx.x + 256 * i;
        const int r = r0 + idx / TILE, c = c0 + idx % TILE;
        if (r < H && c < W) {
            const size_t p = (size_t)r * W + c;
            acc += S[p] - f[p];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += red[i];
        partials[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// R = S + c on every pixel (deferred apply of a coarse level) and, in the same
// pass, the 32 x 32 tile sums of R - f that the next coarse level takes its
// block sums from (the order of tile_sums_kernel, so the sums are the same).
// S and R may be the same buffer (every pixel is read and written by one
// thread).
__global__ void __launch_bounds__(256) apply_kernel(const float* S, float* R,
                                                    const float* __restrict__ f,
                                                    const float* __restrict__ cj, int H, int W,
                                                    int lb, int nbj, float* __restrict__ partials,
                                                    const int* __restrict__ active) {
    if (active && *active == 0) return;
    __shared__ float red[8];
    const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * TILE;
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < TILE * TILE / 256; ++i) {
        const int idx = threadIdx.x + 256 * i;
        const int r = r0 + idx / TILE, c = c0 + idx % TILE;
        if (r < H && c < W) {
            const size_t p = (size_t)r * W + c;
            const float v = S[p] + cj[(size_t)(r >> lb) * nbj + (c >> lb)];
            R[p] = v;
            acc += v - f[p];
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += red[i];
        partials[blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

// Non-portable cluster sizes of every kind's coarse kernels.
cudaError_t coarse_setup() {
    cudaError_t e = coarse_setup_kind<KIND_MEAN>();
    if (e == cudaSuccess) e = coarse_setup_kind<KIND_GAUSS>();
    if (e == cudaSuccess) e = coarse_setup_kind<KIND_MEAN_EULER>();
    if (e == cudaSuccess) e = coarse_setup_kind<KIND_GAUSS_EULER>();
    return e;
}

static cudaError_t coarse_phase(const PhaseArgs& A, const float* partials, float* cj,
                                cudaStream_t st) {
    switch (A.kind) {
        case KIND_MEAN: return coarse_phase_kind<KIND_MEAN>(A, partials, cj, st);
        case KIND_GAUSS: return coarse_phase_kind<KIND_GAUSS>(A, partials, cj, st);
        case KIND_MEAN_EULER: return coarse_phase_kind<KIND_MEAN_EULER>(A, partials, cj, st);
        case KIND_GAUSS_EULER: return coarse_phase_kind<KIND_GAUSS_EULER>(A, partials, cj, st);
        default: return cudaErrorInvalidValue;
    }
}

size_t coarse_partials_needed(int H, int W) {
    return (size_t)((H + TILE - 1) / TILE) * (size_t)((W + TILE - 1) / TILE);
}

size_t coarse_c_needed(int H, int W) {
    const int b = 1 << COARSE_LB;
    return (size_t)((H + b - 1) / b) * (size_t)((W + b - 1) / b);
}

int coarse_level_log2() { return COARSE_LB; }

// One whole level on the coarse path: tile sums, every colour's search, apply.
cudaError_t launch_level_coarse(const PhaseArgs& A0, float* partials, float* cj,
                                cudaStream_t st, bool sums_ready) {
    dim3 tg((A0.W + TILE - 1) / TILE, (A0.H + TILE - 1) / TILE);
    cudaError_t e = cudaSuccess;
    if (!sums_ready)
        e = launch_k(tile_sums_kernel, tg, dim3(256), st, 1, A0.S, A0.f, A0.H, A0.W, partials,
                     A0.active);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < A0.ncolors; ++k) {
        PhaseArgs A = A0;
        A.colour = k;
        e = coarse_phase(A, partials, cj, st);
        if (e != cudaSuccess) return e;
    }
    const int b = 1 << A0.lb;
    const int nbj = (A0.W + b - 1) / b;
    return launch_k(apply_kernel, tg, dim3(256), st, 1, (const float*)A0.S, A0.R, A0.f,
                    (const float*)cj, A0.H, A0.W, A0.lb, nbj, partials, A0.active);
}

static cudaError_t launch_phase_odd(const PhaseArgs& A, cudaStream_t st) {
    switch (A.kind) {
        case KIND_MEAN: return blocks_phase_odd_kind<KIND_MEAN>(A, st);
        case KIND_GAUSS: return blocks_phase_odd_kind<KIND_GAUSS>(A, st);
        case KIND_MEAN_EULER: return blocks_phase_odd_kind<KIND_MEAN_EULER>(A, st);
        case KIND_GAUSS_EULER: return blocks_phase_odd_kind<KIND_GAUSS_EULER>(A, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_phase_blocks(const PhaseArgs& A, cudaStream_t st) {
    if (A.bs != (1 << A.lb)) return launch_phase_odd(A, st);
    switch (A.kind) {
        case KIND_MEAN: return blocks_phase_kind<KIND_MEAN>(A, st);
        case KIND_GAUSS: return blocks_phase_kind<KIND_GAUSS>(A, st);
        case KIND_MEAN_EULER: return blocks_phase_kind<KIND_MEAN_EULER>(A, st);
        case KIND_GAUSS_EULER: return blocks_phase_kind<KIND_GAUSS_EULER>(A, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_phase(const PhaseArgs& A, cudaStream_t st) {
    if (A.bs == 1) return launch_phase_b1(A, st);
    return launch_phase_blocks(A, st);
}

int max_level_log2() { return 11; }

}  // namespace cm
