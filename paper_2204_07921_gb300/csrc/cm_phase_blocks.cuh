// cm_phase_blocks.cuh -- kernels of the sweep levels with block side b >= 2
// (Sec. 2.2), templates on the curvature kind.
//
//  phase_warp_kernel     b = 2, 4 and 8: 8, 16 or 32 lanes of one warp per
//                        block, two ring pixels per lane; candidate energies
//                        are warp-shuffle reductions.
//  phase_cluster_kernel  b >= 16: one CTA, or a thread-block cluster of up to 8
//                        CTAs on different SMs, per block, one ring pixel per
//                        thread; candidate energies reduce through shared
//                        memory and, across the cluster, distributed shared
//                        memory with one cluster barrier per reduction.
//
// Each thread holds its ring pixel as the affine coefficients of its four
// direction curvatures in the block shift c (AffPix), so a candidate costs
// ~55 FP32 operations and 8 rsqrt per ring pixel.
//
// Included only by the per-kind translation units cm_blocks_<kind>.cu, which
// instantiate the entry points of cm_phase_kinds.h for one kind each.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "cm_device.cuh"
#include "cm_kernels.h"
#include "cm_phase_kinds.h"
#include "cm_search.cuh"

// Lanes per block on the warp-group levels (b = 2: ring 16, b = 4: ring 32,
// b = 8: ring 64 on 32 lanes); each lane holds ring / lanes ring pixels.
#ifndef CM_B2_GT
#define CM_B2_GT 8
#endif
#ifndef CM_B4_GT
#define CM_B4_GT 16
#endif
// b = 2: rotation-specialised kernel (1) or the generic warp groups (0), and
// its minimum CTAs per SM (register cap).
#ifndef CM_B2_FAST
#define CM_B2_FAST 1
#endif
#ifndef CM_B2_MINB
#define CM_B2_MINB 4
#endif


namespace cm {


// Block pixels [r0, r0 + bh) x [c0, c0 + bw), visited with stride `stride`
// from index `first` (row-major within the block).
template <class F>
__device__ __forceinline__ void for_block_pixels(int first, int stride, int r0, int c0, int bh,
                                                 int bw, int lb, bool full_w, int W, F&& fn) {
    const int npx = bh * bw;
#pragma unroll 4
    for (int idx = first; idx < npx; idx += stride) {
        int rr = full_w ? (idx >> lb) : idx / bw;
        fn((size_t)(r0 + rr) * W + (c0 + idx - rr * bw));
    }
}

// One block per group of GT lanes of a warp (every lane of the warp runs
// this with its group's active-block number a, valid or not).  LIGHT keeps
// the ring windows and rebuilds the affine coefficients per candidate (fewer
// registers, more arithmetic).
// rk: reads take R for blocks of colours below rk (the colour k, or 0 when
// the level runs in place and S is the state being updated).  S and R are
// then one buffer, so neither is declared __restrict__ in the kernels that
// write R (a block reads each of its own pixels before writing it, and no
// other block of the phase reads them).
template <int KIND, int GT, int RPT, bool LIGHT = false, bool POW2 = true>
__device__ __forceinline__ void warp_group_block(const float* S, float* R,
                                                 const float* __restrict__ f, int H, int W,
                                                 const SearchParams& sp, int lb, int ncol, int k,
                                                 int rk, float* __restrict__ c_out, int a,
                                                 int bs = 0) {
    static_assert(GT == 4 || GT == 8 || GT == 16 || GT == 32, "warp groups only");
    const int lane = threadIdx.x % GT;
    // block side 1 << lb, or (POW2 false) bs < 1 << lb
    const int b = POW2 ? 1 << lb : bs;
    const int nbi = block_of<POW2>(H + b - 1, lb, b), nbj = block_of<POW2>(W + b - 1, lb, b);
    int bi, bj;
    const bool blk_on = active_block(a, nbi, nbj, ncol, k, bi, bj);
    // Groups without a block still take part in the shuffles of their warp.
    const int r0 = blk_on ? bi * b : 0, c0 = blk_on ? bj * b : 0;
    const int r1 = blk_on ? min(r0 + b, H) : 0, c1 = blk_on ? min(c0 + b, W) : 0;
    const int bh = r1 - r0, bw = c1 - c0;
    float s1 = 0.0f;
    if (blk_on)
        for_block_pixels(lane, GT, r0, c0, bh, bw, lb, POW2 && bw == b, W,
                         [&](size_t p) { s1 += S[p] - f[p]; });
#pragma unroll
    for (int off = GT / 2; off > 0; off >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, off, GT);
    constexpr int NPX = LIGHT ? 1 : RPT;
    constexpr int NWIN = LIGHT ? RPT : 1;
    AffPix px[NPX];
    float win[NWIN][9];
    unsigned msk[RPT];
    bool has[RPT];
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        float w[9];
        msk[t] = 0;
        has[t] = blk_on && ring_slot<POW2>(lane + t * GT, r0, r1, c0, c1, H, W, S, R, lb, ncol,
                                           rk, w, msk[t], b);
        if constexpr (LIGHT) {
#pragma unroll
            for (int i = 0; i < 9; ++i) win[t][i] = has[t] ? w[i] : 0.0f;
        } else if (has[t]) {
            px[t] = aff_pix(w, msk[t]);
        } else {
#pragma unroll
            for (int d = 0; d < 4; ++d) px[t].d[d] = AffDir{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        }
    }
    auto ring = [&](float c) {
        float v = 0.0f;
#pragma unroll
        for (int t = 0; t < RPT; ++t) {
            if constexpr (LIGHT) {
                if (has[t]) v += aff_abs_curv<KIND>(aff_pix(win[t], msk[t]), c);
            } else {
                v += has[t] ? aff_abs_curv<KIND>(px[t], c) : 0.0f;
            }
        }
#pragma unroll
        for (int off = GT / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, GT);
        return v;
    };
    const float s = blk_on ? (float)(bh * bw) : 1.0f;
    const float S1b = blk_on ? s1 : 0.0f;
    float cbest;
    if (sp.one_step)
        cbest = block_search_onestep(ring, sp, s, S1b, fbs_step(sp, s, S1b));
    else if constexpr (LIGHT)
        cbest = block_search_1site(ring, sp, s, S1b, false, 0.0f);
    else
        cbest = block_search(ring, sp, s, S1b, false, 0.0f);
    if (!blk_on) return;
    for_block_pixels(lane, GT, r0, c0, bh, bw, lb, POW2 && bw == b, W,
                     [&](size_t p) { R[p] = S[p] + cbest; });
    if (c_out && lane == 0) c_out[(size_t)bi * nbj + bj] = cbest;
}

template <int KIND, int GT, int RPT, bool POW2 = true>
__global__ void __launch_bounds__(128) phase_warp_kernel(
    const float* S, float* R, const float* __restrict__ f, int H, int W,
    SearchParams sp, int lb, int bs, int ncol, int k, int rk, float* __restrict__ c_out,
    const int* __restrict__ active) {
    if (active && *active == 0) return;
    constexpr int GPC = 128 / GT;
    warp_group_block<KIND, GT, RPT, false, POW2>(S, R, f, H, W, sp, lb, ncol, k, rk, c_out,
                                                 blockIdx.x * GPC + threadIdx.x / GT, bs);
}

// ---------------------------------------------------------------------------
// b = 2, interior blocks: four lanes per block, lane q taking the quarter of
// the ring that a rotation by q x 90 degrees about the block centre maps from
// quarter 0 = {outer corner (-1, -1), outer sides (-1, 0) and (-1, 1), block
// pixel (0, 0)} (offsets from the block's top-left pixel).  Each lane reads
// its windows rotated back into the frame of quarter 0, so every lane runs
// the same code with the window entries that lie in the block known at
// compile time.  The eight-plane curvature is invariant under the rotation
// (the four line directions are permuted, a line's end points may swap, which
// negates Dq exactly and leaves every other term as it is), so each direction
// value is the one the generic evaluation computes.  Terms that do not depend
// on c are computed once per block instead of once per candidate: 22 instead
// of 32 rsqrt per lane and candidate.

// Direction T of a ring pixel whose window entries in the block are MASK.
template <unsigned MASK, int T>
struct SpecDir {
    static constexpr int X = line_x(T), Y = line_y(T), Z1 = line_z1(T), Z2 = line_z2(T);
    static constexpr int mx = (MASK >> X) & 1, my = (MASK >> Y) & 1, mo = (MASK >> 4) & 1;
    static constexpr int mz1 = (MASK >> Z1) & 1, mz2 = (MASK >> Z2) & 1;
    static constexpr float DQ1 = 0.5f * (float)(my - mx);
    static constexpr float DL1 = line_two_h(T) * (0.5f * (float)(mx + my) - (float)mo);
    static constexpr float E11 = (float)(mx + my - 2 * mz1);
    static constexpr float E21 = (float)(mx + my - 2 * mz2);
    static constexpr bool LINE = DQ1 != 0.0f;   // Dq (so ds) varies with c
    static constexpr bool CONST = !LINE && DL1 == 0.0f && E11 == 0.0f && E21 == 0.0f;
    // LINE: dq0, dl0, e10, e20.  Otherwise: fds = 4 ds^2, ds4, dl0, and per
    // plane its constant rsqrt term or e_i0.  CONST: kb.
    float a0, a1, a2, a3, a4;

    __device__ __forceinline__ void init(const float w[9]) {
        const float two_h = line_two_h(T);
        const float dq0 = 0.5f * (w[Y] - w[X]);
        const float dl0 = two_h * fmaf(0.5f, w[X] + w[Y], -w[4]);
        const float Sxy = w[X] + w[Y];
        const float e10 = fmaf(-2.0f, w[Z1], Sxy);
        const float e20 = fmaf(-2.0f, w[Z2], Sxy);
        if constexpr (LINE) {
            a0 = dq0;
            a1 = dl0;
            a2 = e10;
            a3 = e20;
        } else {
            const float ds2 = fmaf(dq0, dq0, line_h2(T));
            const float fds = 4.0f * ds2;
            const float ds4 = ds2 * ds2;
            const float t1 = E11 == 0.0f ? rsqrtf(fmaf(e10, e10, fds) * ds4) : e10;
            const float t2 = E21 == 0.0f ? rsqrtf(fmaf(e20, e20, fds) * ds4) : e20;
            if constexpr (CONST) {
                a0 = dl0 * (t1 + t2);
            } else {
                a0 = fds;
                a1 = ds4;
                a2 = dl0;
                a3 = t1;
                a4 = t2;
            }
        }
    }

    __device__ __forceinline__ float eval(float c) const {
        if constexpr (CONST) {
            return a0;
        } else if constexpr (LINE) {
            const float Dq = fmaf(DQ1, c, a0);
            const float ds2 = fmaf(Dq, Dq, line_h2(T));
            const float fds = 4.0f * ds2;
            const float ds4 = ds2 * ds2;
            const float e1 = E11 == 0.0f ? a2 : fmaf(E11, c, a2);
            const float e2 = E21 == 0.0f ? a3 : fmaf(E21, c, a3);
            const float r = rsqrtf(fmaf(e1, e1, fds) * ds4) + rsqrtf(fmaf(e2, e2, fds) * ds4);
            return (DL1 == 0.0f ? a1 : fmaf(DL1, c, a1)) * r;
        } else {
            float r1, r2;
            if constexpr (E11 == 0.0f) {
                r1 = a3;
            } else {
                const float e = fmaf(E11, c, a3);
                r1 = rsqrtf(fmaf(e, e, a0) * a1);
            }
            if constexpr (E21 == 0.0f) {
                r2 = a4;
            } else {
                const float e = fmaf(E21, c, a4);
                r2 = rsqrtf(fmaf(e, e, a0) * a1);
            }
            return (DL1 == 0.0f ? a2 : fmaf(DL1, c, a2)) * (r1 + r2);
        }
    }
};

template <unsigned MASK>
struct SpecPix {
    SpecDir<MASK, 0> d0;
    SpecDir<MASK, 1> d1;
    SpecDir<MASK, 2> d2;
    SpecDir<MASK, 3> d3;
    __device__ __forceinline__ void init(const float w[9]) {
        d0.init(w);
        d1.init(w);
        d2.init(w);
        d3.init(w);
    }
    template <int KIND>
    __device__ __forceinline__ float abs_curv(float c) const {
        const float k0 = d0.eval(c), k1 = d1.eval(c), k2 = d2.eval(c), k3 = d3.eval(c);
        return kappa_abs<KIND>(k0, k1, k2, k3);
    }
};

// Window entries (row-major 3 x 3, index 3a + b) in the block, quarter 0.
constexpr unsigned B2_M0 = 1u << 8;                                // corner (-1, -1)
constexpr unsigned B2_M1 = (1u << 7) | (1u << 8);                  // side (-1, 0)
constexpr unsigned B2_M2 = (1u << 6) | (1u << 7);                  // side (-1, 1)
constexpr unsigned B2_M3 = (1u << 4) | (1u << 5) | (1u << 7) | (1u << 8);   // pixel (0, 0)

template <int KIND>
__global__ void __launch_bounds__(128, CM_B2_MINB) phase_b2_kernel(
    const float* S, float* R, const float* __restrict__ f, int H, int W,
    SearchParams sp, int ncol, int k, int rk, float* __restrict__ c_out,
    const int* __restrict__ active) {
    if (active && *active == 0) return;
    const int a = blockIdx.x * 32 + threadIdx.x / 4;
    const int q = threadIdx.x & 3;
    const int nbi = (H + 1) >> 1, nbj = (W + 1) >> 1;
    int bi, bj;
    const bool blk_on = active_block(a, nbi, nbj, ncol, k, bi, bj);
    const int r0 = bi << 1, c0 = bj << 1;
    const bool interior = r0 >= 2 && c0 >= 2 && r0 + 3 < H && c0 + 3 < W;
    if (!__all_sync(0xffffffffu, !blk_on || interior)) {
        // a warp with a border block runs the generic four-lane search
        warp_group_block<KIND, 4, 4, true>(S, R, f, H, W, sp, 1, ncol, k, rk, c_out, a);
        return;
    }
    // Frame of quarter 0 -> image: offset (dr, dc) from (r0, c0) rotated q
    // quarter turns about the block centre.
    auto img = [&](int dr, int dc, int& r, int& c) {
        int rr = dr, cc = dc;
        if (q == 1) { rr = dc; cc = 1 - dr; }
        else if (q == 2) { rr = 1 - dr; cc = 1 - dc; }
        else if (q == 3) { rr = 1 - dc; cc = dr; }
        r = r0 + rr;
        c = c0 + cc;
    };
    // v[dr + 2][dc + 2]: rows -2 .. 1, columns -2 .. 2 of the frame (row 1
    // only columns -1 .. 1)
    float v[4][5];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            v[i][j] = 0.0f;
            if (blk_on && (i < 3 || (j >= 1 && j <= 3))) {
                int r, c;
                img(i - 2, j - 2, r, c);
                v[i][j] = phase_read(S, R, r, c, W, 1, ncol, rk);
            }
        }
    int pr, pc;
    img(0, 0, pr, pc);
    const size_t p = (size_t)pr * W + pc;
    float s1 = blk_on ? v[2][2] - f[p] : 0.0f;
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    SpecPix<B2_M0> P0;
    SpecPix<B2_M1> P1;
    SpecPix<B2_M2> P2;
    SpecPix<B2_M3> P3;
    {
        float w[9];
        auto win = [&](int i0, int j0) {
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) w[3 * x + y] = v[i0 + x][j0 + y];
        };
        win(0, 0);
        P0.init(w);
        win(0, 1);
        P1.init(w);
        win(0, 2);
        P2.init(w);
        win(1, 1);
        P3.init(w);
    }
    auto ring = [&](float c) {
        float t = P0.template abs_curv<KIND>(c) + P1.template abs_curv<KIND>(c) +
                  P2.template abs_curv<KIND>(c) + P3.template abs_curv<KIND>(c);
        t = blk_on ? t : 0.0f;
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        return t;
    };
    const float sb = blk_on ? 4.0f : 1.0f;
    const float cbest = sp.one_step
                            ? block_search_onestep(ring, sp, sb, s1, fbs_step(sp, sb, s1))
                            : block_search_1site(ring, sp, sb, s1, false, 0.0f);
    if (!blk_on) return;
    R[p] = v[2][2] + cbest;
    if (c_out && q == 0) c_out[(size_t)bi * nbj + bj] = cbest;
}

template <int KIND, int CT, int Q, int RPT, bool POW2 = true>
__global__ void __cluster_dims__(Q, 1, 1) __launch_bounds__(CT) phase_cluster_kernel(
    const float* S, float* R, const float* __restrict__ f, int H, int W,
    SearchParams sp, int lb, int bs, int ncol, int k, int rk, float* __restrict__ c_out,
    const int* __restrict__ active) {
    namespace cg = cooperative_groups;
    if (active && *active == 0) return;   // uniform over the grid
    constexpr int GT = CT * Q;         // threads searching one block
    constexpr int NW = CT / 32;
    constexpr int MB = 9;              // candidates per batched reduction (the grid)
    __shared__ float red[2][MB][NW];   // per-warp partials, double-buffered
    __shared__ float part[2][Q][MB];   // CTA partials pushed by every cluster rank
    const int rank = Q > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int a = blockIdx.x / Q;
    const int g = rank * CT + threadIdx.x;
    // block side 1 << lb, or (POW2 false) bs < 1 << lb
    const int b = POW2 ? 1 << lb : bs;
    const int nbi = block_of<POW2>(H + b - 1, lb, b), nbj = block_of<POW2>(W + b - 1, lb, b);
    int bi, bj;
    if (!active_block(a, nbi, nbj, ncol, k, bi, bj)) return;   // uniform over the cluster
    const int r0 = bi * b, c0 = bj * b;
    const int r1 = min(r0 + b, H), c1 = min(c0 + b, W);
    const int bh = r1 - r0, bw = c1 - c0;
    int flip = 0;

    // Sum m values over the group: warp shuffles, shared memory, then (Q > 1)
    // every CTA pushes its partials into each rank's shared memory and one
    // cluster barrier publishes them; every thread adds them in rank order.
    auto reduce_vec = [&](float* v, int m) {
#pragma unroll
        for (int j = 0; j < MB; ++j)
            if (j < m) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
            }
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int j = 0; j < MB; ++j)
                if (j < m) red[flip][j][threadIdx.x >> 5] = v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < MB; ++j)
            if (j < m) {
                float t = 0.0f;
#pragma unroll
                for (int i = 0; i < NW; ++i) t += red[flip][j][i];
                v[j] = t;
            }
        if (Q > 1) {
            cg::cluster_group cl = cg::this_cluster();
            if (threadIdx.x < Q) {
                float* dst = cl.map_shared_rank(&part[flip][rank][0], threadIdx.x);
#pragma unroll
                for (int j = 0; j < MB; ++j)
                    if (j < m) dst[j] = v[j];
            }
            cl.sync();
#pragma unroll
            for (int j = 0; j < MB; ++j)
                if (j < m) {
                    float t = 0.0f;
#pragma unroll
                    for (int q = 0; q < Q; ++q) t += part[flip][q][j];
                    v[j] = t;
                }
        }
        flip ^= 1;
    };

    float s1 = 0.0f;
    for_block_pixels(g, GT, r0, c0, bh, bw, lb, POW2 && bw == b, W,
                     [&](size_t p) { s1 += S[p] - f[p]; });
    reduce_vec(&s1, 1);
    const float S1 = s1;

    AffPix px[RPT];
    bool has[RPT];
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        float w[9];
        unsigned mask = 0;
        has[t] = ring_slot<POW2>(g + t * GT, r0, r1, c0, c1, H, W, S, R, lb, ncol, rk, w, mask, b);
        if (has[t]) {
            px[t] = aff_pix(w, mask);
        } else {
#pragma unroll
            for (int d = 0; d < 4; ++d) px[t].d[d] = AffDir{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        }
    }
    auto ringv = [&](const float* cs, int m, float* out) {
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            float acc = 0.0f;
            if (j < m) {
#pragma unroll
                for (int t = 0; t < RPT; ++t)
                    if (has[t]) acc += aff_abs_curv<KIND>(px[t], cs[j]);
            }
            out[j] = acc;
        }
        reduce_vec(out, m);
    };
    const float cbest = block_search_batched<MB>(ringv, sp, (float)(bh * bw), S1);
    for_block_pixels(g, GT, r0, c0, bh, bw, lb, POW2 && bw == b, W,
                     [&](size_t p) { R[p] = S[p] + cbest; });
    if (c_out && g == 0) c_out[(size_t)bi * nbj + bj] = cbest;
    // No CTA may exit while another still reads its shared memory.
    if (Q > 1) cg::this_cluster().sync();
}

// ---------------------------------------------------------------------------
// Coarse levels (b >= 64): few blocks, so every step is made short.
//  * S1 comes from 32 x 32 tile sums of S - f computed by one wide kernel per
//    level (a block of side >= 64 is a union of whole tiles);
//  * the search kernel writes only the block's c; pixels of blocks of earlier
//    colours of the level are read as S + c (the value R would hold);
//  * one wide kernel writes R = S + c after the last colour.
// The result is the same as the direct phases up to the FP32 order of the
// S1 sum.

// Warp-transposed sum of 16 values: four exchange steps halve the values a
// lane holds, so 16 shuffles (not 5 x 16) leave in lanes 2q and 2q + 1 the
// warp sum of value red16_index(2q).  The order of the additions is fixed.
__device__ __forceinline__ int red16_index(int lane) {
    return (((lane >> 4) & 1) << 3) | (((lane >> 3) & 1) << 2) | (((lane >> 2) & 1) << 1) |
           ((lane >> 1) & 1);
}

template <int H>
__device__ __forceinline__ void red16_step(float (&v)[16], int lane) {
    const bool up = (lane & (2 * H)) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float send = up ? v[i] : v[i + H];
        const float keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * H);
    }
}

__device__ __forceinline__ float warp_red16(float (&v)[16], int lane) {
    red16_step<8>(v, lane);
    red16_step<4>(v, lane);
    red16_step<2>(v, lane);
    red16_step<1>(v, lane);
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// One block per CTA (Q = 1) or per cluster of Q CTAs; RPT ring pixels per
// thread.  Launched with the cluster size as a launch attribute.
template <int KIND, int CT, int Q, int RPT>
__global__ void __launch_bounds__(CT) phase_coarse_kernel(
    const float* __restrict__ S, const float* __restrict__ partials, float* __restrict__ cj,
    int H, int W, SearchParams sp, int lb, int ncol, int k, float* __restrict__ c_out,
    const int* __restrict__ active) {
    namespace cg = cooperative_groups;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NW = CT / 32;
    static_assert(NW >= 2 && (NW & (NW - 1)) == 0 && Q >= 1 && Q <= 32 && (Q & (Q - 1)) == 0,
                  "power-of-two warps and cluster ranks");
    if (active && *active == 0) return;   // uniform over the grid
    __shared__ float red[2][16][NW + 1];   // warp partials per candidate, double-buffered
    __shared__ float part[2][Q][16];       // CTA totals pushed by every cluster rank
    __shared__ float red1[NW];
    const int rank = Q > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int a = blockIdx.x / Q;
    const int g = rank * CT + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = 1 << lb;
    const int nbi = (H + b - 1) >> lb, nbj = (W + b - 1) >> lb;
    int bi, bj;
    if (!active_block(a, nbi, nbj, ncol, k, bi, bj)) return;   // uniform over the cluster
    const int r0 = bi << lb, c0 = bj << lb;
    const int r1 = min(r0 + b, H), c1 = min(c0 + b, W);
    const int bh = r1 - r0, bw = c1 - c0;

    // ring windows from the lazy phase state (loads issued before the S1 sum)
    auto value = [&](int r, int c) {
        float v = S[(size_t)r * W + c];
        if (k > 0 && pixel_colour(r, c, lb, ncol) < k) v += cj[(size_t)(r >> lb) * nbj + (c >> lb)];
        return v;
    };
    float win[RPT][9];
    unsigned mask[RPT];
    bool has[RPT];
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        mask[t] = 0;
        has[t] = ring_slot_v(g + t * CT * Q, r0, r1, c0, c1, H, W, value, win[t], mask[t]);
    }
    // S1 from the tile sums of the block, summed by every CTA in the same
    // order (no cluster barrier)
    const int ntc = (W + TILE - 1) / TILE;
    const int tw = (bw + TILE - 1) / TILE, th = (bh + TILE - 1) / TILE;
    float s1 = 0.0f;
    for (int t = threadIdx.x; t < tw * th; t += CT) {
        const int ti = t / tw, tj = t - ti * tw;
        s1 += partials[(size_t)(r0 / TILE + ti) * ntc + (c0 / TILE + tj)];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s1 += __shfl_xor_sync(FULL, s1, off);
    if (lane == 0) red1[warp] = s1;
    __syncthreads();
    float S1 = lane < NW ? red1[lane] : 0.0f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) S1 += __shfl_xor_sync(FULL, S1, off);

    AffPix px[RPT];
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        if (has[t]) {
            px[t] = aff_pix(win[t], mask[t]);
        } else {
#pragma unroll
            for (int d = 0; d < 4; ++d) px[t].d[d] = AffDir{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        }
    }

    // One round: every thread evaluates its ring pixels at the 16 candidates,
    // warps reduce (transposed), CTAs fold the warps and, in a cluster, push
    // their totals to every rank; each warp then folds the ranks (or, Q = 1,
    // the warps) itself: lane l ends with the total of candidate l / 2.
    int flip = 0;
    auto round = [&](float mine, int m) -> float {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float c = __shfl_sync(FULL, mine, j);
            float acc = 0.0f;
            if (j < m) {
#pragma unroll
                for (int t = 0; t < RPT; ++t)
                    if (has[t]) acc += aff_abs_curv<KIND>(px[t], c);
            }
            v[j] = acc;
        }
        const float ws = warp_red16(v, lane);
        if ((lane & 1) == 0) red[flip][red16_index(lane)][warp] = ws;
        __syncthreads();
        const int jc = lane >> 1, half = lane & 1;
        float tot = 0.0f;
        if (Q == 1) {
#pragma unroll
            for (int i = 0; i < NW / 2; ++i) tot += red[flip][jc][half * (NW / 2) + i];
        } else {
            cg::cluster_group cl = cg::this_cluster();
            if (threadIdx.x < 16 * NW) {
                const int j = threadIdx.x / NW, i = threadIdx.x % NW;
                float t = red[flip][j][i];
#pragma unroll
                for (int off = NW / 2; off > 0; off >>= 1) t += __shfl_xor_sync(FULL, t, off);
                for (int q = i; q < Q; q += NW) {
                    float* dst = cl.map_shared_rank(&part[flip][0][0], q);
                    dst[rank * 16 + j] = t;
                }
            }
            cl.sync();
            if (Q == 2) {
                tot = part[flip][half][jc];
            } else {
#pragma unroll
                for (int q = 0; q < Q / 2; ++q) tot += part[flip][half * (Q / 2) + q][jc];
            }
        }
        tot += __shfl_xor_sync(FULL, tot, 1);
        flip ^= 1;
        return tot;
    };
    const float cbest = block_search_rounds(round, sp, (float)(bh * bw), S1);
    // Blocks of this colour read cj only for blocks of earlier colours, so
    // writing this block's entry races with no reader.  The last DSMEM store
    // precedes the last cluster barrier, so CTAs may exit without another.
    if (g == 0) {
        cj[(size_t)bi * nbj + bj] = cbest;
        if (c_out) c_out[(size_t)bi * nbj + bj] = cbest;
    }
}

template <int KIND, int CT, int Q, int RPT>
static cudaError_t launch_coarse(const PhaseArgs& A, const float* partials, float* cj, int nact,
                                 int spec, int dmax, cudaStream_t st) {
    SearchParams sp{A.alpha, A.G, A.K, spec, dmax, A.one_step};
    return launch_k(phase_coarse_kernel<KIND, CT, Q, RPT>, dim3(nact * Q), dim3(CT), st, Q, A.S,
                    partials, cj, A.H, A.W, sp, A.lb, A.ncolors, A.colour, A.c_out, A.active);
}

// Level -> kernel shape (threads, cluster CTAs, ring pixels per thread; the
// ring of a full block, 8b pixels, is CT * Q * RPT) and search rounds
// (speculative first pair, golden steps per round).
#ifndef CM_L6_CT
#define CM_L6_CT 256
#endif
#ifndef CM_L6_Q
#define CM_L6_Q 2
#endif
#ifndef CM_L6_SPEC
#define CM_L6_SPEC 1
#endif
#ifndef CM_L6_DMAX
#define CM_L6_DMAX 4
#endif
#ifndef CM_L79_SPEC
#define CM_L79_SPEC 0
#endif
#ifndef CM_L79_DMAX
#define CM_L79_DMAX 4
#endif
#define CM_COARSE_SHAPES(X)              \
    X(6, CM_L6_CT, CM_L6_Q, 1, CM_L6_SPEC, CM_L6_DMAX) \
    X(7, 256, 4, 1, CM_L79_SPEC, CM_L79_DMAX)          \
    X(8, 256, 8, 1, CM_L79_SPEC, CM_L79_DMAX)          \
    X(9, 512, 8, 1, CM_L79_SPEC, CM_L79_DMAX)          \
    X(10, 512, 8, 2, 1, 4)               \
    X(11, 512, 16, 2, 1, 4)

template <int KIND>
static cudaError_t launch_coarse_kind(const PhaseArgs& A, const float* partials, float* cj,
                                      cudaStream_t st) {
    const int b = 1 << A.lb;
    const int nbi = (A.H + b - 1) / b, nbj = (A.W + b - 1) / b;
    const int nact = active_slots(nbi, nbj, A.ncolors);
    switch (A.lb) {
#define CM_CASE(LB, CT, Q, RPT, SPEC, DMAX)                                                  \
    case LB:                                                                                  \
        return launch_coarse<KIND, CT, Q, RPT>(A, partials, cj, nact,                         \
                                               A.coarse_spec >= 0 ? A.coarse_spec : (SPEC),   \
                                               A.coarse_dmax > 0 ? A.coarse_dmax : (DMAX), st);
        CM_COARSE_SHAPES(CM_CASE)
#undef CM_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Colour bound of the kernels' R reads: the phase's colour, or the
// caller's read_colour (0 for a level run in place).
static inline int read_colour(const PhaseArgs& A) {
    return A.read_colour < 0 ? A.colour : A.read_colour;
}

template <int KIND, int GT, int RPT, bool POW2 = true>
static cudaError_t launch_warp(const PhaseArgs& A, int nact, cudaStream_t st) {
    constexpr int GPC = 128 / GT;
    SearchParams sp{A.alpha, A.G, A.K};
    sp.one_step = A.one_step;
    return launch_k(phase_warp_kernel<KIND, GT, RPT, POW2>, dim3((nact + GPC - 1) / GPC),
                    dim3(128), st, 1, A.S, A.R, A.f, A.H, A.W, sp, A.lb, A.bs, A.ncolors,
                    A.colour, read_colour(A), A.c_out, A.active);
}

template <int KIND, int CT, int Q, int RPT, bool POW2 = true>
static cudaError_t launch_cluster(const PhaseArgs& A, int nact, cudaStream_t st) {
    SearchParams sp{A.alpha, A.G, A.K};
    sp.one_step = A.one_step;
    return launch_k(phase_cluster_kernel<KIND, CT, Q, RPT, POW2>, dim3(nact * Q), dim3(CT), st, 1,
                    A.S, A.R, A.f, A.H, A.W, sp, A.lb, A.bs, A.ncolors, A.colour,
                    read_colour(A), A.c_out, A.active);
}

template <int KIND>
static cudaError_t launch_blocks_kind(const PhaseArgs& A, cudaStream_t st) {
    const int b = 1 << A.lb;
    const int nbi = (A.H + b - 1) / b, nbj = (A.W + b - 1) / b;
    const int nact = active_slots(nbi, nbj, A.ncolors);
    // ring of a full block: 8b pixels = Q * CT * RPT slots.  Bit lb - 1 of
    // A.shapes (levels b = 2 .. 32) selects the level's alternative shape.
    const bool alt = A.lb >= 1 && A.lb <= 5 && ((A.shapes >> (A.lb - 1)) & 1);
    switch (A.lb) {
        case 1:
            if (CM_B2_FAST && !alt)
                return launch_k(phase_b2_kernel<KIND>, dim3((nact + 31) / 32), dim3(128), st, 1,
                                A.S, A.R, A.f, A.H, A.W,
                                SearchParams{A.alpha, A.G, A.K, 1, 4, A.one_step},
                                A.ncolors, A.colour, read_colour(A), A.c_out, A.active);
            return launch_warp<KIND, CM_B2_GT, 16 / CM_B2_GT>(A, nact, st);
        case 2:
            if (alt) return launch_warp<KIND, 32, 1>(A, nact, st);
            return launch_warp<KIND, CM_B4_GT, 32 / CM_B4_GT>(A, nact, st);
        case 3:
            if (alt) return launch_cluster<KIND, 64, 1, 1>(A, nact, st);
            return launch_warp<KIND, 32, 2>(A, nact, st);
        case 4:
            if (alt) return launch_warp<KIND, 32, 4>(A, nact, st);
            return launch_cluster<KIND, 128, 1, 1>(A, nact, st);
        case 5:
            if (alt) return launch_cluster<KIND, 128, 1, 2>(A, nact, st);
            return launch_cluster<KIND, 256, 1, 1>(A, nact, st);
        case 6: return launch_cluster<KIND, 256, 2, 1>(A, nact, st);
        case 7: return launch_cluster<KIND, 256, 4, 1>(A, nact, st);
        case 8: return launch_cluster<KIND, 256, 8, 1>(A, nact, st);
        case 9: return launch_cluster<KIND, 512, 8, 1>(A, nact, st);
        case 10: return launch_cluster<KIND, 1024, 8, 1>(A, nact, st);
        case 11: return launch_cluster<KIND, 1024, 8, 2>(A, nact, st);
        default: return cudaErrorInvalidValue;
    }
}

// The paper's block sides b = 2^lb - 1 (Sec. 2.2) on the kernel shapes of
// side 1 << lb, whose 8 << lb ring slots cover the 8b ring pixels.
template <int KIND>
static cudaError_t launch_blocks_odd_kind(const PhaseArgs& A, cudaStream_t st) {
    const int b = A.bs;
    if (b < 2 || b > (1 << A.lb) || b <= (1 << (A.lb - 1))) return cudaErrorInvalidValue;
    const int nbi = (A.H + b - 1) / b, nbj = (A.W + b - 1) / b;
    const int nact = active_slots(nbi, nbj, A.ncolors);
    switch (A.lb) {
        case 2: return launch_warp<KIND, CM_B4_GT, 32 / CM_B4_GT, false>(A, nact, st);
        case 3: return launch_warp<KIND, 32, 2, false>(A, nact, st);
        case 4: return launch_cluster<KIND, 128, 1, 1, false>(A, nact, st);
        case 5: return launch_cluster<KIND, 256, 1, 1, false>(A, nact, st);
        case 6: return launch_cluster<KIND, 256, 2, 1, false>(A, nact, st);
        case 7: return launch_cluster<KIND, 256, 4, 1, false>(A, nact, st);
        case 8: return launch_cluster<KIND, 256, 8, 1, false>(A, nact, st);
        case 9: return launch_cluster<KIND, 512, 8, 1, false>(A, nact, st);
        case 10: return launch_cluster<KIND, 1024, 8, 1, false>(A, nact, st);
        case 11: return launch_cluster<KIND, 1024, 8, 2, false>(A, nact, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int KIND>
cudaError_t blocks_phase_kind(const PhaseArgs& A, cudaStream_t st) {
    return launch_blocks_kind<KIND>(A, st);
}

template <int KIND>
cudaError_t blocks_phase_odd_kind(const PhaseArgs& A, cudaStream_t st) {
    return launch_blocks_odd_kind<KIND>(A, st);
}

template <int KIND>
cudaError_t coarse_phase_kind(const PhaseArgs& A, const float* partials, float* cj,
                              cudaStream_t st) {
    return launch_coarse_kind<KIND>(A, partials, cj, st);
}

// Clusters of more than 8 CTAs need the non-portable size allowed per kernel;
// run once per process before the first launch (outside stream capture).
template <int KIND>
cudaError_t coarse_setup_kind() {
    cudaError_t e = cudaSuccess;
#define CM_SETUP(LB, CT, Q, RPT, SPEC, DMAX)                                                  \
    if (Q > 8 && e == cudaSuccess)                                                            \
        e = cudaFuncSetAttribute(phase_coarse_kernel<KIND, CT, Q, RPT>,                       \
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    CM_COARSE_SHAPES(CM_SETUP)
#undef CM_SETUP
    return e;
}

}  // namespace cm

// Explicit instantiation of one kind's entry points (in its own unit), and of
// its odd-side entry point (in another).
#define CM_BLOCKS_INSTANTIATE(KIND)                                                           \
    namespace cm {                                                                            \
    template cudaError_t blocks_phase_kind<KIND>(const PhaseArgs&, cudaStream_t);             \
    template cudaError_t coarse_phase_kind<KIND>(const PhaseArgs&, const float*, float*,      \
                                                 cudaStream_t);                               \
    template cudaError_t coarse_setup_kind<KIND>();                                           \
    }

#define CM_BLOCKS_ODD_INSTANTIATE(KIND)                                                       \
    namespace cm {                                                                            \
    template cudaError_t blocks_phase_odd_kind<KIND>(const PhaseArgs&, cudaStream_t);         \
    }
