// cm_phase_b1.cu -- the finest level of the sweep (1x1 blocks).
//
// Alg. 1 of the paper made colour-parallel: one thread per pixel of the
// active colour; the CTA stages the phase state of its tile plus a 2-pixel
// halo in shared memory; each thread runs the block search on its pixel.
//
// Interior fast path.  With p interior, the only window entry that moves
// with c is p itself, so per candidate c:
//  * at p, the plane normals do not move and only delta does:
//    kbar_t(c) = 2h (rsqrt(q1) + rsqrt(q2)) (delta_t - c), one FMA;
//  * at a neighbour q of p, p is an end point of one line of q (recomputed
//    from affine coefficients: 13 FP32 operations, two rsqrt) and a flanking
//    point of one plane of another line (one rsqrt); the two remaining
//    directions are constant and enter only through their min and max.
// This is the same function of c as the generic ring evaluation (used at the
// image border, where clamping duplicates p); only FP32 rounding differs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cm_device.cuh"
#include "cm_kernels.h"
#include "cm_search.cuh"

namespace cm {

// The paper's finest-level estimate: Alg. 2 with t = 0, c_0 = 0, eta_0 = 1:
// c_1 = (c_{1/2} + alpha f*) / (2 + alpha), c_{1/2} from paper_chalf.
template <int KIND>
__device__ __forceinline__ float paper_candidate(const float w[9], float fstar, float alpha) {
    return (paper_chalf<KIND>(w) + alpha * fstar) / (2.0f + alpha);
}

// For p at window position POS of its neighbour: the line with p as an end
// point (TF) and the line with p as a flank (TH), flank index ZI (0/1).
template <int POS> struct PosLines;
template <> struct PosLines<3> { static constexpr int TF = 0, TH = 1, ZI = 0; };
template <> struct PosLines<5> { static constexpr int TF = 0, TH = 1, ZI = 1; };
template <> struct PosLines<1> { static constexpr int TF = 1, TH = 0, ZI = 0; };
template <> struct PosLines<7> { static constexpr int TF = 1, TH = 0, ZI = 1; };
template <> struct PosLines<0> { static constexpr int TF = 2, TH = 3, ZI = 0; };
template <> struct PosLines<8> { static constexpr int TF = 2, TH = 3, ZI = 1; };
template <> struct PosLines<2> { static constexpr int TF = 3, TH = 2, ZI = 0; };
template <> struct PosLines<6> { static constexpr int TF = 3, TH = 2, ZI = 1; };

struct NbConst {
    float dq0, dl0, e10, e20;             // full direction at c = 0
    float eh0, fds, ds4, thd, kh0;        // half direction
    // the two constant directions ka, kb: (min, max) for the extreme-direction
    // kinds; (ka + kb, ((ka - kb) / 2)^2) for the Euler-fit kinds, whose
    // constant pair is the other orthogonal pair of lines
    float kab0, kab1;
};

template <int DR, int DC>
__device__ __forceinline__ void nb_window(const float w25[25], float w[9]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) w[3 * a + b] = w25[5 * (1 + DR + a) + (1 + DC + b)];
}

template <int KIND, int DR, int DC>
__device__ __forceinline__ NbConst nb_init(const float w25[25]) {
    constexpr int POS = 4 - 3 * DR - DC;
    constexpr int TF = PosLines<POS>::TF, TH = PosLines<POS>::TH, ZI = PosLines<POS>::ZI;
    static_assert((TF >> 1) == (TH >> 1), "the moving lines are one orthogonal pair");
    float w[9];
    nb_window<DR, DC>(w25, w);
    NbConst n;
    const KBar4 k = direction_curvatures(w);
    float ka = 0.0f, kb = 0.0f;
    bool first = true;
#pragma unroll
    for (int t = 0; t < 4; ++t)
        if (t != TF && t != TH) {
            if (first) {
                ka = k.k[t];
                first = false;
            } else {
                kb = k.k[t];
            }
        }
    if (KIND == KIND_MEAN || KIND == KIND_GAUSS) {
        n.kab0 = fminf(ka, kb);
        n.kab1 = fmaxf(ka, kb);
    } else {
        const float hd = 0.5f * (ka - kb);
        n.kab0 = ka + kb;
        n.kab1 = hd * hd;
    }
    {   // full direction: affine coefficients at c = 0
        const int X = line_x(TF), Y = line_y(TF);
        const float two_h = line_two_h(TF);
        n.dq0 = 0.5f * (w[Y] - w[X]);
        n.dl0 = two_h * fmaf(0.5f, w[X] + w[Y], -w[4]);
        const float S = w[X] + w[Y];
        n.e10 = fmaf(-2.0f, w[line_z1(TF)], S);
        n.e20 = fmaf(-2.0f, w[line_z2(TF)], S);
    }
    {   // half direction: one plane moves with its flank
        const int X = line_x(TH), Y = line_y(TH);
        const float two_h = line_two_h(TH), h2 = line_h2(TH);
        const float Dq = 0.5f * (w[Y] - w[X]);
        const float ds2 = fmaf(Dq, Dq, h2);
        const float S = w[X] + w[Y];
        const float Zm = ZI == 0 ? w[line_z1(TH)] : w[line_z2(TH)];
        const float Zc = ZI == 0 ? w[line_z2(TH)] : w[line_z1(TH)];
        const float ec = fmaf(-2.0f, Zc, S);
        n.fds = 4.0f * ds2;
        n.ds4 = ds2 * ds2;
        n.thd = two_h * fmaf(0.5f, S, -w[4]);
        n.kh0 = n.thd * rsqrtf(fmaf(ec, ec, n.fds) * n.ds4);
        n.eh0 = fmaf(-2.0f, Zm, S);
    }
    return n;
}

template <int KIND, int DR, int DC>
__device__ __forceinline__ float nb_eval(const NbConst& n, float c) {
    constexpr int POS = 4 - 3 * DR - DC;
    constexpr int TF = PosLines<POS>::TF;
    constexpr float dq1 = line_y(TF) == POS ? 0.5f : -0.5f;
    constexpr float h2 = TF < 2 ? 1.0f : 2.0f;
    constexpr float dl1 = 0.5f * (TF < 2 ? 2.0f : 2.8284271247461903f);
    const float Dq = fmaf(dq1, c, n.dq0);
    const float ds2 = fmaf(Dq, Dq, h2);
    const float fds = 4.0f * ds2;
    const float ds4 = ds2 * ds2;
    const float e1 = c + n.e10, e2 = c + n.e20;
    const float r = rsqrtf(fmaf(e1, e1, fds) * ds4) + rsqrtf(fmaf(e2, e2, fds) * ds4);
    const float kf = fmaf(dl1, c, n.dl0) * r;
    const float e = fmaf(-2.0f, c, n.eh0);
    const float kh = fmaf(n.thd, rsqrtf(fmaf(e, e, n.fds) * n.ds4), n.kh0);
    if (KIND == KIND_MEAN || KIND == KIND_GAUSS) {
        const float kmin = fminf(fminf(kf, kh), n.kab0);
        const float kmax = fmaxf(fmaxf(kf, kh), n.kab1);
        return KIND == KIND_MEAN ? 0.5f * fabsf(kmin + kmax) : fabsf(kmin * kmax);
    }
    // Euler fit (kappa_signed): a = (kf + kh + ka + kb) / 4; the moving pair
    // contributes ((kf - kh) / 2)^2 and the constant pair kab1 to b^2 + s^2
    const float a = 0.25f * ((kf + kh) + n.kab0);
    if (KIND == KIND_MEAN_EULER) return fabsf(a);
    const float hd = 0.5f * (kf - kh);
    return fabsf(fmaf(a, a, -fmaf(hd, hd, n.kab1)));
}

// Tile of one CTA: 128 active pixels of the colour.  Checkerboard: 32 x 8
// (every other pixel); p x p colours: 16p x 8p (every p-th pixel each way).
template <int NCOL>
struct B1Tile {
    static constexpr int P = NCOL == 16 ? 4 : (NCOL == 9 ? 3 : 2);
    static constexpr int TW = NCOL == 2 ? 32 : 16 * P;  // tile columns
    static constexpr int TH = NCOL == 2 ? 8 : 8 * P;    // tile rows
    static constexpr int THREADS = 128;                 // one per active pixel
};

#ifndef CM_B1_MIN_BLOCKS
#define CM_B1_MIN_BLOCKS 3
#endif

template <int KIND, int NCOL>
__global__ void __launch_bounds__(128, CM_B1_MIN_BLOCKS) phase_b1_kernel(const float* __restrict__ S,
                                                       float* __restrict__ R,
                                                       const float* __restrict__ f, int H,
                                                       int W, SearchParams sp, int k,
                                                       int use_paper, float* __restrict__ c_out,
                                                       const int* __restrict__ active) {
    if (active && *active == 0) return;
    constexpr int TW = B1Tile<NCOL>::TW, TH = B1Tile<NCOL>::TH;
    __shared__ float tile[TH + 4][TW + 5];
    const int r0 = blockIdx.y * TH, c0 = blockIdx.x * TW;
    // Tiles away from the left and right edges of an image whose rows are
    // 16-byte aligned: the halo columns c0 - 2 .. c0 + TW + 1 lie in the
    // aligned span c0 - 4 .. c0 + TW + 3, read as float4 words; each pixel
    // keeps the array that holds its phase state (R for colours < k).  A row
    // of 1 x 1 blocks holds the colours cmin .. cmax (both for the
    // checkerboard, p (r mod p) + 0 .. p - 1 for p x p colourings), so R is
    // read only on rows with a colour < k and S only on rows with a colour
    // >= k.  Rows clamp as in the scalar path.
    const bool vec = (W & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(S) | reinterpret_cast<uintptr_t>(R)) & 15) == 0 &&
                     c0 >= 4 && c0 + TW + 4 <= W;
    if (vec) {
        constexpr int NV = (TW + 8) / 4;   // float4 words per tile row
        for (int i = threadIdx.x; i < (TH + 4) * NV; i += 128) {
            const int lr = i / NV, v = i - lr * NV;
            const int r = clampi(r0 - 2 + lr, 0, H - 1);
            const int cb = c0 - 4 + 4 * v;   // column of the word's first element
            const size_t off = (size_t)r * W + cb;
            constexpr int P = B1Tile<NCOL>::P;
            const int cmin = NCOL == 2 ? 0 : P * (r % P);
            const int cmax = NCOL == 2 ? 1 : cmin + P - 1;
            float4 sv = make_float4(0.0f, 0.0f, 0.0f, 0.0f), rv = sv;
            if (cmax >= k) sv = *reinterpret_cast<const float4*>(S + off);
            if (k > cmin) rv = *reinterpret_cast<const float4*>(R + off);
            float e[4] = {sv.x, sv.y, sv.z, sv.w};
            const float o[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (pixel_colour(r, cb + q, 0, NCOL) < k) e[q] = o[q];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int lc = 4 * v - 2 + q;   // cb + q - (c0 - 2)
                if (lc >= 0 && lc < TW + 4) tile[lr][lc] = e[q];
            }
        }
    } else {
        for (int i = threadIdx.x; i < (TH + 4) * (TW + 4); i += 128) {
            int lr = i / (TW + 4), lc = i - lr * (TW + 4);
            int r = clampi(r0 - 2 + lr, 0, H - 1), c = clampi(c0 - 2 + lc, 0, W - 1);
            tile[lr][lc] = phase_read(S, R, r, c, W, 0, NCOL, k);
        }
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int r, c;
    if (NCOL == 2) {
        r = r0 + ty;
        c = c0 + 2 * tx + ((r + k) & 1);
    } else {
        constexpr int P = B1Tile<NCOL>::P;
        r = r0 + P * ty + k / P;
        c = c0 + P * tx + k % P;
    }
    if (r >= H || c >= W) return;
    const int lr = r - r0, lc = c - c0;   // window (i, j) = tile[lr + i][lc + j]
    float w25[25];
    unsigned mask = 0;   // window entries that are the pixel itself after clamping
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            w25[5 * i + j] = tile[lr + i][lc + j];
            bool self = clampi(r + i - 2, 0, H - 1) == r && clampi(c + j - 2, 0, W - 1) == c;
            mask |= (self ? 1u : 0u) << (5 * i + j);
        }
    const size_t p = (size_t)r * W + c;
    const float up = w25[12];
    const float S1 = up - f[p];
    float cp = 0.0f;
    if (use_paper || sp.one_step) {
        float w[9];
        nb_window<0, 0>(w25, w);
        cp = paper_candidate<KIND>(w, -S1, sp.alpha);
    }
    const bool interior = r >= 1 && r <= H - 2 && c >= 1 && c <= W - 2;
    float cbest;
    if (interior) {
        float ncs[4], csd[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float w[9];
            nb_window<0, 0>(w25, w);
            const AffDir d = aff_dir(w, 1u << 4, t);
            const float ds2 = fmaf(d.dq0, d.dq0, line_h2(t));
            const float fds = 4.0f * ds2, ds4 = ds2 * ds2;
            const float sr = line_two_h(t) * (rsqrtf(fmaf(d.e10, d.e10, fds) * ds4) +
                                              rsqrtf(fmaf(d.e20, d.e20, fds) * ds4));
            // kbar_t(c) = sr (delta_t - c) = csd - sr c
            ncs[t] = -sr;
            csd[t] = sr * fmaf(0.5f, w[line_x(t)] + w[line_y(t)], -w[4]);
        }
        const NbConst n0 = nb_init<KIND, -1, -1>(w25), n1 = nb_init<KIND, -1, 0>(w25),
                      n2 = nb_init<KIND, -1, 1>(w25), n3 = nb_init<KIND, 0, -1>(w25),
                      n4 = nb_init<KIND, 0, 1>(w25), n5 = nb_init<KIND, 1, -1>(w25),
                      n6 = nb_init<KIND, 1, 0>(w25), n7 = nb_init<KIND, 1, 1>(w25);
        auto ring_fast = [&](float cc) {
            const float k0 = fmaf(ncs[0], cc, csd[0]), k1 = fmaf(ncs[1], cc, csd[1]);
            const float k2 = fmaf(ncs[2], cc, csd[2]), k3 = fmaf(ncs[3], cc, csd[3]);
            float acc = kappa_abs<KIND>(k0, k1, k2, k3);
            acc += nb_eval<KIND, -1, -1>(n0, cc);
            acc += nb_eval<KIND, -1, 0>(n1, cc);
            acc += nb_eval<KIND, -1, 1>(n2, cc);
            acc += nb_eval<KIND, 0, -1>(n3, cc);
            acc += nb_eval<KIND, 0, 1>(n4, cc);
            acc += nb_eval<KIND, 1, -1>(n5, cc);
            acc += nb_eval<KIND, 1, 0>(n6, cc);
            acc += nb_eval<KIND, 1, 1>(n7, cc);
            return acc;
        };
        cbest = sp.one_step ? block_search_onestep(ring_fast, sp, 1.0f, S1, cp)
                            : block_search_1site(ring_fast, sp, 1.0f, S1, use_paper != 0, cp);
    } else {
        // Border pixel: clamping may duplicate p inside a neighbour's window;
        // evaluate every in-image ring pixel from the shifted 5x5 window.
        unsigned ringv = 0;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr)
#pragma unroll
            for (int dc = -1; dc <= 1; ++dc) {
                bool in = r + dr >= 0 && r + dr < H && c + dc >= 0 && c + dc < W;
                ringv |= (in ? 1u : 0u) << (3 * (dr + 1) + (dc + 1));
            }
        auto ring = [&](float cs) {
            float v[25];
#pragma unroll
            for (int i = 0; i < 25; ++i) v[i] = ((mask >> i) & 1u) ? w25[i] + cs : w25[i];
            float acc = 0.0f;
#pragma unroll
            for (int qr = 0; qr < 3; ++qr)
#pragma unroll
                for (int qc = 0; qc < 3; ++qc) {
                    float w[9];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) w[3 * a + b] = v[5 * (qr + a) + (qc + b)];
                    float t = abs_curvature<KIND>(w);
                    acc += ((ringv >> (3 * qr + qc)) & 1u) ? t : 0.0f;
                }
            return acc;
        };
        cbest = sp.one_step ? block_search_onestep(ring, sp, 1.0f, S1, cp)
                            : block_search_1site(ring, sp, 1.0f, S1, use_paper != 0, cp);
    }
    R[p] = up + cbest;
    if (c_out) c_out[p] = cbest;
}

template <int KIND>
static cudaError_t launch_b1_kind(const PhaseArgs& A, cudaStream_t st) {
    SearchParams sp{A.alpha, A.G, A.K};
    sp.one_step = A.one_step;
    auto go = [&](auto kern, int TW, int TH) {
        dim3 grid((A.W + TW - 1) / TW, (A.H + TH - 1) / TH);
        return launch_k(kern, grid, dim3(128), st, 1, A.S, A.R, A.f, A.H, A.W, sp, A.colour,
                        A.use_paper, A.c_out, A.active);
    };
    switch (A.ncolors) {
        case 2: return go(phase_b1_kernel<KIND, 2>, B1Tile<2>::TW, B1Tile<2>::TH);
        case 4: return go(phase_b1_kernel<KIND, 4>, B1Tile<4>::TW, B1Tile<4>::TH);
        case 9: return go(phase_b1_kernel<KIND, 9>, B1Tile<9>::TW, B1Tile<9>::TH);
        case 16: return go(phase_b1_kernel<KIND, 16>, B1Tile<16>::TW, B1Tile<16>::TH);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_phase_b1(const PhaseArgs& A, cudaStream_t st) {
    switch (A.kind) {
        case KIND_MEAN: return launch_b1_kind<KIND_MEAN>(A, st);
        case KIND_GAUSS: return launch_b1_kind<KIND_GAUSS>(A, st);
        case KIND_MEAN_EULER: return launch_b1_kind<KIND_MEAN_EULER>(A, st);
        case KIND_GAUSS_EULER: return launch_b1_kind<KIND_GAUSS_EULER>(A, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace cm
