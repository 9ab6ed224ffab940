// cm_kernels.cu -- sm_103a kernels of the coloured block-subspace sweep.
//
//  energy_kernel       F(u) = sum |kappa| + alpha/2 (u - f)^2 (Eq. MCM / Eq. GCM):
//                      smem halo tile, FP32 per pixel, FP64 CTA partials and a
//                      fixed-order FP64 finish in the last CTA (deterministic).
//  curvature_kernel    signed kappa per pixel (diagnostics and tests).
//  phase_b1_kernel     finest level (1x1 blocks, Alg. 1 made colour-parallel):
//                      one thread per active pixel, 5x5 window from a smem tile.
//  phase_block_kernel  levels with block side b >= 2 (Sec. 2.2): a group of GT
//                      threads per block; the block's ring windows live in
//                      registers; every candidate energy is a group reduction.
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

template <int KIND>
__global__ void __launch_bounds__(256) energy_kernel(const float* __restrict__ u,
                                                     const float* __restrict__ f, int H, int W,
                                                     float alpha, double* __restrict__ partials,
                                                     unsigned int* __restrict__ ticket,
                                                     double* __restrict__ E_out) {
    __shared__ float tile[E_TH + 2][E_TW + 3];
    __shared__ double wsum[8];
    __shared__ bool is_last;
    const int r0 = blockIdx.y * E_TH, c0 = blockIdx.x * E_TW;
    for (int i = threadIdx.x; i < (E_TH + 2) * (E_TW + 2); i += 256) {
        int lr = i / (E_TW + 2), lc = i - lr * (E_TW + 2);
        int r = clampi(r0 - 1 + lr, 0, H - 1), c = clampi(c0 - 1 + lc, 0, W - 1);
        tile[lr][lc] = u[(size_t)r * W + c];
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
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
            float e = w[4] - f[(size_t)r * W + c];
            acc += abs_curvature(w, KIND) + 0.5f * alpha * e * e;
        }
    }
    double d = (double)acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (tx == 0) wsum[ty] = d;
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += wsum[i];
        partials[bid] = s;
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
    if (tx == 0) wsum[ty] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += wsum[i];
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
    KBar4 k = direction_curvatures(w);
    float kmin = fminf(fminf(k.k[0], k.k[1]), fminf(k.k[2], k.k[3]));
    float kmax = fmaxf(fmaxf(k.k[0], k.k[1]), fmaxf(k.k[2], k.k[3]));
    out[(size_t)r * W + c] = KIND == KIND_MEAN ? 0.5f * (kmin + kmax) : kmin * kmax;
}

// ---------------------------------------------------------------------------
// Block search shared by both phase kernels.
//
// ring(c) returns sum_{q in ring(A)} |kappa_q(u + c phi_A)|, uniform over the
// threads that search the same block.  The fidelity part is carried as
// alpha s/2 (c - c_fid)^2, which differs from alpha/2 (s c^2 + 2 c S1) by the
// constant alpha s c_fid^2 / 2 and so selects the same c, without the FP32
// cancellation of the expanded form on large blocks.

struct SearchParams {
    float alpha;
    int G;   // grid points (odd)
    int K;   // golden-section evaluations
};

template <class Ring>
__device__ __forceinline__ float block_search(Ring&& ring, const SearchParams& p, float s,
                                              float S1, bool has_paper, float c_paper) {
    const float c_fid = -S1 / s;
    const float half_as = 0.5f * p.alpha * s;
    auto energy = [&](float c, float rk) {
        float t = c - c_fid;
        return fmaf(half_as * t, t, rk);
    };
    Best best;
    best.c = 0.0f;
    best.E = energy(0.0f, ring(0.0f));
    if (has_paper) {
        float Ep = energy(c_paper, ring(c_paper));
        consider(best, c_paper, Ep);
    }
    const float Rk = ring(c_fid);
    const float rho = sqrtf(2.0f * Rk / (p.alpha * s));
    const int mid = (p.G - 1) / 2;
    float gbest = c_fid, Egbest = INFINITY;
    for (int i = 0; i < p.G; ++i) {
        float t = (2.0f * (float)i) / (float)(p.G - 1) - 1.0f;
        float g = c_fid + rho * t;
        float rk = (i == mid) ? Rk : ring(g);
        float E = energy(g, rk);
        consider(best, g, E);
        if (E < Egbest) {
            Egbest = E;
            gbest = g;
        }
    }
    const float D = 2.0f * rho / (float)(p.G - 1);
    float lo = gbest - D, hi = gbest + D;
    float x1 = hi - GOLDEN * (hi - lo), x2 = lo + GOLDEN * (hi - lo);
    float E1 = energy(x1, ring(x1));
    consider(best, x1, E1);
    float E2 = energy(x2, ring(x2));
    consider(best, x2, E2);
    for (int it = 2; it < p.K; ++it) {
        const bool left = E1 < E2;
        float xn;
        if (left) {
            hi = x2;
            x2 = x1;
            E2 = E1;
            xn = hi - GOLDEN * (hi - lo);
        } else {
            lo = x1;
            x1 = x2;
            E1 = E2;
            xn = lo + GOLDEN * (hi - lo);
        }
        const float En = energy(xn, ring(xn));
        consider(best, xn, En);
        if (left) {
            x1 = xn;
            E1 = En;
        } else {
            x2 = xn;
            E2 = En;
        }
    }
    return best.c;
}

// Plane distances of one line (for the paper's one-step candidate).
__device__ __forceinline__ void dir_dist(float A, float B, float O, float Z1, float Z2,
                                         float four_h2, float two_h, float& d1, float& d2) {
    const float D = B - A, S = A + B;
    const float delta = fmaf(0.5f, S, -O);
    const float base = fmaf(D, D, four_h2);
    const float e1 = fmaf(-2.0f, Z1, S), e2 = fmaf(-2.0f, Z2, S);
    d1 = two_h * delta * rsqrtf(fmaf(e1, e1, base));
    d2 = two_h * delta * rsqrtf(fmaf(e2, e2, base));
}

// The paper's finest-level estimate: Alg. 2 with t = 0, c_0 = 0, eta_0 = 1:
// c_1 = (c_{1/2} + alpha f*) / (2 + alpha) with c_{1/2} the mean plane
// distance (Eq. c-sol1) or, for Gaussian curvature, the distance pair of the
// extreme direction curvature with the smaller magnitude (Prop. 2).
template <int KIND>
__device__ __forceinline__ float paper_candidate(const float w[9], float fstar, float alpha) {
    const float SQ2x2 = 2.8284271247461903f;
    float d[8];
    dir_dist(w[3], w[5], w[4], w[1], w[7], 4.0f, 2.0f, d[0], d[1]);
    dir_dist(w[1], w[7], w[4], w[3], w[5], 4.0f, 2.0f, d[2], d[3]);
    dir_dist(w[0], w[8], w[4], w[2], w[6], 8.0f, SQ2x2, d[4], d[5]);
    dir_dist(w[2], w[6], w[4], w[0], w[8], 8.0f, SQ2x2, d[6], d[7]);
    float chalf;
    if (KIND == KIND_MEAN) {
        chalf = 0.125f * (((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])));
    } else {
        KBar4 k = direction_curvatures(w);
        int tmin = 0, tmax = 0;
#pragma unroll
        for (int t = 1; t < 4; ++t) {
            if (k.k[t] < k.k[tmin]) tmin = t;
            if (k.k[t] > k.k[tmax]) tmax = t;
        }
        int ts = fabsf(k.k[tmin]) <= fabsf(k.k[tmax]) ? tmin : tmax;
        float dd0 = d[0], dd1 = d[1];
#pragma unroll
        for (int t = 1; t < 4; ++t)
            if (ts == t) {
                dd0 = d[2 * t];
                dd1 = d[2 * t + 1];
            }
        chalf = 0.5f * (dd0 + dd1);
    }
    return (chalf + alpha * fstar) / (2.0f + alpha);
}

// ---------------------------------------------------------------------------
// Finest level: every pixel is a block.

template <int NCOL>
struct B1Tile {
    static constexpr int TW = 32;
    static constexpr int TH = NCOL == 2 ? 16 : 32;
};

template <int KIND, int NCOL>
__global__ void __launch_bounds__(256) phase_b1_kernel(const float* __restrict__ S,
                                                       float* __restrict__ R,
                                                       const float* __restrict__ f, int H,
                                                       int W, SearchParams sp, int k,
                                                       int use_paper, float* __restrict__ c_out) {
    constexpr int TW = B1Tile<NCOL>::TW, TH = B1Tile<NCOL>::TH;
    __shared__ float tile[TH + 4][TW + 5];
    const int r0 = blockIdx.y * TH, c0 = blockIdx.x * TW;
    for (int i = threadIdx.x; i < (TH + 4) * (TW + 4); i += 256) {
        int lr = i / (TW + 4), lc = i - lr * (TW + 4);
        int r = clampi(r0 - 2 + lr, 0, H - 1), c = clampi(c0 - 2 + lc, 0, W - 1);
        tile[lr][lc] = phase_read(S, R, r, c, W, 0, NCOL, k);
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int r, c;
    if (NCOL == 2) {
        r = r0 + ty;
        c = c0 + 2 * tx + ((r + k) & 1);
    } else {
        r = r0 + 2 * ty + (k >> 1);
        c = c0 + 2 * tx + (k & 1);
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
    unsigned ringv = 0;   // 3x3 neighbours inside the image
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
                float t = abs_curvature(w, KIND);
                acc += ((ringv >> (3 * qr + qc)) & 1u) ? t : 0.0f;
            }
        return acc;
    };
    const size_t p = (size_t)r * W + c;
    const float up = w25[12];
    const float S1 = up - f[p];
    float cp = 0.0f;
    if (use_paper) {
        float w[9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) w[3 * a + b] = w25[5 * (a + 1) + (b + 1)];
        cp = paper_candidate<KIND>(w, -S1, sp.alpha);
    }
    float cbest = block_search(ring, sp, 1.0f, S1, use_paper != 0, cp);
    R[p] = up + cbest;
    if (c_out) c_out[p] = cbest;
}

// ---------------------------------------------------------------------------
// Levels with b >= 2.

__device__ __forceinline__ int perim_count(int h, int w) {
    return h == 1 ? w : (w == 1 ? h : 2 * w + 2 * (h - 2));
}

// Position (i, j) of the t-th cell on the perimeter of an h x w box: top row,
// bottom row, then the left and right cells of the middle rows.
__device__ __forceinline__ void perim_pos(int t, int h, int w, int& i, int& j) {
    if (h == 1) {
        i = 0;
        j = t;
    } else if (w == 1) {
        i = t;
        j = 0;
    } else if (t < w) {
        i = 0;
        j = t;
    } else if (t < 2 * w) {
        i = h - 1;
        j = t - w;
    } else {
        int u = t - 2 * w;
        i = 1 + (u >> 1);
        j = (u & 1) ? w - 1 : 0;
    }
}

template <int GT>
__device__ __forceinline__ float group_sum(float v, float* red /* smem, 2 x 32 */, int& flip) {
    if (GT <= 32) {
#pragma unroll
        for (int off = GT / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, GT);
        return v;
    } else {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        constexpr int NW = GT / 32;
        float* buf = red + 32 * flip;
        flip ^= 1;
        if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = v;
        __syncthreads();
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < NW; ++i) s += buf[i];
        return s;
    }
}

template <int KIND, int GT, int RPT>
__global__ void __launch_bounds__(GT > 32 ? GT : 128) phase_block_kernel(
    const float* __restrict__ S, float* __restrict__ R, const float* __restrict__ f, int H, int W,
    SearchParams sp, int lb, int ncol, int k, float* __restrict__ c_out) {
    constexpr int CTA = GT > 32 ? GT : 128;
    constexpr int GPC = CTA / GT;
    __shared__ float red[64];
    int flip = 0;
    const int b = 1 << lb;
    const int nbi = (H + b - 1) >> lb, nbj = (W + b - 1) >> lb;
    const int gid = threadIdx.x / GT, lane = threadIdx.x % GT;
    const int a = blockIdx.x * GPC + gid;
    int bi, bj, nact;
    if (ncol == 2) {
        int half = (nbj + 1) >> 1;
        bi = a / half;
        bj = 2 * (a - bi * half) + ((bi + k) & 1);
        nact = nbi * half;
    } else {
        int hj = (nbj + 1) >> 1, hi = (nbi + 1) >> 1;
        int ai = a / hj;
        bi = 2 * ai + (k >> 1);
        bj = 2 * (a - ai * hj) + (k & 1);
        nact = hi * hj;
    }
    const bool active = a < nact && bi < nbi && bj < nbj;
    if (GT > 32 && !active) return;   // whole CTA idle
    const int r0 = bi << lb, c0 = bj << lb;
    const int r1 = min(r0 + b, H), c1 = min(c0 + b, W);
    const int bh = active ? r1 - r0 : 0, bw = active ? c1 - c0 : 0;
    const float s = (float)(bh * bw);

    // S1 = sum over the block of u - f (the block's own pixels still hold S).
    float s1 = 0.0f;
    if (active) {
        const int npx = bh * bw;
        if (bw >= GT) {
            for (int rr = r0; rr < r1; ++rr)
                for (int cc = c0 + lane; cc < c1; cc += GT) {
                    size_t p = (size_t)rr * W + cc;
                    s1 += S[p] - f[p];
                }
        } else {
            for (int idx = lane; idx < npx; idx += GT) {
                int rr = idx / bw, cc = idx - rr * bw;
                size_t p = (size_t)(r0 + rr) * W + (c0 + cc);
                s1 += S[p] - f[p];
            }
        }
    }
    const float S1 = group_sum<GT>(s1, red, flip);

    // Ring windows: the outer frame (one pixel outside the block) and the
    // inner frame (the block's boundary pixels), less pixels outside the
    // image and block pixels whose clamped stencil lies inside the block.
    float win[RPT][9];
    unsigned msk[RPT];
    const int Pout = active ? perim_count(bh + 2, bw + 2) : 0;
    const int Pin = active ? perim_count(bh, bw) : 0;
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
        msk[t] = 0;
        const int j = lane + t * GT;
        bool ok = false;
        int rr = 0, cc = 0;
        if (j < Pout + Pin) {
            int li, lj;
            if (j < Pout) {
                perim_pos(j, bh + 2, bw + 2, li, lj);
                rr = r0 - 1 + li;
                cc = c0 - 1 + lj;
                ok = rr >= 0 && rr < H && cc >= 0 && cc < W;
            } else {
                perim_pos(j - Pout, bh, bw, li, lj);
                rr = r0 + li;
                cc = c0 + lj;
                bool interior = (rr - 1 >= r0 || rr == 0) && (rr + 1 < r1 || rr == H - 1) &&
                                (cc - 1 >= c0 || cc == 0) && (cc + 1 < c1 || cc == W - 1);
                ok = !interior;
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) win[t][q] = 0.0f;
        if (ok) {
            unsigned m = 1u << 9;   // bit 9: slot holds a ring pixel
#pragma unroll
            for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                for (int bb = 0; bb < 3; ++bb) {
                    int qr = clampi(rr + aa - 1, 0, H - 1), qc = clampi(cc + bb - 1, 0, W - 1);
                    win[t][3 * aa + bb] = phase_read(S, R, qr, qc, W, lb, ncol, k);
                    bool inA = qr >= r0 && qr < r1 && qc >= c0 && qc < c1;
                    m |= (inA ? 1u : 0u) << (3 * aa + bb);
                }
            msk[t] = m;
        }
    }
    auto ring = [&](float cs) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < RPT; ++t) {
            float w[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) w[q] = ((msk[t] >> q) & 1u) ? win[t][q] + cs : win[t][q];
            float v = abs_curvature(w, KIND);
            acc += ((msk[t] >> 9) & 1u) ? v : 0.0f;
        }
        return group_sum<GT>(acc, red, flip);
    };
    const float cbest = block_search(ring, sp, active ? s : 1.0f, S1, false, 0.0f);
    if (!active) return;
    // Apply: R = S + c on the block (prolongation L_j c_j of Sec. 2.2).
    if (bw >= GT) {
        for (int rr = r0; rr < r1; ++rr)
            for (int cc = c0 + lane; cc < c1; cc += GT) {
                size_t p = (size_t)rr * W + cc;
                R[p] = S[p] + cbest;
            }
    } else {
        const int npx = bh * bw;
        for (int idx = lane; idx < npx; idx += GT) {
            int rr = idx / bw, cc = idx - rr * bw;
            size_t p = (size_t)(r0 + rr) * W + (c0 + cc);
            R[p] = S[p] + cbest;
        }
    }
    if (c_out && lane == 0) c_out[(size_t)bi * nbj + bj] = cbest;
}

// ---------------------------------------------------------------------------
// Launchers.

cudaError_t launch_energy(const float* u, const float* f, int H, int W, float alpha, int kind,
                          double* partials, unsigned int* ticket, double* E_out,
                          cudaStream_t st) {
    dim3 grid((W + E_TW - 1) / E_TW, (H + E_TH - 1) / E_TH);
    if (kind == KIND_MEAN)
        energy_kernel<KIND_MEAN><<<grid, 256, 0, st>>>(u, f, H, W, alpha, partials, ticket, E_out);
    else
        energy_kernel<KIND_GAUSS><<<grid, 256, 0, st>>>(u, f, H, W, alpha, partials, ticket, E_out);
    return cudaGetLastError();
}

size_t energy_partials_needed(int H, int W) {
    return (size_t)((W + E_TW - 1) / E_TW) * (size_t)((H + E_TH - 1) / E_TH);
}

cudaError_t launch_curvature(const float* u, int H, int W, int kind, float* out,
                             cudaStream_t st) {
    dim3 blk(32, 8), grid((W + 31) / 32, (H + 7) / 8);
    if (kind == KIND_MEAN)
        curvature_kernel<KIND_MEAN><<<grid, blk, 0, st>>>(u, H, W, out);
    else
        curvature_kernel<KIND_GAUSS><<<grid, blk, 0, st>>>(u, H, W, out);
    return cudaGetLastError();
}

template <int KIND, int GT, int RPT>
static void launch_block(const PhaseArgs& A, int nact, cudaStream_t st) {
    constexpr int CTA = GT > 32 ? GT : 128;
    constexpr int GPC = CTA / GT;
    int grid = (nact + GPC - 1) / GPC;
    SearchParams sp{A.alpha, A.G, A.K};
    phase_block_kernel<KIND, GT, RPT><<<grid, CTA, 0, st>>>(A.S, A.R, A.f, A.H, A.W, sp, A.lb,
                                                             A.ncolors, A.colour, A.c_out);
}

template <int KIND>
static cudaError_t launch_phase_kind(const PhaseArgs& A, cudaStream_t st) {
    SearchParams sp{A.alpha, A.G, A.K};
    if (A.lb == 0) {
        if (A.ncolors == 2) {
            dim3 grid((A.W + 31) / 32, (A.H + 15) / 16);
            phase_b1_kernel<KIND, 2><<<grid, 256, 0, st>>>(A.S, A.R, A.f, A.H, A.W, sp, A.colour,
                                                           A.use_paper, A.c_out);
        } else {
            dim3 grid((A.W + 31) / 32, (A.H + 31) / 32);
            phase_b1_kernel<KIND, 4><<<grid, 256, 0, st>>>(A.S, A.R, A.f, A.H, A.W, sp, A.colour,
                                                           A.use_paper, A.c_out);
        }
        return cudaGetLastError();
    }
    const int b = 1 << A.lb;
    const int nbi = (A.H + b - 1) / b, nbj = (A.W + b - 1) / b;
    const int nact = A.ncolors == 2 ? nbi * ((nbj + 1) / 2) : ((nbi + 1) / 2) * ((nbj + 1) / 2);
    switch (A.lb) {
        case 1: launch_block<KIND, 16, 1>(A, nact, st); break;
        case 2: launch_block<KIND, 32, 1>(A, nact, st); break;
        case 3: launch_block<KIND, 32, 2>(A, nact, st); break;
        case 4: launch_block<KIND, 32, 4>(A, nact, st); break;
        case 5: launch_block<KIND, 64, 4>(A, nact, st); break;
        case 6: launch_block<KIND, 128, 4>(A, nact, st); break;
        case 7: launch_block<KIND, 256, 4>(A, nact, st); break;
        case 8: launch_block<KIND, 256, 8>(A, nact, st); break;
        case 9: launch_block<KIND, 512, 8>(A, nact, st); break;
        case 10: launch_block<KIND, 1024, 8>(A, nact, st); break;
        case 11: launch_block<KIND, 1024, 16>(A, nact, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_phase(const PhaseArgs& A, cudaStream_t st) {
    return A.kind == KIND_MEAN ? launch_phase_kind<KIND_MEAN>(A, st)
                               : launch_phase_kind<KIND_GAUSS>(A, st);
}

int max_level_log2() { return 11; }

}  // namespace cm
