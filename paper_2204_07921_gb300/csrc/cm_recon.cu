// cm_recon.cu -- reconstruction extension (Sec. 5) with an MRI-like operator.
//
// Minimises J(u) = 1/2 ||A u - b||^2 + alpha sum |kappa(u)| for a real image u,
// with A = M F (MRI: M a 0/1 mask of sampled k-space entries, F the
// orthonormal 2-D DFT) or A = R (CT: a parallel-beam Radon transform with
// linear-interpolation weights, see radon_pos).  The sweep visits the levels fine to coarse and the colours in order
// (Alg. 3); the blocks phi_i of one colour are solved together, because A
// couples them: Sec. 5 replaces each block's curvature term by
// alpha (c_i - d_i)^2 around the curvature-only estimate d_i and solves
//   [Re<A phi_i, A phi_j> + 2 alpha delta_ij] c = Re<b - A u, A phi_i> + 2 alpha d_i
// by conjugate gradients, matrix-free: one product is a scatter of the block
// values, an FFT, the mask, an inverse FFT and block sums.  d_i is c_{1/2} of
// Eq. c-sol1 (Prop. 2 for Gaussian curvature) on the finest level and 0 on
// coarser ones; CG runs a fixed number of iterations from c = 0 and stops
// early only on a zero residual or a non-positive p.Ap.  The start is the
// zero-filled Re(A^H b) for MRI, the filtered backprojection (Ram-Lak) for CT.
//
// The transforms are the library's own (cm_fft.cu: single-precision
// complex, unnormalised; the two 1/sqrt(HW) factors of the orthonormal pair
// are folded into the mask kernels).  Every other step is a kernel of this
// file.  The
// CG scalars stay on the device; the reductions are FP64 with a fixed order
// (per-CTA partials, the last CTA finishes), so a run is deterministic.  One
// cycle is captured as a CUDA graph and launched once per cycle.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "cm_device.cuh"
#include "cm_fft.h"
#include "cm_kernels.h"
#include "cm_recon.h"
#include "cm_search.cuh"

namespace cm {

// ---------------------------------------------------------------------------
// Kernels.

constexpr int RT = 256;              // threads per CTA of every kernel here
constexpr int RED_CTAS = 1024;       // grid of the grid-stride reductions
constexpr int MAX_CTAS = 1 << 16;    // largest reduction grid (partials size)

// Slot of block (bi, bj) among the blocks of its colour: the inverse of
// active_block.
__device__ __forceinline__ int slot_of(int bi, int bj, int nbj, int ncol) {
    if (ncol == 2) return bi * ((nbj + 1) >> 1) + (bj >> 1);
    const int p = colour_side(ncol);
    return (bi / p) * ((nbj + p - 1) / p) + bj / p;
}

// Sum of v over the CTA; the last CTA to finish adds the per-CTA partials in
// a fixed order into *out and clears the ticket.  Every thread must call it.
__device__ void cta_sum_finish(double v, double* partials, unsigned* ticket, double* out) {
    __shared__ double ws[RT / 32];
    __shared__ bool last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < RT / 32; ++i) t += ws[i];
        partials[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += RT) s += ((volatile double*)partials)[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < RT / 32; ++i) t += ws[i];
        *out = t;
        *ticket = 0u;
    }
}

__global__ void __launch_bounds__(RT) to_complex_kernel(const float* __restrict__ u,
                                                        float2* __restrict__ X, size_t N) {
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT)
        X[i] = make_float2(u[i], 0.0f);
}

// After X = F_unnormalised u: X <- M (b - s X) s, so that the inverse
// transform gives A^H (b - A u) (s = 1 / sqrt(HW)).
__global__ void __launch_bounds__(RT) resid_kernel(float2* __restrict__ X,
                                                   const float2* __restrict__ bk,
                                                   const uint8_t* __restrict__ mask, size_t N,
                                                   float s) {
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT) {
        const float2 x = X[i], y = bk[i];
        X[i] = mask[i] ? make_float2((y.x - s * x.x) * s, (y.y - s * x.y) * s)
                       : make_float2(0.0f, 0.0f);
    }
}

// X <- M b s (the zero-filled start A^H b after the inverse transform).
__global__ void __launch_bounds__(RT) masked_data_kernel(float2* __restrict__ X,
                                                         const float2* __restrict__ bk,
                                                         const uint8_t* __restrict__ mask, size_t N,
                                                         float s) {
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT) {
        const float2 y = bk[i];
        X[i] = mask[i] ? make_float2(y.x * s, y.y * s) : make_float2(0.0f, 0.0f);
    }
}

__global__ void __launch_bounds__(RT) real_part_kernel(const float2* __restrict__ X,
                                                       float* __restrict__ u, size_t N) {
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT)
        u[i] = X[i].x;
}

// Z <- sum_i v_i phi_i over the blocks of colour k (zero elsewhere).  Starts a
// CG iteration: a zero residual (rr == 0) ends the iteration loop.
__global__ void __launch_bounds__(RT) scatter_kernel(const float* __restrict__ v,
                                                     float2* __restrict__ Z, int H, int W, int b,
                                                     int ncol, int k, const double* rr, int* stop) {
    if (*stop) return;
    if (*rr == 0.0) {
        *stop = 1;
        return;
    }
    const int nbj = (W + b - 1) / b;
    const size_t N = (size_t)H * W;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT) {
        const int r = (int)(i / W), c = (int)(i - (size_t)r * W);
        const int bi = r / b, bj = c / b;
        Z[i] = block_colour(bi, bj, ncol) == k ? make_float2(v[slot_of(bi, bj, nbj, ncol)], 0.0f)
                                               : make_float2(0.0f, 0.0f);
    }
}

// Z <- M Z s2 (s2 = 1 / HW: both normalisations of A^H A).
__global__ void __launch_bounds__(RT) mask_scale_kernel(float2* __restrict__ Z,
                                                        const uint8_t* __restrict__ mask, size_t N,
                                                        float s2, const int* stop) {
    if (*stop) return;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT) {
        const float2 z = Z[i];
        Z[i] = mask[i] ? make_float2(z.x * s2, z.y * s2) : make_float2(0.0f, 0.0f);
    }
}

enum { GATHER_RHS = 0, GATHER_Q = 1 };

// Block sums of Re(Y) over the blocks of colour k, GS threads per block.
//  GATHER_RHS: r_a = sum + 2 alpha d_a (d_a = c_{1/2}(u) when b = 1), p_a = r_a,
//              c_a = 0; *dot = r.r.
//  GATHER_Q:   q_a = sum + 2 alpha p_a; *dot = p.q.
template <int GS, int MODE, int KIND>
__global__ void __launch_bounds__(RT) gather_kernel(const float2* __restrict__ Y,
                                                    const float* __restrict__ u, int H, int W,
                                                    int b, int ncol, int k, int nslots,
                                                    float twoalpha, float* __restrict__ out,
                                                    float* __restrict__ p, float* __restrict__ c,
                                                    const int* stop, double* partials,
                                                    unsigned* ticket, double* dot) {
    if (MODE == GATHER_Q && *stop) return;
    constexpr int GPC = RT / GS;
    __shared__ double gs[RT / 32];
    const int g = threadIdx.x / GS, lane = threadIdx.x % GS;
    const int a = blockIdx.x * GPC + g;
    const int nbi = (H + b - 1) / b, nbj = (W + b - 1) / b;
    int bi = 0, bj = 0;
    const bool on = a < nslots && active_block(a, nbi, nbj, ncol, k, bi, bj);
    double s = 0.0;
    if (on) {
        const int r0 = bi * b, c0 = bj * b;
        const int bh = min(b, H - r0), bw = min(b, W - c0);
        for (int i = lane; i < bh * bw; i += GS) {
            const int rr = i / bw, cc = i - rr * bw;
            s += (double)Y[(size_t)(r0 + rr) * W + (c0 + cc)].x;
        }
    }
    if (GS > 1) {
#pragma unroll
        for (int off = (GS < 32 ? GS : 32) / 2; off > 0; off >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, off);
    }
    if (GS > 32) {   // one group per CTA: add the warps
        if ((threadIdx.x & 31) == 0) gs[threadIdx.x >> 5] = s;
        __syncthreads();
        s = 0.0;
        for (int i = 0; i < RT / 32; ++i) s += gs[i];
    }
    double contrib = 0.0;
    if (lane == 0 && a < nslots) {
        if (MODE == GATHER_RHS) {
            float d = 0.0f;
            if (on && b == 1) {
                float w[9];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        w[3 * i + j] = u[(size_t)clampi(bi + i - 1, 0, H - 1) * W +
                                         clampi(bj + j - 1, 0, W - 1)];
                d = paper_chalf<KIND>(w);
            }
            const float v = on ? fmaf(twoalpha, d, (float)s) : 0.0f;
            out[a] = v;
            p[a] = v;
            c[a] = 0.0f;
            contrib = (double)v * v;
        } else {
            const float pa = p[a];
            const float v = on ? fmaf(twoalpha, pa, (float)s) : 0.0f;
            out[a] = v;
            contrib = (double)pa * v;
        }
    }
    cta_sum_finish(contrib, partials, ticket, dot);
}

// c += a p, r -= a q with a = rr / pq; *rr_next = r.r.  A non-positive p.q
// (a singular system) ends the iteration loop.
__global__ void __launch_bounds__(RT) cg_update_kernel(float* __restrict__ c,
                                                       float* __restrict__ r,
                                                       const float* __restrict__ p,
                                                       const float* __restrict__ q, int n,
                                                       const double* rr, const double* pq,
                                                       int* stop, double* partials,
                                                       unsigned* ticket, double* rr_next) {
    if (*stop) return;
    const double pqv = *pq;
    if (!(pqv > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *stop = 1;
        return;
    }
    const float al = (float)(*rr / pqv);
    double acc = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT) {
        c[i] = fmaf(al, p[i], c[i]);
        const float ri = fmaf(-al, q[i], r[i]);
        r[i] = ri;
        acc += (double)ri * ri;
    }
    cta_sum_finish(acc, partials, ticket, rr_next);
}

// p <- r + (rr_next / rr) p.
__global__ void __launch_bounds__(RT) cg_dir_kernel(float* __restrict__ p,
                                                    const float* __restrict__ r, int n,
                                                    const double* rr, const double* rr_next,
                                                    const int* stop) {
    if (*stop) return;
    const float beta = (float)(*rr_next / *rr);
    for (int i = blockIdx.x * RT + threadIdx.x; i < n; i += gridDim.x * RT)
        p[i] = fmaf(beta, p[i], r[i]);
}

// u += sum_i c_i phi_i over the blocks of colour k.
__global__ void __launch_bounds__(RT) apply_blocks_kernel(float* __restrict__ u,
                                                          const float* __restrict__ c, int H,
                                                          int W, int b, int ncol, int k) {
    const int nbj = (W + b - 1) / b;
    const size_t N = (size_t)H * W;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT) {
        const int r = (int)(i / W), cc = (int)(i - (size_t)r * W);
        const int bi = r / b, bj = cc / b;
        if (block_colour(bi, bj, ncol) == k) u[i] += c[slot_of(bi, bj, nbj, ncol)];
    }
}

// *out = sum |M s X - b|^2 (X = F_unnormalised u): twice the data term.
__global__ void __launch_bounds__(RT) data_term_kernel(const float2* __restrict__ X,
                                                       const float2* __restrict__ bk,
                                                       const uint8_t* __restrict__ mask, size_t N,
                                                       float s, double* partials,
                                                       unsigned* ticket, double* out) {
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * RT + threadIdx.x; i < N; i += (size_t)gridDim.x * RT) {
        const float2 y = bk[i];
        const float2 x = mask[i] ? make_float2(s * X[i].x, s * X[i].y) : make_float2(0.0f, 0.0f);
        const double dx = (double)x.x - y.x, dy = (double)x.y - y.y;
        acc += dx * dx + dy * dy;
    }
    cta_sum_finish(acc, partials, ticket, out);
}

// trace[(*count)++] = data2 / 2 + alpha * curv.
__global__ void objective_kernel(const double* data2, const double* curv, float alpha,
                                 double* trace, int* count, int cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int l = *count;
    if (l < cap) trace[l] = 0.5 * *data2 + (double)alpha * *curv;
    *count = l + 1;
}

// ---------------------------------------------------------------------------
// CT: n angles theta_a = pi a / n (cos, sin tables from the host); the
// centre of pixel (r, c) sits at x = c - (W-1)/2, y = r - (H-1)/2 and projects
// to the detector position p = x cos + y sin + (D-1)/2 of D unit bins; its
// value is shared by bins floor(p) and floor(p) + 1 with weights 1 - frac(p)
// and frac(p).  D = 2 ceil(hypot(H-1, W-1)/2) + 3 keeps every p in [1, D-2].
// Forward and adjoint are both gathers that call radon_pos with the same
// arguments, so the pair is exactly matched (and needs no atomics).

__device__ __forceinline__ float radon_pos(int r, int c, int H, int W, float cs, float sn,
                                           float half) {
    const float x = (float)c - 0.5f * (float)(W - 1);
    const float y = (float)r - 0.5f * (float)(H - 1);
    return fmaf(x, cs, fmaf(y, sn, half));
}

// S[a][j] = sum over pixels of weight(p, j) U[pixel].x; RADON_LANES
// consecutive lanes per bin, lane g taking the rows (or columns) g, g +
// RADON_LANES, ..., their partial sums added by a fixed butterfly.  Along the
// dominant axis of the angle's direction, p is linear with slope >=
// 1/sqrt(2), so only pixels whose p lies in [j - 1, j + 1) contribute: at
// most three per row (or column), searched in a window one pixel wider on
// each side than the exact interval.
constexpr int RADON_LANES = 8;
__global__ void __launch_bounds__(RT) radon_fwd_kernel(const float2* __restrict__ U,
                                                       float* __restrict__ S, int H, int W,
                                                       int n, int D, const float* __restrict__ cs,
                                                       const float* __restrict__ sn,
                                                       const int* stop) {
    if (stop && *stop) return;   // uniform over the grid
    const long long gi = (long long)blockIdx.x * RT + threadIdx.x;
    const int g = (int)(gi & (RADON_LANES - 1));
    const long long bin = gi / RADON_LANES;
    float acc = 0.0f;
    if (bin < (long long)n * D) {
        const int idx = (int)bin;
        const int a = idx / D, j = idx - a * D;
        const float c = cs[a], sv = sn[a], half = 0.5f * (float)(D - 1);
        const bool rows = fabsf(c) >= fabsf(sv);
        const int outer = rows ? H : W, inner = rows ? W : H;
        const float slope = rows ? c : sv, other = rows ? sv : c;
        const float off_in = 0.5f * (float)(inner - 1), off_out = 0.5f * (float)(outer - 1);
        // the window needs no exact division: it is one pixel wider on each side
        // than the interval, and membership is decided by radon_pos itself
        const float inv = 1.0f / slope;
        for (int o = g; o < outer; o += RADON_LANES) {
            const float base = fmaf((float)o - off_out, other, half);
            float x0 = ((float)(j - 1) - base) * inv, x1 = ((float)(j + 1) - base) * inv;
            if (x0 > x1) {
                const float t = x0;
                x0 = x1;
                x1 = t;
            }
            const int i0 = max((int)floorf(x0 + off_in) - 1, 0);
            const int i1 = min((int)ceilf(x1 + off_in) + 1, inner - 1);
            for (int i = i0; i <= i1; ++i) {
                const int r = rows ? o : i, col = rows ? i : o;
                const float p = radon_pos(r, col, H, W, c, sv, half);
                const float fl = floorf(p);
                const int f = (int)fl;
                const float w = p - fl;
                const float v = U[(size_t)r * W + col].x;
                if (f == j) acc = fmaf(1.0f - w, v, acc);
                else if (f == j - 1) acc = fmaf(w, v, acc);
            }
        }
    }
#pragma unroll
    for (int off = RADON_LANES / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (g == 0 && bin < (long long)n * D) S[bin] = acc;
}

// U[pixel] = scale sum_a ((1 - w) S[a][f] + w S[a][f + 1]) (imaginary part 0);
// RADJ_LANES consecutive lanes per pixel, lane g taking the angles g, g +
// RADJ_LANES, ..., their partial sums added by a fixed butterfly.  A warp
// holds 32 / RADJ_LANES consecutive pixels and every warp runs the same
// number of grid sweeps, so all its lanes reach the shuffles.
constexpr int RADJ_LANES = 4;
__global__ void __launch_bounds__(RT) radon_adj_kernel(const float* __restrict__ S,
                                                       float2* __restrict__ U, int H, int W,
                                                       int n, int D, const float* __restrict__ cs,
                                                       const float* __restrict__ sn, float scale,
                                                       const int* stop) {
    if (stop && *stop) return;   // uniform over the grid
    const float half = 0.5f * (float)(D - 1);
    const size_t N = (size_t)H * W;
    constexpr int PPW = 32 / RADJ_LANES;   // pixels per warp
    const int g = threadIdx.x & (RADJ_LANES - 1), slot = (threadIdx.x & 31) / RADJ_LANES;
    const size_t sweep = (size_t)gridDim.x * (RT / RADJ_LANES);
    for (size_t w0 = (size_t)blockIdx.x * (RT / RADJ_LANES) + (threadIdx.x >> 5) * PPW; w0 < N;
         w0 += sweep) {
        const size_t i = w0 + slot;
        float acc = 0.0f;
        if (i < N) {
            const int r = (int)(i / W), col = (int)(i - (size_t)r * W);
            for (int a = g; a < n; a += RADJ_LANES) {
                const float p = radon_pos(r, col, H, W, cs[a], sn[a], half);
                const float fl = floorf(p);
                const int f = (int)fl;
                const float w = p - fl;
                const float* row = S + (size_t)a * D;
                acc = fmaf(1.0f - w, row[f], acc);
                acc = fmaf(w, row[f + 1], acc);
            }
        }
#pragma unroll
        for (int off = RADJ_LANES / 2; off > 0; off >>= 1)
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (g == 0 && i < N) U[i] = make_float2(scale * acc, 0.0f);
    }
}

// T = b - T over the sinogram.
__global__ void __launch_bounds__(RT) sino_resid_kernel(float* __restrict__ T,
                                                        const float* __restrict__ b, int m) {
    for (int i = blockIdx.x * RT + threadIdx.x; i < m; i += gridDim.x * RT) T[i] = b[i] - T[i];
}

// Each angle's projection convolved with the Ram-Lak kernel h[0] = 1/4,
// h[k] = -1 / (pi k)^2 for odd k, 0 for even k != 0, over the D bins.
__global__ void __launch_bounds__(RT) ramp_filter_kernel(const float* __restrict__ S,
                                                         float* __restrict__ T, int n, int D) {
    const int idx = blockIdx.x * RT + threadIdx.x;
    if (idx >= n * D) return;
    const int a = idx / D, j = idx - a * D;
    const float* row = S + (size_t)a * D;
    const float inv_pi2 = 0.10132118364233778f;   // 1 / pi^2
    float acc = 0.25f * row[j];
    // odd offsets m = j - k: k = j - 1, j - 3, ... and j + 1, j + 3, ...
    for (int k = j - 1; k >= 0; k -= 2) {
        const float m = (float)(j - k);
        acc = fmaf(-inv_pi2 / (m * m), row[k], acc);
    }
    for (int k = j + 1; k < D; k += 2) {
        const float m = (float)(k - j);
        acc = fmaf(-inv_pi2 / (m * m), row[k], acc);
    }
    T[idx] = acc;
}

// *out = sum (T - b)^2 over the sinogram (twice the CT data term).
__global__ void __launch_bounds__(RT) sino_sq_kernel(const float* __restrict__ T,
                                                     const float* __restrict__ b, int m,
                                                     double* partials, unsigned* ticket,
                                                     double* out) {
    double acc = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < m; i += gridDim.x * RT) {
        const double d = (double)T[i] - (double)b[i];
        acc += d * d;
    }
    cta_sum_finish(acc, partials, ticket, out);
}

// ---------------------------------------------------------------------------
// Host side.

// Everything the captured cycle bakes in: the problem, and every buffer it
// reads or writes (the trace buffer included: it is reallocated when a call
// asks for more cycles).
struct ReconKey {
    const void *kspace, *mask, *sino, *u, *trace;
    int op, n_angles, H, W, kind, levels, sides, ncolors, cg_iters, trace_cap;
    float alpha;
    bool operator==(const ReconKey& o) const { return memcmp(this, &o, sizeof(ReconKey)) == 0; }
};

struct ReconWork {
    int H = 0, W = 0;
    FftPlan plan;                 // MRI: the 2-D DFT tables
    float2 *X = nullptr, *Z = nullptr;
    float *c = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    size_t nslots = 0;
    double* partials = nullptr;   // MAX_CTAS
    unsigned* ticket = nullptr;
    double* scal = nullptr;       // 0, 1: rr (alternating); 2: p.q; 3: data term; 4: curvature
    int* stop = nullptr;
    double* epart = nullptr;      // energy kernel partials
    unsigned* eticket = nullptr;
    double* trace = nullptr;
    int* count = nullptr;
    int trace_cap = 0;
    int op = -1, n_angles = 0;    // operator the buffers were made for
    float *S = nullptr, *S2 = nullptr;     // CT: sinogram scratch
    float *cos_t = nullptr, *sin_t = nullptr;
    cudaStream_t cs = nullptr;    // capture stream
    cudaGraphExec_t graph = nullptr;
    ReconKey key{};
};

ReconWork* recon_work_create() { return new ReconWork(); }

static void free_buffers(ReconWork* w) {
    cudaFree(w->X);
    cudaFree(w->Z);
    cudaFree(w->c);
    cudaFree(w->r);
    cudaFree(w->p);
    cudaFree(w->q);
    cudaFree(w->partials);
    cudaFree(w->ticket);
    cudaFree(w->scal);
    cudaFree(w->stop);
    cudaFree(w->epart);
    cudaFree(w->eticket);
    cudaFree(w->S);
    cudaFree(w->S2);
    cudaFree(w->cos_t);
    cudaFree(w->sin_t);
    w->S = w->S2 = w->cos_t = w->sin_t = nullptr;
    w->op = -1;
    w->n_angles = 0;
    w->X = w->Z = nullptr;
    w->c = w->r = w->p = w->q = nullptr;
    w->partials = w->scal = w->epart = nullptr;
    w->ticket = w->eticket = nullptr;
    w->stop = nullptr;
    fft_plan_free(&w->plan);
    w->H = w->W = 0;
}

void recon_work_destroy(ReconWork* w) {
    if (!w) return;
    free_buffers(w);
    cudaFree(w->trace);
    cudaFree(w->count);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->cs) cudaStreamDestroy(w->cs);
    delete w;
}

static int grid_for(size_t n) {
    return (int)std::min<size_t>((n + RT - 1) / RT, RED_CTAS);
}

// The largest slot count of any level of the cycle.
static size_t max_slots(const ReconArgs& a) {
    size_t m = 1;
    for (int j = 0; j < a.levels; ++j) {
        const int b = level_side(j, a.sides);
        const int nbi = (a.H + b - 1) / b, nbj = (a.W + b - 1) / b;
        m = std::max(m, (size_t)active_slots(nbi, nbj, level_colours(a.ncolors, b)));
    }
    return m;
}

#define RC(x)                                                  \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) {                               \
            *msg = cudaGetErrorString(e_);                     \
            return e_ == cudaErrorMemoryAllocation ? 3 : 2;    \
        }                                                      \
    } while (0)

static int ensure_buffers(ReconWork* w, const ReconArgs& a, const char** msg) {
    const size_t need = max_slots(a);
    if (w->H == a.H && w->W == a.W && w->nslots >= need && w->op == a.op &&
        (a.op != RECON_CT || w->n_angles == a.n_angles))
        return 0;
    if (w->graph) cudaGraphExecDestroy(w->graph);   // it points at the old buffers
    w->graph = nullptr;
    free_buffers(w);
    const size_t N = (size_t)a.H * a.W;
    RC(cudaMalloc(&w->X, N * sizeof(float2)));
    RC(cudaMalloc(&w->Z, N * sizeof(float2)));
    RC(cudaMalloc(&w->c, need * sizeof(float)));
    RC(cudaMalloc(&w->r, need * sizeof(float)));
    RC(cudaMalloc(&w->p, need * sizeof(float)));
    RC(cudaMalloc(&w->q, need * sizeof(float)));
    RC(cudaMalloc(&w->partials, MAX_CTAS * sizeof(double)));
    RC(cudaMalloc(&w->ticket, sizeof(unsigned)));
    RC(cudaMemset(w->ticket, 0, sizeof(unsigned)));
    RC(cudaMalloc(&w->scal, 8 * sizeof(double)));
    RC(cudaMemset(w->scal, 0, 8 * sizeof(double)));
    RC(cudaMalloc(&w->stop, sizeof(int)));
    RC(cudaMalloc(&w->epart, energy_partials_needed(a.H, a.W) * sizeof(double)));
    RC(cudaMalloc(&w->eticket, sizeof(unsigned)));
    RC(cudaMemset(w->eticket, 0, sizeof(unsigned)));
    w->nslots = need;
    if (a.op == RECON_MRI) {
        const int frc = fft_plan_make(&w->plan, a.H, a.W);
        if (frc != 0) {
            *msg = frc == 1 ? "image size beyond the transform's limits" : "FFT tables failed";
            return frc == 3 ? 3 : 2;
        }
    } else {
        const size_t m = (size_t)a.n_angles * radon_bins(a.H, a.W);
        RC(cudaMalloc(&w->S, m * sizeof(float)));
        RC(cudaMalloc(&w->S2, m * sizeof(float)));
        RC(cudaMalloc(&w->cos_t, a.n_angles * sizeof(float)));
        RC(cudaMalloc(&w->sin_t, a.n_angles * sizeof(float)));
        std::vector<float> ch(a.n_angles), sh(a.n_angles);
        for (int i = 0; i < a.n_angles; ++i) {
            const double th = 3.14159265358979323846 * i / a.n_angles;
            ch[i] = (float)cos(th);
            sh[i] = (float)sin(th);
        }
        RC(cudaMemcpy(w->cos_t, ch.data(), a.n_angles * sizeof(float), cudaMemcpyHostToDevice));
        RC(cudaMemcpy(w->sin_t, sh.data(), a.n_angles * sizeof(float), cudaMemcpyHostToDevice));
        w->n_angles = a.n_angles;
    }
    w->op = a.op;
    w->H = a.H;
    w->W = a.W;
    return 0;
}

enum { FFT_FORWARD = 0, FFT_INVERSE = 1 };

static cudaError_t fft(ReconWork* w, float2* X, int dir, cudaStream_t st) {
    return fft2d(w->plan, X, dir == FFT_INVERSE, st);
}

int radon_bins(int H, int W) {
    return 2 * (int)ceil(0.5 * hypot((double)(H - 1), (double)(W - 1))) + 3;
}

// CT: S <- R U (U's real parts), optionally stopped by the CG flag.
static cudaError_t ct_forward(ReconWork* w, const ReconArgs& a, const float2* U, float* S,
                              const int* stop, cudaStream_t st) {
    const int D = radon_bins(a.H, a.W), m = a.n_angles * D;
    const long long nt = (long long)m * RADON_LANES;
    radon_fwd_kernel<<<(unsigned)((nt + RT - 1) / RT), RT, 0, st>>>(U, S, a.H, a.W, a.n_angles, D,
                                                                    w->cos_t, w->sin_t, stop);
    return cudaGetLastError();
}

// CT: U <- scale R^T S.
static cudaError_t ct_adjoint(ReconWork* w, const ReconArgs& a, const float* S, float2* U,
                              float scale, const int* stop, cudaStream_t st) {
    radon_adj_kernel<<<grid_for((size_t)a.H * a.W * RADJ_LANES), RT, 0, st>>>(
        S, U, a.H, a.W, a.n_angles, radon_bins(a.H, a.W), w->cos_t, w->sin_t, scale, stop);
    return cudaGetLastError();
}

template <int GS, int MODE>
static cudaError_t launch_gather(ReconWork* w, const ReconArgs& a, int b, int nc, int k,
                                 int nslots, float* out, cudaStream_t st) {
    const int grid = (nslots + RT / GS - 1) / (RT / GS);
    if (grid > MAX_CTAS) return cudaErrorInvalidValue;
    auto kern = a.kind == KIND_MEAN         ? gather_kernel<GS, MODE, KIND_MEAN>
                : a.kind == KIND_GAUSS      ? gather_kernel<GS, MODE, KIND_GAUSS>
                : a.kind == KIND_MEAN_EULER ? gather_kernel<GS, MODE, KIND_MEAN_EULER>
                                            : gather_kernel<GS, MODE, KIND_GAUSS_EULER>;
    const float2* Y = MODE == GATHER_RHS ? w->X : w->Z;
    kern<<<grid, RT, 0, st>>>(Y, a.u, a.H, a.W, b, nc, k, nslots, 2.0f * a.alpha, out, w->p, w->c,
                              w->stop, w->partials, w->ticket,
                              MODE == GATHER_RHS ? w->scal + 0 : w->scal + 2);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t gather(ReconWork* w, const ReconArgs& a, int b, int nc, int k, int nslots,
                          float* out, cudaStream_t st) {
    if (b <= 2) return launch_gather<1, MODE>(w, a, b, nc, k, nslots, out, st);
    if (b <= 16) return launch_gather<32, MODE>(w, a, b, nc, k, nslots, out, st);
    return launch_gather<RT, MODE>(w, a, b, nc, k, nslots, out, st);
}

// J(u) into the trace (on the device).
static cudaError_t enqueue_objective(ReconWork* w, const ReconArgs& a, cudaStream_t st) {
    const size_t N = (size_t)a.H * a.W;
    const float s = 1.0f / sqrtf((float)N);
    const int gN = grid_for(N);
    cudaError_t e;
    to_complex_kernel<<<gN, RT, 0, st>>>(a.u, w->X, N);
    if (a.op == RECON_MRI) {
        if ((e = fft(w, w->X, FFT_FORWARD, st)) != cudaSuccess) return e;
        data_term_kernel<<<gN, RT, 0, st>>>(w->X, a.kspace, a.mask, N, s, w->partials, w->ticket,
                                            w->scal + 3);
    } else {
        if ((e = ct_forward(w, a, w->X, w->S, nullptr, st)) != cudaSuccess) return e;
        const int m = a.n_angles * radon_bins(a.H, a.W);
        sino_sq_kernel<<<grid_for((size_t)m), RT, 0, st>>>(w->S, a.sino, m, w->partials,
                                                           w->ticket, w->scal + 3);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // sum |kappa(u)|: the energy with f = u has no fidelity part
    if ((e = launch_energy(a.u, a.u, a.H, a.W, 1.0f, a.kind, w->epart, w->eticket, w->scal + 4,
                           st)) != cudaSuccess)
        return e;
    objective_kernel<<<1, 32, 0, st>>>(w->scal + 3, w->scal + 4, a.alpha, w->trace, w->count,
                                       w->trace_cap);
    return cudaGetLastError();
}

// One cycle: every level, every colour: right-hand side, CG, apply.
static cudaError_t enqueue_cycle(ReconWork* w, const ReconArgs& a, cudaStream_t st) {
    const size_t N = (size_t)a.H * a.W;
    const float s = 1.0f / sqrtf((float)N);
    const float s2 = 1.0f / (float)N;
    const int gN = grid_for(N);
    cudaError_t e;
    for (int j = 0; j < a.levels; ++j) {
        const int b = level_side(j, a.sides);
        const int nc = level_colours(a.ncolors, b);
        const int nbi = (a.H + b - 1) / b, nbj = (a.W + b - 1) / b;
        const int nslots = active_slots(nbi, nbj, nc);
        const int gs = grid_for((size_t)nslots);
        for (int k = 0; k < nc; ++k) {
            // right-hand side: Re <b - A u, A phi_i> + 2 alpha d_i
            to_complex_kernel<<<gN, RT, 0, st>>>(a.u, w->X, N);
            if (a.op == RECON_MRI) {
                if ((e = fft(w, w->X, FFT_FORWARD, st)) != cudaSuccess) return e;
                resid_kernel<<<gN, RT, 0, st>>>(w->X, a.kspace, a.mask, N, s);
                if ((e = fft(w, w->X, FFT_INVERSE, st)) != cudaSuccess) return e;
            } else {
                if ((e = ct_forward(w, a, w->X, w->S, nullptr, st)) != cudaSuccess) return e;
                const int m = a.n_angles * radon_bins(a.H, a.W);
                sino_resid_kernel<<<grid_for((size_t)m), RT, 0, st>>>(w->S, a.sino, m);
                if ((e = ct_adjoint(w, a, w->S, w->X, 1.0f, nullptr, st)) != cudaSuccess) return e;
            }
            if ((e = gather<GATHER_RHS>(w, a, b, nc, k, nslots, w->r, st)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(w->stop, 0, sizeof(int), st)) != cudaSuccess) return e;
            for (int it = 0; it < a.cg_iters; ++it) {
                double* rr = w->scal + (it & 1);
                double* rr_next = w->scal + ((it + 1) & 1);
                scatter_kernel<<<gN, RT, 0, st>>>(w->p, w->Z, a.H, a.W, b, nc, k, rr, w->stop);
                if (a.op == RECON_MRI) {
                    // M Z s2 in the forward transform's last store (N > 1);
                    // with the CG stopped its result is not read
                    if (N > 1) {
                        if ((e = fft2d(w->plan, w->Z, false, st, a.mask, s2)) != cudaSuccess)
                            return e;
                    } else {
                        if ((e = fft(w, w->Z, FFT_FORWARD, st)) != cudaSuccess) return e;
                        mask_scale_kernel<<<gN, RT, 0, st>>>(w->Z, a.mask, N, s2, w->stop);
                    }
                    if ((e = fft(w, w->Z, FFT_INVERSE, st)) != cudaSuccess) return e;
                } else {
                    if ((e = ct_forward(w, a, w->Z, w->S, w->stop, st)) != cudaSuccess) return e;
                    if ((e = ct_adjoint(w, a, w->S, w->Z, 1.0f, w->stop, st)) != cudaSuccess)
                        return e;
                }
                if ((e = gather<GATHER_Q>(w, a, b, nc, k, nslots, w->q, st)) != cudaSuccess)
                    return e;
                cg_update_kernel<<<gs, RT, 0, st>>>(w->c, w->r, w->p, w->q, nslots, rr,
                                                    w->scal + 2, w->stop, w->partials, w->ticket,
                                                    rr_next);
                cg_dir_kernel<<<gs, RT, 0, st>>>(w->p, w->r, nslots, rr, rr_next, w->stop);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            apply_blocks_kernel<<<gN, RT, 0, st>>>(a.u, w->c, a.H, a.W, b, nc, k);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return enqueue_objective(w, a, st);
}

int recon_run(ReconWork* w, const ReconArgs& a, cudaStream_t st, const char** msg) {
    *msg = "";
    if (a.op == RECON_MRI && (!fft_length_ok(a.H) || !fft_length_ok(a.W))) {
        *msg = "image size beyond the transform's limits";
        return 1;
    }
    int rc = ensure_buffers(w, a, msg);
    if (rc) return rc;
    if (w->trace_cap < a.cycles + 1) {
        if (w->graph) cudaGraphExecDestroy(w->graph);   // it points at the old trace
        w->graph = nullptr;
        cudaFree(w->trace);
        w->trace = nullptr;
        RC(cudaMalloc(&w->trace, (size_t)(a.cycles + 1) * sizeof(double)));
        w->trace_cap = a.cycles + 1;
    }
    if (!w->count) RC(cudaMalloc(&w->count, sizeof(int)));
    if (!w->cs) RC(cudaStreamCreateWithFlags(&w->cs, cudaStreamNonBlocking));
    const size_t N = (size_t)a.H * a.W;
    const float s = 1.0f / sqrtf((float)N);
    RC(cudaMemsetAsync(w->count, 0, sizeof(int), st));
    if (a.u0) {
        if (a.u0 != a.u)
            RC(cudaMemcpyAsync(a.u, a.u0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    } else if (a.op == RECON_MRI) {   // zero-filled start Re(A^H b)
        masked_data_kernel<<<grid_for(N), RT, 0, st>>>(w->X, a.kspace, a.mask, N, s);
        RC(fft(w, w->X, FFT_INVERSE, st));
        real_part_kernel<<<grid_for(N), RT, 0, st>>>(w->X, a.u, N);
        RC(cudaGetLastError());
    } else {   // filtered backprojection (pi / n) R^T (h * b)
        const int D = radon_bins(a.H, a.W), m = a.n_angles * D;
        ramp_filter_kernel<<<(m + RT - 1) / RT, RT, 0, st>>>(a.sino, w->S2, a.n_angles, D);
        RC(cudaGetLastError());
        RC(ct_adjoint(w, a, w->S2, w->X, 3.14159265358979323846f / (float)a.n_angles, nullptr,
                      st));
        real_part_kernel<<<grid_for(N), RT, 0, st>>>(w->X, a.u, N);
        RC(cudaGetLastError());
    }
    RC(enqueue_objective(w, a, st));
    // one cycle as a graph, captured once per problem and reused
    ReconKey key;
    memset(&key, 0, sizeof key);   // padding included: the key is compared bytewise
    key.op = a.op;
    key.kspace = a.kspace;
    key.mask = a.mask;
    key.sino = a.sino;
    key.n_angles = a.n_angles;
    key.u = a.u;
    key.trace = w->trace;
    key.H = a.H;
    key.W = a.W;
    key.kind = a.kind;
    key.levels = a.levels;
    key.sides = a.sides;
    key.ncolors = a.ncolors;
    key.cg_iters = a.cg_iters;
    key.trace_cap = w->trace_cap;
    key.alpha = a.alpha;
    if (a.cycles > 0 && !(w->graph && w->key == key)) {
        if (w->graph) cudaGraphExecDestroy(w->graph);
        w->graph = nullptr;
        RC(cudaStreamBeginCapture(w->cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = enqueue_cycle(w, a, w->cs);
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(w->cs, &g);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            *msg = cudaGetErrorString(ce != cudaSuccess ? ce : ee);
            return 2;
        }
        cudaError_t ie = cudaGraphInstantiate(&w->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            w->graph = nullptr;
            *msg = cudaGetErrorString(ie);
            return 2;
        }
        w->key = key;
    }
    for (int l = 0; l < a.cycles; ++l) RC(cudaGraphLaunch(w->graph, st));
    if (a.trace_host)
        RC(cudaMemcpyAsync(a.trace_host, w->trace, (size_t)(a.cycles + 1) * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
    RC(cudaStreamSynchronize(st));
    return 0;
}

// The operator pair alone, on temporaries (a ReconWork of its own).
static int radon_apply(const float* in, int H, int W, int n_angles, float* out, bool adjoint,
                       cudaStream_t st, const char** msg) {
    *msg = "";
    ReconWork w;
    ReconArgs a;
    a.op = RECON_CT;
    a.kspace = nullptr;
    a.mask = nullptr;
    a.sino = nullptr;
    a.n_angles = n_angles;
    a.H = H;
    a.W = W;
    a.levels = 1;
    a.sides = 0;
    a.ncolors = 4;
    int rc = ensure_buffers(&w, a, msg);
    const size_t N = (size_t)H * W;
    cudaError_t e = cudaSuccess;
    if (rc == 0) {
        if (!adjoint) {
            to_complex_kernel<<<grid_for(N), RT, 0, st>>>(in, w.X, N);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = ct_forward(&w, a, w.X, out, nullptr, st);
        } else {
            e = ct_adjoint(&w, a, in, w.X, 1.0f, nullptr, st);
            if (e == cudaSuccess) {
                real_part_kernel<<<grid_for(N), RT, 0, st>>>(w.X, out, N);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            *msg = cudaGetErrorString(e);
            rc = 2;
        }
    }
    free_buffers(&w);
    return rc;
}

int radon_forward(const float* u, int H, int W, int n_angles, float* sino, cudaStream_t st,
                  const char** msg) {
    return radon_apply(u, H, W, n_angles, sino, false, st, msg);
}

int radon_adjoint(const float* sino, int n_angles, int H, int W, float* u, cudaStream_t st,
                  const char** msg) {
    return radon_apply(sino, H, W, n_angles, u, true, st, msg);
}

}  // namespace cm
