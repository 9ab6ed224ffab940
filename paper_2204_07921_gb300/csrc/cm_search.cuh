// cm_search.cuh -- the block search and block geometry shared by the phase
// kernels.
//
// Block search (the 1-D subproblem of Alg. 3, min_c F(u + c phi_A)):
//   c_fid = -S1/s; E_A(c) = alpha s/2 (c - c_fid)^2 + sum_ring |kappa(c)| (up to
//   a constant); bracket rho = sqrt(2 sum_ring|kappa(c_fid)| / (alpha s)); E_A at
//   G equispaced points of [c_fid - rho, c_fid + rho]; K golden-section
//   evaluations on [g* - D, g* + D]; also c = 0 and (finest level) the
//   paper's one-step estimate; the best evaluated c wins (ties: smaller |c|,
//   then smaller c).
#pragma once
#include "cm_device.cuh"

namespace cm {

struct SearchParams {
    float alpha;
    int G;   // grid points (odd)
    int K;   // golden-section evaluations
};

// ring(c) returns the group-uniform sum over the block's ring.  The
// fidelity part is carried as alpha s/2 (c - c_fid)^2, which differs from the
// expanded alpha/2 (s c^2 + 2 c S1) by the constant alpha s c_fid^2 / 2, so it
// selects the same c without the FP32 cancellation of the expanded form.
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

// The same search written with a single call site of ring(): each iteration
// picks the next candidate from the search state, evaluates it and updates
// the state.  It visits the same candidates in the same order and takes the
// same decisions as block_search, so the selected c is identical; the ring
// evaluation is inlined once, which keeps large ring bodies out of the
// instruction cache's way.
template <class Ring>
__device__ __forceinline__ float block_search_1site(Ring&& ring, const SearchParams& p, float s,
                                                    float S1, bool has_paper, float c_paper) {
    const float c_fid = -S1 / s;
    const float half_as = 0.5f * p.alpha * s;
    const int mid = (p.G - 1) / 2;
    // evaluation order: 0, [paper], c_fid, grid i != mid, x1, x2, golden steps
    const int n_pre = has_paper ? 3 : 2;
    const int n_grid = p.G - 1;
    const int n_eval = n_pre + n_grid + p.K;
    Best best;
    best.c = 0.0f;
    best.E = INFINITY;
    float Rk = 0.0f, rho = 0.0f;
    float gbest = c_fid, Egbest = INFINITY;
    float lo = 0.0f, hi = 0.0f, x1 = 0.0f, x2 = 0.0f, E1 = 0.0f, E2 = 0.0f;
    bool left = false;
    for (int e = 0; e < n_eval; ++e) {
        // --- next candidate
        float c;
        int gi = 0;   // grid index for grid evaluations
        if (e == 0) {
            c = 0.0f;
        } else if (has_paper && e == 1) {
            c = c_paper;
        } else if (e == n_pre - 1) {
            c = c_fid;
        } else if (e < n_pre + n_grid) {
            gi = e - n_pre;
            gi += (gi >= mid) ? 1 : 0;
            float t = (2.0f * (float)gi) / (float)(p.G - 1) - 1.0f;
            c = c_fid + rho * t;
        } else if (e == n_pre + n_grid) {
            const float D = 2.0f * rho / (float)(p.G - 1);
            lo = gbest - D;
            hi = gbest + D;
            x1 = hi - GOLDEN * (hi - lo);
            x2 = lo + GOLDEN * (hi - lo);
            c = x1;
        } else if (e == n_pre + n_grid + 1) {
            c = x2;
        } else {
            left = E1 < E2;
            if (left) {
                hi = x2;
                x2 = x1;
                E2 = E1;
                c = hi - GOLDEN * (hi - lo);
            } else {
                lo = x1;
                x1 = x2;
                E1 = E2;
                c = lo + GOLDEN * (hi - lo);
            }
        }
        // --- evaluate
        const float rk = ring(c);
        const float t = c - c_fid;
        const float E = fmaf(half_as * t, t, rk);
        // --- update
        if (e == 0) {
            best.c = 0.0f;
            best.E = E;
        } else {
            consider(best, c, E);
        }
        if (e == n_pre - 1) {
            Rk = rk;
            rho = sqrtf(2.0f * Rk / (p.alpha * s));
            // the middle grid point is c_fid itself
            Egbest = E;
            gbest = c_fid;
            // grid points below the middle must be able to win a tie-free "<":
            // evaluate them in index order below; c_fid keeps index mid.
        } else if (e >= n_pre && e < n_pre + n_grid) {
            (void)gi;
        } else if (e == n_pre + n_grid) {
            E1 = E;
        } else if (e == n_pre + n_grid + 1) {
            E2 = E;
        } else if (e > n_pre + n_grid + 1) {
            if (left) {
                x1 = c;
                E1 = E;
            } else {
                x2 = c;
                E2 = E;
            }
        }
        if (e >= n_pre && e < n_pre + n_grid) {
            // grid bookkeeping in index order: the sequential search scans
            // i = 0..G-1 with a strict "<", so the first minimum wins.  Here
            // index mid was seen first; a lower index with an equal energy
            // must still win, a higher index must not.
            if (E < Egbest || (E == Egbest && gi < mid && gbest == c_fid)) {
                Egbest = E;
                gbest = c;
            }
        }
    }
    return best.c;
}

// The same search for groups whose reductions each cost a barrier: ringv(cs,
// m, out) evaluates m <= MB candidates in one reduction.  ring(0) and
// ring(c_fid) share one reduction and the grid points share one (the middle
// point reuses ring(c_fid)); the golden section stays sequential.  Every
// value is computed as in block_search, so the selected c is identical.
template <int MB, class RingV>
__device__ __forceinline__ float block_search_batched(RingV&& ringv, const SearchParams& p,
                                                      float s, float S1) {
    const float c_fid = -S1 / s;
    const float half_as = 0.5f * p.alpha * s;
    auto energy = [&](float c, float rk) {
        float t = c - c_fid;
        return fmaf(half_as * t, t, rk);
    };
    float cs[MB], rk[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) cs[j] = 0.0f;
    cs[1] = c_fid;
    ringv(cs, 2, rk);
    Best best;
    best.c = 0.0f;
    best.E = energy(0.0f, rk[0]);
    const float Rk = rk[1];
    const float rho = sqrtf(2.0f * Rk / (p.alpha * s));
    const int mid = (p.G - 1) / 2;
    float gbest = c_fid, Egbest = INFINITY;
    for (int i0 = 0; i0 < p.G; i0 += MB) {
        const int m = min(MB, p.G - i0);
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            float t = (2.0f * (float)(i0 + j)) / (float)(p.G - 1) - 1.0f;
            cs[j] = c_fid + rho * t;
        }
        ringv(cs, m, rk);
#pragma unroll
        for (int j = 0; j < MB; ++j)
            if (j < m) {
                float E = energy(cs[j], (i0 + j == mid) ? Rk : rk[j]);
                consider(best, cs[j], E);
                if (E < Egbest) {
                    Egbest = E;
                    gbest = cs[j];
                }
            }
    }
    const float D = 2.0f * rho / (float)(p.G - 1);
    float lo = gbest - D, hi = gbest + D;
    float x1 = hi - GOLDEN * (hi - lo), x2 = lo + GOLDEN * (hi - lo);
    cs[0] = x1;
    cs[1] = x2;
    ringv(cs, 2, rk);
    float E1 = energy(x1, rk[0]);
    consider(best, x1, E1);
    float E2 = energy(x2, rk[1]);
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
        cs[0] = xn;
        ringv(cs, 1, rk);
        const float En = energy(xn, rk[0]);
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

// ---------------------------------------------------------------------------
// Block geometry.

// Active block number a of colour k -> (bi, bj); false if a is past the end.
__device__ __forceinline__ bool active_block(int a, int nbi, int nbj, int ncol, int k, int& bi,
                                             int& bj) {
    int nact;
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
    return a < nact && bi < nbi && bj < nbj;
}

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

// Ring slot j of block [r0, r1) x [c0, c1): the outer frame (one pixel
// outside the block, clipped to the image) then the inner frame (the block's
// boundary pixels, less those whose clamped 3x3 stencil lies in the block).
// Returns false when the slot holds no ring pixel; else loads the pixel's
// clamped window from the phase state and the mask of window entries that
// lie in the block.
__device__ __forceinline__ bool ring_slot(int j, int r0, int r1, int c0, int c1, int H, int W,
                                          const float* __restrict__ S,
                                          const float* __restrict__ R, int lb, int ncol, int k,
                                          float w[9], unsigned& mask) {
    const int bh = r1 - r0, bw = c1 - c0;
    const int Pout = perim_count(bh + 2, bw + 2);
    const int Pin = perim_count(bh, bw);
    if (j >= Pout + Pin) return false;
    int li, lj, rr, cc;
    if (j < Pout) {
        perim_pos(j, bh + 2, bw + 2, li, lj);
        rr = r0 - 1 + li;
        cc = c0 - 1 + lj;
        if (rr < 0 || rr >= H || cc < 0 || cc >= W) return false;
    } else {
        perim_pos(j - Pout, bh, bw, li, lj);
        rr = r0 + li;
        cc = c0 + lj;
        bool interior = (rr - 1 >= r0 || rr == 0) && (rr + 1 < r1 || rr == H - 1) &&
                        (cc - 1 >= c0 || cc == 0) && (cc + 1 < c1 || cc == W - 1);
        if (interior) return false;
    }
    mask = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            int qr = clampi(rr + a - 1, 0, H - 1), qc = clampi(cc + b - 1, 0, W - 1);
            w[3 * a + b] = phase_read(S, R, qr, qc, W, lb, ncol, k);
            bool inA = qr >= r0 && qr < r1 && qc >= c0 && qc < c1;
            mask |= (inA ? 1u : 0u) << (3 * a + b);
        }
    return true;
}

}  // namespace cm
