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
    int G;          // grid points (odd)
    int K;          // golden-section evaluations
    int spec = 1;       // block_search_rounds: speculate the first golden pair
    int dmax = 4;       // block_search_rounds: golden steps per round (1..4)
    int one_step = 0;   // 1: the paper's single step instead of the search
};

// One step of Alg. 2 from c_0 = 0 (t = 0, eta = 1) on a block with c_1/2 = 0:
// c_1 = alpha f* / (2 + alpha), f* = c_fid the block mean of f - u (the
// finest level uses the plane-distance estimate for c_1/2 instead).
__device__ __forceinline__ float fbs_step(const SearchParams& p, float s, float S1) {
    const float c_fid = -S1 / s;
    return p.alpha * c_fid / (2.0f + p.alpha);
}

// The single-step mode: the block keeps c1 if it lowers E_A, else 0 (two
// evaluations; the tie rule of the search).
template <class Ring>
__device__ __forceinline__ float block_search_onestep(Ring&& ring, const SearchParams& p, float s,
                                                      float S1, float c1) {
    const float c_fid = -S1 / s;
    const float half_as = 0.5f * p.alpha * s;
    auto energy = [&](float c, float rk) {
        const float t = c - c_fid;
        return fmaf(half_as * t, t, rk);
    };
    Best best;
    best.c = 0.0f;
    best.E = energy(0.0f, ring(0.0f));
    consider(best, c1, energy(c1, ring(c1)));
    return best.c;
}

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
    if (p.one_step) {
        cs[1] = fbs_step(p, s, S1);
        ringv(cs, 2, rk);
        Best b1;
        b1.c = 0.0f;
        b1.E = energy(0.0f, rk[0]);
        consider(b1, cs[1], energy(cs[1], rk[1]));
        return b1.c;
    }
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

// Golden-section state of the round-based search below.
struct GoldenState {
    float lo, hi, x1, x2, E1, E2;
};

// One golden step from a state whose comparison is decided by `left`;
// returns the new point (its energy goes in with golden_put).
__device__ __forceinline__ float golden_take(GoldenState& st, bool left) {
    if (left) {
        st.hi = st.x2;
        st.x2 = st.x1;
        st.E2 = st.E1;
        return st.hi - GOLDEN * (st.hi - st.lo);
    }
    st.lo = st.x1;
    st.x1 = st.x2;
    st.E1 = st.E2;
    return st.lo + GOLDEN * (st.hi - st.lo);
}

__device__ __forceinline__ void golden_put(GoldenState& st, bool left, float x, float E) {
    if (left) {
        st.x1 = x;
        st.E1 = E;
    } else {
        st.x2 = x;
        st.E2 = E;
    }
}

// ---------------------------------------------------------------------------
// Search in rounds, for groups in which every warp holds the same search state
// (one CTA or one cluster per block, all threads taking part).  A round
// evaluates up to 16 candidates with one reduction: lane j of each warp
// generates candidate j as `mine`, and round(mine, m) returns in lane l the
// ring sum of candidate l / 2.
//   the first round: c = 0 and c_fid;
//   the second: the grid points other than c_fid and, when they fit, the
//            first golden pair of every grid point that may win (else the grid in
//            chunks of 16 and the pair in a round of its own);
//   then golden rounds of up to dmax <= 4 steps, which evaluate the
//   2^dmax - 1 points of every outcome path of the next dmax comparisons.
// Only points on the path taken are considered, each computed by the formula
// of block_search, so the candidates and the decisions are those of
// block_search.  With speculation and dmax = 4 the reductions of G = 5,
// K = 6 drop from 7 (one per step) to 3 at 31 instead of 12 evaluations; the
// kernel picks the trade per level.

__device__ __forceinline__ float grid_t(int i, int G) {
    return (2.0f * (float)i) / (float)(G - 1) - 1.0f;
}

__device__ __forceinline__ float grid_point(float c_fid, float rho, int i, int G) {
    return __fmaf_rn(rho, grid_t(i, G), c_fid);
}

// Point of node n (heap order: node 1 is the next point, nodes 2n / 2n + 1
// follow it when the comparison after it goes left / right) of the golden
// tree grown from st, whose next comparison is known.
__device__ __forceinline__ float golden_tree_point(GoldenState st, int n) {
    const int depth = 31 - __clz(n);
    bool left = st.E1 < st.E2;
    float x = golden_take(st, left);
    for (int q = depth - 1; q >= 0; --q) {
        golden_put(st, left, x, 0.0f);
        left = ((n >> q) & 1) == 0;
        x = golden_take(st, left);
    }
    return x;
}

template <class RoundFn>
__device__ __forceinline__ float block_search_rounds(RoundFn&& round, const SearchParams& p,
                                                     float s, float S1) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float c_fid = -S1 / s;
    const float half_as = 0.5f * p.alpha * s;
    auto energy = [&](float c, float rk) {
        const float t = c - c_fid;
        return fmaf(half_as * t, t, rk);
    };
    const int mid = (p.G - 1) / 2;
    const int ng = p.G - 1;                    // grid points other than c_fid
    const bool spec = p.spec && ng + 2 * p.G <= 16;
    if (p.one_step) {
        const float c1 = fbs_step(p, s, S1);
        const float t1 = round(lane == 1 ? c1 : 0.0f, 2);
        Best b1;
        b1.c = 0.0f;
        b1.E = energy(0.0f, __shfl_sync(FULL, t1, 0));
        consider(b1, c1, energy(c1, __shfl_sync(FULL, t1, 2)));
        return b1.c;
    }
    // the first round: c = 0, c_fid
    float mine = lane == 1 ? c_fid : 0.0f;
    float tot = round(mine, 2);
    Best best;
    best.c = 0.0f;
    best.E = energy(0.0f, __shfl_sync(FULL, tot, 0));
    const float Rk = __shfl_sync(FULL, tot, 2);
    const float rho = sqrtf(2.0f * Rk / (p.alpha * s));
    const float D = 2.0f * rho / (float)(p.G - 1);
    // grid (+ speculative first pairs)
    float gbest = c_fid, Egbest = INFINITY;
    int gwin = mid;
    int mg = 0;
    for (int g0 = 0; g0 < ng; g0 += 16) {
        mg = min(ng - g0, 16);
        const int m = mg + (spec ? 2 * p.G : 0);
        mine = 0.0f;
        if (lane < mg) {
            const int gi = g0 + lane + ((g0 + lane >= mid) ? 1 : 0);
            mine = grid_point(c_fid, rho, gi, p.G);
        } else if (spec && lane < m) {
            const int q = lane - mg;
            const float g = grid_point(c_fid, rho, q >> 1, p.G);
            const float lo = g - D, hi = g + D;
            mine = (q & 1) ? lo + GOLDEN * (hi - lo) : hi - GOLDEN * (hi - lo);
        }
        tot = round(mine, m);
        for (int j = 0; j < mg; ++j) {
            const int k = g0 + j;
            if (k == mid) {   // c_fid, the middle grid point, in index order
                const float cm = grid_point(c_fid, rho, mid, p.G);
                const float Em = energy(cm, Rk);
                consider(best, cm, Em);
                if (Em < Egbest) {
                    Egbest = Em;
                    gbest = cm;
                    gwin = mid;
                }
            }
            const float c = __shfl_sync(FULL, mine, j);
            const float E = energy(c, __shfl_sync(FULL, tot, 2 * j));
            consider(best, c, E);
            if (E < Egbest) {
                Egbest = E;
                gbest = c;
                gwin = k + (k >= mid ? 1 : 0);
            }
        }
    }
    // first golden pair
    GoldenState st;
    st.lo = gbest - D;
    st.hi = gbest + D;
    if (spec) {
        const int i1 = mg + 2 * gwin;
        st.x1 = __shfl_sync(FULL, mine, i1);
        st.x2 = __shfl_sync(FULL, mine, i1 + 1);
        st.E1 = energy(st.x1, __shfl_sync(FULL, tot, 2 * i1));
        st.E2 = energy(st.x2, __shfl_sync(FULL, tot, 2 * i1 + 2));
    } else {
        st.x1 = st.hi - GOLDEN * (st.hi - st.lo);
        st.x2 = st.lo + GOLDEN * (st.hi - st.lo);
        mine = lane == 0 ? st.x1 : (lane == 1 ? st.x2 : 0.0f);
        tot = round(mine, 2);
        st.E1 = energy(st.x1, __shfl_sync(FULL, tot, 0));
        st.E2 = energy(st.x2, __shfl_sync(FULL, tot, 2));
    }
    consider(best, st.x1, st.E1);
    consider(best, st.x2, st.E2);
    // golden rounds
    for (int steps = p.K - 2; steps > 0;) {
        const int d = min(steps, p.dmax);
        const int m = (1 << d) - 1;
        mine = lane < m ? golden_tree_point(st, lane + 1) : 0.0f;
        tot = round(mine, m);
        int n = 1;
        for (int q = 0; q < d; ++q) {
            const bool left = st.E1 < st.E2;
            golden_take(st, left);
            const float x = __shfl_sync(FULL, mine, n - 1);
            const float E = energy(x, __shfl_sync(FULL, tot, 2 * (n - 1)));
            consider(best, x, E);
            golden_put(st, left, x, E);
            n = 2 * n + (st.E1 < st.E2 ? 0 : 1);
        }
        steps -= d;
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
        const int p = colour_side(ncol);
        const int kr = k / p, kc = k - kr * p;
        const int hj = (nbj + p - 1) / p, hi = (nbi + p - 1) / p;
        const int ai = a / hj;
        bi = p * ai + kr;
        bj = p * (a - ai * hj) + kc;
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
// clamped window through value(r, c) (the phase state) and the mask of window
// entries that lie in the block.
template <class Value>
__device__ __forceinline__ bool ring_slot_v(int j, int r0, int r1, int c0, int c1, int H, int W,
                                            Value&& value, float w[9], unsigned& mask) {
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
            w[3 * a + b] = value(qr, qc);
            bool inA = qr >= r0 && qr < r1 && qc >= c0 && qc < c1;
            mask |= (inA ? 1u : 0u) << (3 * a + b);
        }
    return true;
}

// Ring slot j read from the phase state; the level's block side is 1 << lb
// (POW2) or b.
template <bool POW2 = true>
__device__ __forceinline__ bool ring_slot(int j, int r0, int r1, int c0, int c1, int H, int W,
                                          const float* __restrict__ S,
                                          const float* __restrict__ R, int lb, int ncol, int k,
                                          float w[9], unsigned& mask, int b = 0) {
    return ring_slot_v(j, r0, r1, c0, c1, H, W,
                       [&](int r, int c) {
                           return phase_read_b<POW2>(S, R, r, c, W, lb, b, ncol, k);
                       },
                       w, mask);
}

}  // namespace cm
