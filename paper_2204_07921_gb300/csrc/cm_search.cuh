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

// The batched search with the golden section advanced LA = 3 steps per
// reduction.  From a state whose next comparison is known the next point is
// fixed; the point after it depends on one unknown comparison (2 choices),
// the one after that on two (4 choices): 7 points cover every path of 3
// steps.  Only the points on the path actually taken are considered, and
// each is computed by the same operations as in block_search, so the
// selected c is identical; the extra evaluations trade idle threads for
// fewer barriers on levels with few blocks.
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

template <int MB, class RingV>
__device__ __forceinline__ float block_search_lookahead(RingV&& ringv, const SearchParams& p,
                                                        float s, float S1) {
    static_assert(MB >= 7, "a depth-3 lookahead needs 7 candidates per batch");
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
    GoldenState st;
    st.lo = gbest - D;
    st.hi = gbest + D;
    st.x1 = st.hi - GOLDEN * (st.hi - st.lo);
    st.x2 = st.lo + GOLDEN * (st.hi - st.lo);
    cs[0] = st.x1;
    cs[1] = st.x2;
    ringv(cs, 2, rk);
    st.E1 = energy(st.x1, rk[0]);
    consider(best, st.x1, st.E1);
    st.E2 = energy(st.x2, rk[1]);
    consider(best, st.x2, st.E2);
    int steps = p.K - 2;
    while (steps > 0) {
        const int la = steps >= 3 ? 3 : steps;
        // step 1 (decision known)
        const bool l0 = st.E1 < st.E2;
        GoldenState s0 = st;
        const float p0 = golden_take(s0, l0);
        cs[0] = p0;
        int m = 1;
        // step 2 after each outcome o1 of the next comparison (0 = left)
        float p1[2], p2[4];
        GoldenState s1[2];
#pragma unroll
        for (int o1 = 0; o1 < 2; ++o1) {
            s1[o1] = s0;
            golden_put(s1[o1], l0, p0, 0.0f);
            p1[o1] = golden_take(s1[o1], o1 == 0);
#pragma unroll
            for (int o2 = 0; o2 < 2; ++o2) {
                GoldenState s2 = s1[o1];
                golden_put(s2, o1 == 0, p1[o1], 0.0f);
                p2[2 * o1 + o2] = golden_take(s2, o2 == 0);
            }
        }
        if (la >= 2) {
            cs[1] = p1[0];
            cs[2] = p1[1];
            m = 3;
        }
        if (la >= 3) {
#pragma unroll
            for (int q = 0; q < 4; ++q) cs[3 + q] = p2[q];
            m = 7;
        }
        ringv(cs, m, rk);
        // walk the path actually taken
        const float E0 = energy(p0, rk[0]);
        consider(best, p0, E0);
        st = s0;
        golden_put(st, l0, p0, E0);
        if (la >= 2) {
            const bool l1 = st.E1 < st.E2;
            const int o1 = l1 ? 0 : 1;
            const float q1 = golden_take(st, l1);
            const float E1v = energy(q1, rk[1 + o1]);
            consider(best, q1, E1v);
            golden_put(st, l1, q1, E1v);
            if (la >= 3) {
                const bool l2 = st.E1 < st.E2;
                const int o2 = l2 ? 0 : 1;
                const float q2 = golden_take(st, l2);
                const float E2v = energy(q2, rk[3 + 2 * o1 + o2]);
                consider(best, q2, E2v);
                golden_put(st, l2, q2, E2v);
            }
        }
        steps -= la;
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

__device__ __forceinline__ bool ring_slot(int j, int r0, int r1, int c0, int c1, int H, int W,
                                          const float* __restrict__ S,
                                          const float* __restrict__ R, int lb, int ncol, int k,
                                          float w[9], unsigned& mask) {
    return ring_slot_v(j, r0, r1, c0, c1, H, W,
                       [&](int r, int c) { return phase_read(S, R, r, c, W, lb, ncol, k); }, w,
                       mask);
}

}  // namespace cm
