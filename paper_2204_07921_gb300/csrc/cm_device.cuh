// cm_device.cuh -- device-side building blocks of the curvature sweep.
//
// Discrete surface geometry of Sec. 2.1 and Sec. 3 of "Fast Multi-grid
// Methods for Minimizing Curvature Energies" in FP32.
//
// Window layout: w[0..8] = NW N NE / W O E / SW S SE (row-major 3x3 around
// the centre O; rows are image rows, columns image columns).
//
// For a line X-O-Y through the centre (half length h in the image plane:
// h = 1 for W-E and N-S, h = sqrt(2) for the diagonals) and its two flanking
// neighbours Z1, Z2 the tangent planes (X, Y, Zi) of Eq. (distance to tri)
// give, with A = u_X, B = u_Y, D = B - A, S = A + B:
//   delta = S/2 - u_O                      (vertical gap of O under the chord)
//   n_i = XZi x XY,  d_i = XO . n_i / |n_i| = delta |n_z| / |n_i| = delta * 2h / sqrt(D^2 + (S - 2 u_Zi)^2 + 4 h^2)
// (axial lines: |n|^2 = D^2 + (S - 2 u_Z)^2 + 4, |n_z| = 2; diagonal lines:
// |n|^2 = 2 (D^2 + (S - 2 u_Z)^2 + 8), |n_z| = 4).
// (for h = 1 and Zi = N this is the paper's closed form).  The normal
// curvature of the plane is kappa_i = 2 d_i / ds^2 with ds^2 = h^2 + D^2/4 the
// squared 3-D half-chord; the direction curvature is the pair mean
//   kbar = (d_1 + d_2) / ds^2
//        = 2 h delta (rsqrt(m_1^2 ds^4) + rsqrt(m_2^2 ds^4)),
// m_i^2 = D^2 + (S - 2 u_Zi)^2 + 4 h^2, which takes two MUFU reciprocal
// square roots per direction.  kappa_min / kappa_max are the extreme
// direction curvatures; H = (kmin + kmax)/2 (Table I), K = kmin * kmax (Eq. GCM).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cm {

enum { KIND_MEAN = 0, KIND_GAUSS = 1 };

// Direction curvature of one line.  h2 = h^2 (1 or 2), two_h = 2h.
__device__ __forceinline__ float dir_kbar(float A, float B, float O, float Z1, float Z2,
                                          float four_h2, float h2, float two_h) {
    const float D = B - A;
    const float S = A + B;
    const float delta = fmaf(0.5f, S, -O);
    const float e1 = fmaf(-2.0f, Z1, S);
    const float e2 = fmaf(-2.0f, Z2, S);
    const float base = fmaf(D, D, four_h2);
    const float ds2 = fmaf(0.25f * D, D, h2);
    const float ds4 = ds2 * ds2;
    const float q1 = fmaf(e1, e1, base) * ds4;
    const float q2 = fmaf(e2, e2, base) * ds4;
    return two_h * delta * (rsqrtf(q1) + rsqrtf(q2));
}

struct KBar4 {
    float k[4];
};

__device__ __forceinline__ KBar4 direction_curvatures(const float w[9]) {
    const float SQ2x2 = 2.8284271247461903f;   // 2 sqrt(2)
    KBar4 r;
    // W-E, flanked by N and S
    r.k[0] = dir_kbar(w[3], w[5], w[4], w[1], w[7], 4.0f, 1.0f, 2.0f);
    // N-S, flanked by W and E
    r.k[1] = dir_kbar(w[1], w[7], w[4], w[3], w[5], 4.0f, 1.0f, 2.0f);
    // NW-SE, flanked by NE and SW
    r.k[2] = dir_kbar(w[0], w[8], w[4], w[2], w[6], 8.0f, 2.0f, SQ2x2);
    // NE-SW, flanked by NW and SE
    r.k[3] = dir_kbar(w[2], w[6], w[4], w[0], w[8], 8.0f, 2.0f, SQ2x2);
    return r;
}

// |H| or |K| of the pixel whose 3x3 window is w.
__device__ __forceinline__ float abs_curvature(const float w[9], int kind) {
    KBar4 r = direction_curvatures(w);
    float kmin = fminf(fminf(r.k[0], r.k[1]), fminf(r.k[2], r.k[3]));
    float kmax = fmaxf(fmaxf(r.k[0], r.k[1]), fmaxf(r.k[2], r.k[3]));
    return kind == KIND_MEAN ? fabsf(0.5f * (kmin + kmax)) : fabsf(kmin * kmax);
}

// Clamp-to-edge boundary: out-of-image neighbours take the nearest pixel.
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Colour of the block holding pixel (r, c) on the level with block side
// 1 << lb.  ncolors == 2: checkerboard of blocks; ncolors == 4: 2x2 parity.
__device__ __forceinline__ int pixel_colour(int r, int c, int lb, int ncolors) {
    int bi = r >> lb, bj = c >> lb;
    return ncolors == 2 ? ((bi + bj) & 1) : (((bi & 1) << 1) | (bj & 1));
}

// Phase-state read.  During phase k of a level, blocks of colours < k have
// already been written to R; every other pixel still holds its value in S.
__device__ __forceinline__ float phase_read(const float* __restrict__ S,
                                            const float* __restrict__ R, int r, int c, int W,
                                            int lb, int ncolors, int k) {
    size_t i = (size_t)r * W + c;
    if (k > 0 && pixel_colour(r, c, lb, ncolors) < k) return R[i];
    return S[i];
}

// ---------------------------------------------------------------------------
// Candidate bookkeeping of the block search: lowest energy wins; exactly
// equal energies keep the smaller |c|, then the smaller c.
struct Best {
    float c, E;
};

__device__ __forceinline__ void consider(Best& b, float c, float E) {
    bool take = (E < b.E) || (E == b.E && (fabsf(c) < fabsf(b.c) ||
                                           (fabsf(c) == fabsf(b.c) && c < b.c)));
    if (take) {
        b.c = c;
        b.E = E;
    }
}

constexpr float GOLDEN = 0.6180339887498949f;   // (sqrt(5) - 1) / 2

}  // namespace cm
