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

// Curvature kinds: kappa = H or K from the extreme direction curvatures
// (Sec. 3), or from a least-squares fit of Euler's formula to the four
// directions (an extension; see kappa_abs).
enum { KIND_MEAN = 0, KIND_GAUSS = 1, KIND_MEAN_EULER = 2, KIND_GAUSS_EULER = 3 };

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

// Signed kappa of a pixel from its direction curvatures k0 (W-E), k1 (N-S),
// k2 (NW-SE) and k3 (NE-SW).
//  KIND_MEAN, KIND_GAUSS: principal curvatures = the extreme directions,
//    H = (kmin + kmax) / 2, K = kmin kmax (Sec. 3, Eq. MCM / Eq. GCM).
//  KIND_MEAN_EULER, KIND_GAUSS_EULER: Euler's formula
//    kappa(theta) = a + b cos 2 theta + s sin 2 theta sampled at theta = 0,
//    90, 45 and 135 degrees.  The columns (1, cos 2 theta, sin 2 theta) of
//    these four samples are orthogonal, so the least-squares fit is
//    a = (k0 + k1 + k2 + k3) / 4, b = (k0 - k1) / 2, s = (k2 - k3) / 2, and
//    the principal curvatures are a -+ sqrt(b^2 + s^2): H = a,
//    K = a^2 - b^2 - s^2.
template <int KIND>
__device__ __forceinline__ float kappa_signed(float k0, float k1, float k2, float k3) {
    if (KIND == KIND_MEAN || KIND == KIND_GAUSS) {
        const float kmin = fminf(fminf(k0, k1), fminf(k2, k3));
        const float kmax = fmaxf(fmaxf(k0, k1), fmaxf(k2, k3));
        return KIND == KIND_MEAN ? 0.5f * (kmin + kmax) : kmin * kmax;
    }
    const float a = 0.25f * ((k0 + k1) + (k2 + k3));
    if (KIND == KIND_MEAN_EULER) return a;
    const float b = 0.5f * (k0 - k1), s = 0.5f * (k2 - k3);
    return fmaf(a, a, -fmaf(b, b, s * s));
}

template <int KIND>
__device__ __forceinline__ float kappa_abs(float k0, float k1, float k2, float k3) {
    return fabsf(kappa_signed<KIND>(k0, k1, k2, k3));
}

// |kappa| of the pixel whose 3x3 window is w (kind known at compile time).
template <int KIND>
__device__ __forceinline__ float abs_curvature(const float w[9]) {
    const KBar4 r = direction_curvatures(w);
    return kappa_abs<KIND>(r.k[0], r.k[1], r.k[2], r.k[3]);
}

// ---------------------------------------------------------------------------
// Direction curvature as a function of a block shift c.
//
// When the pixels of a block A move by c, each window entry moves by c or
// stays, so every ingredient of a direction is affine in c:
//   Dq = (u_Y - u_X)/2,  two_h * delta,  e_i = u_X + u_Y - 2 u_Zi.
// With ds^2 = h^2 + Dq^2 the plane term D^2 + 4h^2 equals 4 ds^2, so
//   kbar(c) = (two_h delta)(c) * sum_i rsqrt((e_i(c)^2 + 4 ds^2(c)) ds^4(c)),
// 13 FP32 operations and two rsqrt per direction and candidate.
struct AffDir {
    float dq0, dq1;   // Dq = dq0 + dq1 c
    float dl0, dl1;   // 2h delta = dl0 + dl1 c
    float e10, e11;   // e_1 = e10 + e11 c
    float e20, e21;   // e_2 = e20 + e21 c
};

// Line t of the window: end points X, Y, flanks Z1, Z2 (window indices).
__host__ __device__ constexpr int line_x(int t) { return t == 0 ? 3 : t == 1 ? 1 : t == 2 ? 0 : 2; }
__host__ __device__ constexpr int line_y(int t) { return t == 0 ? 5 : t == 1 ? 7 : t == 2 ? 8 : 6; }
__host__ __device__ constexpr int line_z1(int t) { return t == 0 ? 1 : t == 1 ? 3 : t == 2 ? 2 : 0; }
__host__ __device__ constexpr int line_z2(int t) { return t == 0 ? 7 : t == 1 ? 5 : t == 2 ? 6 : 8; }
__host__ __device__ constexpr float line_h2(int t) { return t < 2 ? 1.0f : 2.0f; }
__host__ __device__ constexpr float line_two_h(int t) {
    return t < 2 ? 2.0f : 2.8284271247461903f;
}

// Coefficients of line t for window w whose entries with bit q of `mask`
// belong to the shifted block.
__device__ __forceinline__ AffDir aff_dir(const float w[9], unsigned mask, int t) {
    const int X = line_x(t), Y = line_y(t), Z1 = line_z1(t), Z2 = line_z2(t);
    const float two_h = line_two_h(t);
    const float a = (float)((mask >> X) & 1u), b = (float)((mask >> Y) & 1u);
    const float o = (float)((mask >> 4) & 1u);
    const float z1 = (float)((mask >> Z1) & 1u), z2 = (float)((mask >> Z2) & 1u);
    AffDir d;
    d.dq0 = 0.5f * (w[Y] - w[X]);
    d.dq1 = 0.5f * (b - a);
    d.dl0 = two_h * fmaf(0.5f, w[X] + w[Y], -w[4]);
    d.dl1 = two_h * (0.5f * (a + b) - o);
    const float S = w[X] + w[Y];
    d.e10 = fmaf(-2.0f, w[Z1], S);
    d.e11 = a + b - 2.0f * z1;
    d.e20 = fmaf(-2.0f, w[Z2], S);
    d.e21 = a + b - 2.0f * z2;
    return d;
}

__device__ __forceinline__ float aff_kbar(const AffDir& d, float h2, float c) {
    const float Dq = fmaf(d.dq1, c, d.dq0);
    const float ds2 = fmaf(Dq, Dq, h2);
    const float fds = 4.0f * ds2;
    const float ds4 = ds2 * ds2;
    const float e1 = fmaf(d.e11, c, d.e10);
    const float e2 = fmaf(d.e21, c, d.e20);
    const float r = rsqrtf(fmaf(e1, e1, fds) * ds4) + rsqrtf(fmaf(e2, e2, fds) * ds4);
    return fmaf(d.dl1, c, d.dl0) * r;
}

// Ring pixel: the four directions of one 3x3 window under a block shift.
struct AffPix {
    AffDir d[4];
};

__device__ __forceinline__ AffPix aff_pix(const float w[9], unsigned mask) {
    AffPix p;
#pragma unroll
    for (int t = 0; t < 4; ++t) p.d[t] = aff_dir(w, mask, t);
    return p;
}

template <int KIND>
__device__ __forceinline__ float aff_abs_curv(const AffPix& p, float c) {
    const float k0 = aff_kbar(p.d[0], 1.0f, c), k1 = aff_kbar(p.d[1], 1.0f, c);
    const float k2 = aff_kbar(p.d[2], 2.0f, c), k3 = aff_kbar(p.d[3], 2.0f, c);
    return kappa_abs<KIND>(k0, k1, k2, k3);
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

// c_{1/2} of the pixel whose 3x3 window is w: the shift the curvature term
// alone asks for -- the mean of the eight plane distances (Eq. c-sol1) or,
// for Gaussian curvature, the mean distance of the plane pair of the extreme
// direction curvature with the smaller magnitude (Prop. 2).  The Euler-fit
// kinds use the rule of their base kind.
template <int KIND>
__device__ __forceinline__ float paper_chalf(const float w[9]) {
    const float SQ2x2 = 2.8284271247461903f;
    float d[8];
    dir_dist(w[3], w[5], w[4], w[1], w[7], 4.0f, 2.0f, d[0], d[1]);
    dir_dist(w[1], w[7], w[4], w[3], w[5], 4.0f, 2.0f, d[2], d[3]);
    dir_dist(w[0], w[8], w[4], w[2], w[6], 8.0f, SQ2x2, d[4], d[5]);
    dir_dist(w[2], w[6], w[4], w[0], w[8], 8.0f, SQ2x2, d[6], d[7]);
    float chalf;
    if (KIND == KIND_MEAN || KIND == KIND_MEAN_EULER) {
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
    return chalf;
}

// Clamp-to-edge boundary: out-of-image neighbours take the nearest pixel.
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Side p of a p x p colouring with `ncolors` = p^2 colours (ncolors = 2 is
// the checkerboard; ncolors = 1, one colour: every block in one phase).
__host__ __device__ __forceinline__ int colour_side(int ncolors) {
    return ncolors == 16 ? 4 : (ncolors == 9 ? 3 : (ncolors == 1 ? 1 : 2));
}

// Colour of block (bi, bj): ncolors == 2: checkerboard; ncolors == p^2:
// p (bi mod p) + (bj mod p) (p = 2: the paper's four colours; p = 1: 0).
__host__ __device__ __forceinline__ int block_colour(int bi, int bj, int ncolors) {
    if (ncolors == 2) return (bi + bj) & 1;
    if (ncolors == 4) return ((bi & 1) << 1) | (bj & 1);
    const int p = colour_side(ncolors);
    return p * (bi % p) + (bj % p);
}

// Colour of the block holding pixel (r, c) on the level with block side
// 1 << lb.
__device__ __forceinline__ int pixel_colour(int r, int c, int lb, int ncolors) {
    return block_colour(r >> lb, c >> lb, ncolors);
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

// Block index of pixel row (or column) r on a level whose block side is
// 1 << lb (POW2) or any side b (the paper's sides 2^j - 1).
template <bool POW2>
__device__ __forceinline__ int block_of(int r, int lb, int b) {
    return POW2 ? r >> lb : r / b;
}

template <bool POW2>
__device__ __forceinline__ float phase_read_b(const float* __restrict__ S,
                                              const float* __restrict__ R, int r, int c, int W,
                                              int lb, int b, int ncolors, int k) {
    if (POW2) return phase_read(S, R, r, c, W, lb, ncolors, k);
    size_t i = (size_t)r * W + c;
    if (k > 0 && block_colour(r / b, c / b, ncolors) < k) return R[i];
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
