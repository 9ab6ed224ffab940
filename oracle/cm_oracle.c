/*
 * cm_oracle.c -- FP64 CPU oracle for the multigrid curvature-energy sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow restatement of the
 * paper's method ("Fast Multi-grid Methods for Minimizing Curvature
 * Energies", Zhang, Chen, Tang, Duan) that the CUDA library is checked
 * against.  It shares no code, header, table or constant with the CUDA path,
 * and nothing in the product links it.  Only the tests, the package's smoke
 * check and the benchmark's CPU-baseline leg may load it.
 *
 * Every quantity is IEEE double.  Notation follows the paper: u the current
 * image, f the observation, alpha the fidelity weight, d_l the distance of the
 * centre pixel to tangent plane T_l, kappa the curvature, c the constant
 * correction of one patch (block).  Readings of passages the paper leaves
 * open are marked READING and listed in the design notes.
 *
 * Pinned by tests/test_oracle_*.py: plane distance against Eq. (distance to
 * tri) and hand geometry, curvature against sphere caps and paraboloids
 * (closed forms, O(h^2) order), affine/constant invariants, D4 and
 * translation invariance, the ring-energy identity against the full energy
 * difference, brute-force block minimisation on 8x8 images, the search
 * with a caller-supplied ring sum (orc_block_search) against the whole-image
 * search, and monotone descent in sequential mode.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MEAN 0
#define ORC_GAUSS 1
#define ORC_MEAN_EULER 2   /* extension: principal curvatures from Euler's formula */
#define ORC_GAUSS_EULER 3

/* ------------------------------------------------------------------------ */
/* Image access with the boundary condition.                                 */
/* READING (Sec. 2.2, the domain is prolongated "using boundary              */
/* conditions"): a pixel outside the image takes the value of the nearest    */
/* in-image pixel (clamp to edge, rows and columns independently).           */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* A read-only view of u with an optional constant shift on one block
 * A = [r0, r1) x [c0, c1): value(r, c) = u(clamp(r), clamp(c)) + shift if the
 * clamped pixel lies in A.  This is u + shift * phi_A of Sec. 2.2. */
typedef struct {
    const double *u;
    int H, W;
    int r0, r1, c0, c1;
    double shift;
} field_t;

static double fval(const field_t *F, int r, int c) {
    r = clampi(r, 0, F->H - 1);
    c = clampi(c, 0, F->W - 1);
    double v = F->u[(size_t)r * F->W + c];
    if (r >= F->r0 && r < F->r1 && c >= F->c0 && c < F->c1) v += F->shift;
    return v;
}

/* ------------------------------------------------------------------------ */
/* Tangent-plane distance, Eq. (distance to tri), Sec. 2.1.                  */
/* X, Y, Z are three neighbours of the centre O in 3-D (column, row,        */
/* value).  n = XZ x XY; d = XO . n / |n|.  The paper's worked instance      */
/* (X = W, Y = E, Z = N) gives n_z < 0; every plane here is oriented the     */
/* same way (n_z < 0) so that the eight distances share one sign convention: */
/* d > 0 when O lies below the plane.                                        */

double orc_plane_distance(const double X[3], const double Y[3], const double Z[3],
                          const double O[3]) {
    double a[3] = {Z[0] - X[0], Z[1] - X[1], Z[2] - X[2]};   /* XZ */
    double b[3] = {Y[0] - X[0], Y[1] - X[1], Y[2] - X[2]};   /* XY */
    double n[3] = {a[1] * b[2] - a[2] * b[1],
                   a[2] * b[0] - a[0] * b[2],
                   a[0] * b[1] - a[1] * b[0]};
    if (n[2] > 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
    double xo[3] = {O[0] - X[0], O[1] - X[1], O[2] - X[2]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    return (xo[0] * n[0] + xo[1] * n[1] + xo[2] * n[2]) / nn;
}

/* The eight tangent planes of the 3x3 window (Sec. 2.1, "8 local tangent
 * planes ... pairwise centrosymmetric").  READING: four lines through O
 * (W-E, N-S, NW-SE, NE-SW); for each line X-Y two planes, through X, Y and
 * one of the two remaining neighbours that flank the line on opposite
 * sides.  The two planes of a line are centrosymmetric images of each
 * other about O.  Offsets are (drow, dcol). */
static const int LINE_X[4][2] = {{0, -1}, {-1, 0}, {-1, -1}, {-1, 1}};
static const int LINE_Y[4][2] = {{0, 1}, {1, 0}, {1, 1}, {1, -1}};
static const int LINE_Z1[4][2] = {{-1, 0}, {0, -1}, {-1, 1}, {-1, -1}};
static const int LINE_Z2[4][2] = {{1, 0}, {0, 1}, {1, -1}, {1, 1}};

static void point3(const field_t *F, int r, int c, int dr, int dc, double P[3]) {
    P[0] = (double)dc;           /* x = column offset */
    P[1] = (double)dr;           /* y = row offset    */
    P[2] = fval(F, r + dr, c + dc);
}

/* Direction curvatures at pixel (r, c).
 * d[2*t], d[2*t+1]: distances to the two planes of line t.
 * kbar[t]: pair-averaged normal curvature of line t.
 * READING (Sec. 3, kappa = II/I ~ d/ds^2): kappa_l = 2 d_l / ds^2 with ds^2 =
 * |XY|^2 / 4 the squared half-chord of the line in 3-D.  The factor 2 is the
 * circle-through-three-points relation (sagitta = chord^2 / (8 R)); with it a
 * sampled sphere of radius R gives |kappa| -> 1/R.  Averaging the two
 * centrosymmetric planes cancels the first-order bias of either one. */
void orc_direction_curvatures_f(const field_t *F, int r, int c, double kbar[4], double d[8]) {
    double O[3];
    point3(F, r, c, 0, 0, O);
    for (int t = 0; t < 4; ++t) {
        double X[3], Y[3], Z1[3], Z2[3];
        point3(F, r, c, LINE_X[t][0], LINE_X[t][1], X);
        point3(F, r, c, LINE_Y[t][0], LINE_Y[t][1], Y);
        point3(F, r, c, LINE_Z1[t][0], LINE_Z1[t][1], Z1);
        point3(F, r, c, LINE_Z2[t][0], LINE_Z2[t][1], Z2);
        double d1 = orc_plane_distance(X, Y, Z1, O);
        double d2 = orc_plane_distance(X, Y, Z2, O);
        double dx = Y[0] - X[0], dy = Y[1] - X[1], dz = Y[2] - X[2];
        double ds2 = 0.25 * (dx * dx + dy * dy + dz * dz);
        d[2 * t] = d1;
        d[2 * t + 1] = d2;
        kbar[t] = 0.5 * (2.0 * d1 / ds2 + 2.0 * d2 / ds2);
    }
}

/* Principal curvatures as the extreme direction curvatures (Sec. 3:
 * kappa_min = min_l kappa_l, kappa_max = max_l kappa_l).  Mean curvature
 * H = (kappa_min + kappa_max) / 2 (Table I, Eq. MCM); Gaussian curvature
 * K = kappa_min * kappa_max (Eq. GCM). */
static void euler_fit(const double kbar[4], double *kmin, double *kmax);

static double curv_from_kbar(const double kbar[4], int kind) {
    double kmin = kbar[0], kmax = kbar[0];
    if (kind == ORC_MEAN_EULER || kind == ORC_GAUSS_EULER) {
        euler_fit(kbar, &kmin, &kmax);
    } else {
        for (int t = 1; t < 4; ++t) {
            if (kbar[t] < kmin) kmin = kbar[t];
            if (kbar[t] > kmax) kmax = kbar[t];
        }
    }
    return (kind == ORC_MEAN || kind == ORC_MEAN_EULER) ? 0.5 * (kmin + kmax) : kmin * kmax;
}

/* Extension (not in the paper): principal curvatures from Euler's theorem.
 * The normal curvature of a smooth surface in the tangent direction at angle
 * theta is kappa(theta) = k1 cos^2(theta - phi) + k2 sin^2(theta - phi)
 *                       = a + b cos(2 theta) + s sin(2 theta),
 * a = (k1 + k2)/2, sqrt(b^2 + s^2) = |k1 - k2|/2.  The four direction
 * curvatures are samples of kappa at the angles of their lines in the image
 * plane; (a, b, s) is their least-squares fit, found here from the 3 x 3
 * normal equations (D^T D) x = D^T kbar with rows D_t = (1, cos 2 theta_t,
 * sin 2 theta_t), solved by Gauss-Jordan elimination with partial pivoting.  Then
 * k1,2 = a -+ sqrt(b^2 + s^2).  Unlike the extreme sampled directions, this
 * recovers the principal curvatures of a quadric whose principal axes are not
 * aligned with the pixel grid. */
static void euler_fit(const double kbar[4], double *kmin, double *kmax) {
    double M[3][4];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) M[i][j] = 0.0;
    for (int t = 0; t < 4; ++t) {
        double dx = (double)(LINE_Y[t][1] - LINE_X[t][1]);   /* column direction */
        double dy = (double)(LINE_Y[t][0] - LINE_X[t][0]);   /* row direction    */
        double th = atan2(dy, dx);
        double row[3] = {1.0, cos(2.0 * th), sin(2.0 * th)};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) M[i][j] += row[i] * row[j];
            M[i][3] += row[i] * kbar[t];
        }
    }
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int i = col + 1; i < 3; ++i)
            if (fabs(M[i][col]) > fabs(M[piv][col])) piv = i;
        for (int j = 0; j < 4; ++j) {
            double tmp = M[col][j];
            M[col][j] = M[piv][j];
            M[piv][j] = tmp;
        }
        for (int i = 0; i < 3; ++i) {
            if (i == col) continue;
            double fct = M[i][col] / M[col][col];
            for (int j = col; j < 4; ++j) M[i][j] -= fct * M[col][j];
        }
    }
    double a = M[0][3] / M[0][0], b = M[1][3] / M[1][1], s = M[2][3] / M[2][2];
    double rad = sqrt(b * b + s * s);
    *kmin = a - rad;
    *kmax = a + rad;
}

static double curv_f(const field_t *F, int r, int c, int kind) {
    double kbar[4], d[8];
    orc_direction_curvatures_f(F, r, c, kbar, d);
    return curv_from_kbar(kbar, kind);
}

static field_t plain_field(const double *u, int H, int W) {
    field_t F = {u, H, W, 0, 0, 0, 0, 0.0};
    return F;
}

void orc_direction_curvatures(const double *u, int H, int W, int r, int c,
                              double kbar[4], double d[8]) {
    field_t F = plain_field(u, H, W);
    orc_direction_curvatures_f(&F, r, c, kbar, d);
}

double orc_curvature(const double *u, int H, int W, int r, int c, int kind) {
    field_t F = plain_field(u, H, W);
    return curv_f(&F, r, c, kind);
}

void orc_curvature_map(const double *u, int H, int W, int kind, double *out) {
    field_t F = plain_field(u, H, W);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) out[(size_t)r * W + c] = curv_f(&F, r, c, kind);
}

/* ------------------------------------------------------------------------ */
/* Discrete energy, Eq. (MCM) (mean) and Eq. (GCM) (Gaussian):               */
/* F(u) = sum_pixels |kappa(u)| + alpha/2 (u - f)^2.                         */

double orc_energy(const double *u, const double *f, int H, int W, double alpha, int kind) {
    field_t F = plain_field(u, H, W);
    double E = 0.0;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            double e = u[(size_t)r * W + c] - f[(size_t)r * W + c];
            E += fabs(curv_f(&F, r, c, kind)) + 0.5 * alpha * e * e;
        }
    return E;
}

/* ------------------------------------------------------------------------ */
/* Block (patch) subproblem, Sec. 2.2: minimise F(u + c phi_A) over c.       */
/*                                                                           */
/* The fidelity part of F(u + c phi_A) - F(u) is alpha/2 (s c^2 + 2 c S1)    */
/* with S1 = sum_A (u - f) and s = |A|.  The curvature of a pixel changes    */
/* only if its 3x3 stencil (after clamping) holds pixels both inside and     */
/* outside A; every other pixel's curvature is unchanged because the plane   */
/* distances depend on differences of u only.  Those pixels form ring(A):    */
/* in-image pixels within Chebyshev distance 1 of A, less the pixels of A    */
/* whose whole clamped stencil lies in A.                                    */
/* E_A(c) = alpha/2 (s c^2 + 2 c S1) + sum_{q in ring(A)} |kappa_q(u + c phi_A)| */
/* so that E_A(c) - E_A(0) = F(u + c phi_A) - F(u) exactly.                  */

typedef struct {
    int r0, r1, c0, c1;      /* block, clipped to the image */
} block_t;

static int in_block(const block_t *A, int r, int c) {
    return r >= A->r0 && r < A->r1 && c >= A->c0 && c < A->c1;
}

static int is_ring(const block_t *A, int H, int W, int r, int c) {
    if (!in_block(A, r, c)) return 1;   /* caller iterates the 1-dilation of A */
    for (int dr = -1; dr <= 1; ++dr)
        for (int dc = -1; dc <= 1; ++dc) {
            int rr = clampi(r + dr, 0, H - 1), cc = clampi(c + dc, 0, W - 1);
            if (!in_block(A, rr, cc)) return 1;
        }
    return 0;
}

static double ring_curv_sum(const double *u, int H, int W, const block_t *A,
                            double shift, int kind) {
    field_t F = {u, H, W, A->r0, A->r1, A->c0, A->c1, shift};
    double acc = 0.0;
    int ra = A->r0 - 1 < 0 ? 0 : A->r0 - 1, rb = A->r1 + 1 > H ? H : A->r1 + 1;
    int ca = A->c0 - 1 < 0 ? 0 : A->c0 - 1, cb = A->c1 + 1 > W ? W : A->c1 + 1;
    for (int r = ra; r < rb; ++r)
        for (int c = ca; c < cb; ++c)
            if (is_ring(A, H, W, r, c)) acc += fabs(curv_f(&F, r, c, kind));
    return acc;
}

int orc_ring_size(int H, int W, int r0, int c0, int bh, int bw) {
    block_t A = {r0, r0 + bh, c0, c0 + bw};
    int n = 0;
    for (int r = (r0 - 1 < 0 ? 0 : r0 - 1); r < (A.r1 + 1 > H ? H : A.r1 + 1); ++r)
        for (int c = (c0 - 1 < 0 ? 0 : c0 - 1); c < (A.c1 + 1 > W ? W : A.c1 + 1); ++c)
            n += is_ring(&A, H, W, r, c);
    return n;
}

static double block_S1(const double *u, const double *f, int W, const block_t *A) {
    double S1 = 0.0;
    for (int r = A->r0; r < A->r1; ++r)
        for (int c = A->c0; c < A->c1; ++c)
            S1 += u[(size_t)r * W + c] - f[(size_t)r * W + c];
    return S1;
}

static double local_energy(const double *u, int H, int W, const block_t *A, double c,
                           double alpha, int kind, double S1) {
    double s = (double)(A->r1 - A->r0) * (double)(A->c1 - A->c0);
    return 0.5 * alpha * (s * c * c + 2.0 * c * S1) + ring_curv_sum(u, H, W, A, c, kind);
}

double orc_local_energy(const double *u, const double *f, int H, int W, int r0, int c0,
                        int bh, int bw, double c, double alpha, int kind) {
    block_t A = {r0, r0 + bh, c0, c0 + bw};
    return local_energy(u, H, W, &A, c, alpha, kind, block_S1(u, f, W, &A));
}

/* The paper's one-step estimate on the finest layer (Alg. 2 with t = 0,
 * c_0 = 0, eta_0 = 1, as the remark after Theorem 1 prescribes):
 *   c_{1/2} = (1/8) sum_l d_l                       (Eq. c-sol1, mean)
 *   c_{1/2} = d*, distance to T* (Prop. 2, Gaussian): T* is the plane pair
 *             of the extreme direction curvature with the smaller |kappa|;
 *             READING: d* is the mean of that pair's two distances.
 *   c_1 = (c_0 + c_{1/2} + alpha eta_0 f*) / (2 + alpha eta_0)  (Eq. c-sol2)
 * with f* = f - u at the pixel.  The Eq. (FOBOS step2) form with a single
 * prox term would give 1 + alpha eta; Eq. (c-sol2) and the coarse-layer
 * closed form both use 2 + alpha eta, which is followed here. */
double orc_chalf(const double *u, int H, int W, int r, int c, int kind);

double orc_paper_candidate(const double *u, const double *f, int H, int W, int r, int c,
                           double alpha, int kind) {
    double chalf = orc_chalf(u, H, W, r, c, kind);
    double fstar = f[(size_t)r * W + c] - u[(size_t)r * W + c];
    return (0.0 + chalf + alpha * 1.0 * fstar) / (2.0 + alpha * 1.0);
}

/* c_{1/2} of the pixel (r, c): the shift that the curvature term alone asks
 * for (Eq. c-sol1 for mean curvature, Prop. 2 for Gaussian curvature; the
 * Euler-fit kinds use the rule of their base kind). */
double orc_chalf(const double *u, int H, int W, int r, int c, int kind) {
    double kbar[4], d[8];
    orc_direction_curvatures(u, H, W, r, c, kbar, d);
    double chalf;
    if (kind == ORC_MEAN || kind == ORC_MEAN_EULER) {
        chalf = 0.0;
        for (int l = 0; l < 8; ++l) chalf += d[l];
        chalf /= 8.0;
    } else {
        int tmin = 0, tmax = 0;
        for (int t = 1; t < 4; ++t) {
            if (kbar[t] < kbar[tmin]) tmin = t;
            if (kbar[t] > kbar[tmax]) tmax = t;
        }
        int ts = fabs(kbar[tmin]) <= fabs(kbar[tmax]) ? tmin : tmax;
        chalf = 0.5 * (d[2 * ts] + d[2 * ts + 1]);
    }
    return chalf;
}

void orc_chalf_map(const double *u, int H, int W, int kind, double *out) {
#pragma omp parallel for schedule(static)
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) out[(size_t)r * W + c] = orc_chalf(u, H, W, r, c, kind);
}

/* Candidate bookkeeping: keep the lowest E; energies within the tie
 * tolerance keep the smaller |c|, then the smaller c, so that an already
 * optimal block returns exactly 0. */
typedef struct {
    double c, E;
    int n_eval;
} best_t;

static void consider(best_t *b, double c, double E) {
    b->n_eval++;
    double tau = 1e-12 * (fabs(b->E) > 1.0 ? fabs(b->E) : 1.0);
    if (E < b->E - tau) { b->c = c; b->E = E; return; }
    if (fabs(E - b->E) <= tau) {
        if (fabs(c) < fabs(b->c) || (fabs(c) == fabs(b->c) && c < b->c)) { b->c = c; b->E = E; }
    }
}

typedef struct {
    double c;          /* chosen correction */
    double E_best;     /* E_A(c) */
    double E_zero;     /* E_A(0) */
    double c_fid;      /* -S1/s, the block-mean of f - u (the paper's f*) */
    double rho;        /* bracket half-width */
    double S1;
    int n_eval;
} blockres_t;

/* The search sees the block only through s, S1 and its ring sum
 * R(c) = sum_{q in ring(A)} |kappa_q(u + c phi_A)|, so that the same steps
 * serve a block whose ring is summed by several owners (each adds the ring
 * pixels of its rows).  cand: the closed-form candidate (the paper's c_1 on
 * the finest level), or NaN for none. */
typedef double (*ring_fn)(double c, void *ctx);

static double search_energy(double s, double S1, double alpha, double c, ring_fn ring,
                            void *ctx) {
    return 0.5 * alpha * (s * c * c + 2.0 * c * S1) + ring(c, ctx);
}

static blockres_t block_search(double s, double S1, double alpha, int G, int K, int one_step,
                               double cand, ring_fn ring, void *ctx) {
    blockres_t res;
    double c_fid = -S1 / s;
    best_t b;
    b.c = 0.0;
    b.E = search_energy(s, S1, alpha, 0.0, ring, ctx);
    b.n_eval = 1;
    double E0 = b.E;
    if (one_step) {
        /* One step of Alg. 2 (t = 0, c_0 = 0, eta = 1): c_1 = (c_1/2 + alpha f*) /
         * (2 + alpha), f* = c_fid the block's mean of f - u.  On the finest level
         * c_1/2 is the plane-distance estimate (Eq. c-sol1; Prop. 2 for Gaussian
         * curvature), passed in as cand; on coarser levels READING: c_1/2 = 0
         * (the paper's coarse tangent-plane sets are not recoverable).  The
         * block keeps c_1 only if it lowers E_A (tie rule as below), else 0. */
        double c1 = cand == cand ? cand : alpha * c_fid / (2.0 + alpha);
        consider(&b, c1, search_energy(s, S1, alpha, c1, ring, ctx));
        res.c = b.c;
        res.E_best = b.E;
        res.E_zero = E0;
        res.c_fid = c_fid;
        res.rho = 0.0;
        res.S1 = S1;
        res.n_eval = b.n_eval;
        return res;
    }
    if (cand == cand) consider(&b, cand, search_energy(s, S1, alpha, cand, ring, ctx));
    double Rk = ring(c_fid, ctx);
    double rho = sqrt(2.0 * Rk / (alpha * s));
    /* grid */
    double gbest = c_fid, Egbest = INFINITY;
    for (int i = 0; i < G; ++i) {
        double g = c_fid + rho * (2.0 * i / (double)(G - 1) - 1.0);
        double E = search_energy(s, S1, alpha, g, ring, ctx);
        consider(&b, g, E);
        if (E < Egbest) { Egbest = E; gbest = g; }
    }
    /* golden section */
    double D = 2.0 * rho / (double)(G - 1);
    const double phi = 0.5 * (sqrt(5.0) - 1.0);
    double lo = gbest - D, hi = gbest + D;
    double x1 = hi - phi * (hi - lo), x2 = lo + phi * (hi - lo);
    double E1 = search_energy(s, S1, alpha, x1, ring, ctx);
    double E2 = search_energy(s, S1, alpha, x2, ring, ctx);
    consider(&b, x1, E1);
    consider(&b, x2, E2);
    for (int k = 2; k < K; ++k) {
        if (E1 < E2) {
            hi = x2; x2 = x1; E2 = E1;
            x1 = hi - phi * (hi - lo);
            E1 = search_energy(s, S1, alpha, x1, ring, ctx);
            consider(&b, x1, E1);
        } else {
            lo = x1; x1 = x2; E1 = E2;
            x2 = lo + phi * (hi - lo);
            E2 = search_energy(s, S1, alpha, x2, ring, ctx);
            consider(&b, x2, E2);
        }
    }
    res.c = b.c;
    res.E_best = b.E;
    res.E_zero = E0;
    res.c_fid = c_fid;
    res.rho = rho;
    res.S1 = S1;
    res.n_eval = b.n_eval;
    return res;
}

typedef struct {
    const double *u;
    int H, W, kind;
    const block_t *A;
} image_ring_t;

static double image_ring(double c, void *ctx) {
    const image_ring_t *r = (const image_ring_t *)ctx;
    return ring_curv_sum(r->u, r->H, r->W, r->A, c, r->kind);
}

/* Block minimiser.  The paper solves the 1-D problem approximately with a
 * closed-form FBS step (Alg. 2, Eq. c-sol2, and the coarse closed form of
 * Sec. 2.2); the objective of each subproblem is min_c F(u + c phi_A)
 * (Alg. 3).  This oracle minimises that objective directly:
 *  (i)   c_fid = -S1/s; E_A as above.
 *  (ii)  bracket: every minimiser c* satisfies alpha s (c* - c_fid)^2 / 2 <=
 *        sum_ring |kappa(c_fid)| (from E_A(c*) <= E_A(c_fid)), so c* lies in
 *        [c_fid - rho, c_fid + rho], rho = sqrt(2 sum_ring|kappa(c_fid)| / (alpha s)).
 *  (iii) E_A at G equispaced points of the bracket (G odd, so c_fid is one).
 *  (iv)  golden-section search with K evaluations on [g* - D, g* + D], g* the
 *        best grid point and D the grid step.
 *  (v)   also c = 0 and, on the finest layer, the paper's c_1 above.
 *  (vi)  the result is the best of every evaluated point (tie rule above),
 *        so E_A(c) <= E_A(0): no block update raises F with the others fixed.
 * READING: the paper's closed-form candidate (Alg. 2, Eq. c-sol1) is the
 * pixel step of the finest level; a 1 x 1 block clipped at the image corner
 * on a coarser level is not a level-1 pixel and gets the search alone. */
static blockres_t block_min(const double *u, const double *f, int H, int W, const block_t *A,
                            double alpha, int kind, int G, int K, int use_paper, int one_step,
                            int finest) {
    double s = (double)(A->r1 - A->r0) * (double)(A->c1 - A->c0);
    double S1 = block_S1(u, f, W, A);
    int pixel = finest && A->r1 - A->r0 == 1 && A->c1 - A->c0 == 1;
    double cand = NAN;
    if (pixel && (one_step || use_paper))
        cand = orc_paper_candidate(u, f, H, W, A->r0, A->c0, alpha, kind);
    image_ring_t ctx = {u, H, W, kind, A};
    return block_search(s, S1, alpha, G, K, one_step, cand, image_ring, &ctx);
}

/* The search alone, for a block whose ring sum the caller assembles (e.g.
 * from the partial sums of several row strips): s = |A|, S1 = sum_A (u - f),
 * ring(c) = sum_{q in ring(A)} |kappa_q(u + c phi_A)|, cand = the closed-form
 * candidate or NaN.  info as in orc_block_min. */
double orc_block_search(double s, double S1, double alpha, int G, int K, int one_step,
                        double cand, double (*ring)(double, void *), void *ctx, double *info) {
    blockres_t res = block_search(s, S1, alpha, G, K, one_step, cand, ring, ctx);
    if (info) {
        info[0] = res.E_best; info[1] = res.E_zero; info[2] = res.c_fid;
        info[3] = res.rho; info[4] = res.S1; info[5] = (double)res.n_eval;
    }
    return res.c;
}

double orc_block_min(const double *u, const double *f, int H, int W, int r0, int c0, int bh,
                     int bw, double alpha, int kind, int G, int K, int use_paper, int one_step,
                     int finest, double *info /* nullable: E_best, E_zero, c_fid, rho, S1, n_eval */) {
    block_t A = {r0, r0 + bh > H ? H : r0 + bh, c0, c0 + bw > W ? W : c0 + bw};
    blockres_t res = block_min(u, f, H, W, &A, alpha, kind, G, K, use_paper, one_step, finest);
    if (info) {
        info[0] = res.E_best; info[1] = res.E_zero; info[2] = res.c_fid;
        info[3] = res.rho; info[4] = res.S1; info[5] = (double)res.n_eval;
    }
    return res.c;
}

/* ------------------------------------------------------------------------ */
/* Levels and colours (Sec. 2.2, Sec. 2.3).                                  */
/* READING: the block side on level j (j = 1..L) is 2^(j-1); blocks are      */
/* anchored at (0, 0) and clipped at the right and bottom edges (the paper   */
/* uses sides 2^j - 1 and extends the domain; the extended pixels are not    */
/* part of F).  Colour of block (bi, bj): ncolors = 2 -> (bi + bj) mod 2     */
/* (checkerboard); ncolors = p^2 (p = 2, 3, 4) -> p (bi mod p) + (bj mod p),   */
/* the p x p decomposition (p = 2: the paper's four colours); ncolors = 1 ->  */
/* 0 (a schedule option for the coarse levels: every block in one phase).    */

int orc_block_colour(int bi, int bj, int ncolors) {
    if (ncolors == 1) return 0;
    if (ncolors == 2) return (bi + bj) & 1;
    int p = ncolors == 16 ? 4 : (ncolors == 9 ? 3 : 2);
    return p * (bi % p) + (bj % p);
}

/* Colours of the level with block side b.  ncolors = 0 selects the decoupled
 * colouring: the smallest p >= 2 with (p - 1) b >= 3, so that two blocks of
 * one colour are at least 3 pixels apart and share no stencil (a ring pixel
 * of one is never in the window of a ring pixel of the other); a colour's
 * parallel solve then equals solving its blocks one after another.
 * coarse_ncolors != 0 sets the colour count of the levels with b >= 64 (a
 * schedule option: fewer sequential phases on the coarse levels, whose
 * same-colour blocks then share only corner pixels of their rings). */
int orc_level_colours(int ncolors, int b, int coarse_ncolors) {
    if (coarse_ncolors != 0 && b >= 64) return coarse_ncolors;
    if (ncolors != 0) return ncolors;
    int p = 2;
    while ((p - 1) * b < 3) ++p;
    return p * p;
}

/* Block side of level j = 1, 2, ...  sides = 0: b_j = 2^(j-1) (the reading
 * used by default; see the notes on Sec. 2.2); sides = 1: the paper's
 * patches of (2^j - 1) x (2^j - 1) pixels, m_j = ceil(m / (2^j - 1)) patches
 * down a column (Sec. 2.2). */
int orc_level_side(int j, int sides) { return sides ? (1 << j) - 1 : 1 << (j - 1); }

/* Default level count: the coarsest block side is the largest one <= half
 * the shorter image side. */
int orc_auto_levels(int H, int W, int sides) {
    int m = H < W ? H : W;
    int L = 1;
    while (orc_level_side(L + 1, sides) <= m / 2) ++L;
    return L;
}

/* One phase: every block of colour k on level with side b computes its
 * correction from the state at the start of the phase, then all blocks
 * apply.  READING of Sec. 2.3 (same-colour subproblems "can be solved in
 * parallel"): with a 3x3 stencil same-colour blocks interact unless they are
 * at least 3 pixels apart, so the phase is defined with snapshot (Jacobi)
 * semantics, which is what a parallel solve of the colour computes.
 * Returns the number of blocks; cs (nullable) receives each block's c in
 * block raster order (entries of other colours are left untouched). */
int orc_phase(double *u, const double *f, int H, int W, double alpha, int kind, int b,
              int ncolors, int k, int G, int K, int use_paper, int one_step, double *cs) {
    int nbi = (H + b - 1) / b, nbj = (W + b - 1) / b;
    int nb = nbi * nbj;
    double *cloc = (double *)malloc(sizeof(double) * (size_t)nb);
    int count = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : count)
    for (int idx = 0; idx < nb; ++idx) {
        int bi = idx / nbj, bj = idx % nbj;
        cloc[idx] = 0.0;
        if (orc_block_colour(bi, bj, ncolors) != k) continue;
        block_t A = {bi * b, (bi + 1) * b > H ? H : (bi + 1) * b,
                     bj * b, (bj + 1) * b > W ? W : (bj + 1) * b};
        blockres_t res = block_min(u, f, H, W, &A, alpha, kind, G, K, use_paper, one_step, b == 1);
        cloc[idx] = res.c;
        ++count;
    }
    /* apply: u <- u + L_j c_j on the blocks of this colour */
    for (int idx = 0; idx < nb; ++idx) {
        int bi = idx / nbj, bj = idx % nbj;
        if (orc_block_colour(bi, bj, ncolors) != k) continue;
        if (cs) cs[idx] = cloc[idx];
        for (int r = bi * b; r < (bi + 1) * b && r < H; ++r)
            for (int c = bj * b; c < (bj + 1) * b && c < W; ++c) u[(size_t)r * W + c] += cloc[idx];
    }
    free(cloc);
    return count;
}

/* Sequential (Gauss-Seidel) variant of a level: blocks in raster order, each
 * applied before the next is solved (Alg. 1 generalised to patches).  Every
 * single update satisfies F(u + c phi_A) <= F(u). */
void orc_level_sequential(double *u, const double *f, int H, int W, double alpha, int kind,
                          int b, int G, int K, int use_paper, int one_step) {
    int nbi = (H + b - 1) / b, nbj = (W + b - 1) / b;
    for (int bi = 0; bi < nbi; ++bi)
        for (int bj = 0; bj < nbj; ++bj) {
            block_t A = {bi * b, (bi + 1) * b > H ? H : (bi + 1) * b,
                         bj * b, (bj + 1) * b > W ? W : (bj + 1) * b};
            blockres_t res = block_min(u, f, H, W, &A, alpha, kind, G, K, use_paper, one_step, b == 1);
            for (int r = A.r0; r < A.r1; ++r)
                for (int c = A.c0; c < A.c1; ++c) u[(size_t)r * W + c] += res.c;
        }
}

/* One cycle: fine-to-coarse half V-cycle (Sec. 2.2: the coarse-to-fine half
 * is omitted), colours in ascending order on each level (Alg. 3). */
/* One cycle: levels 1 .. L (the half V-cycle of Alg. 3); with vcycle also
 * back up, levels L - 1 .. 1 (the full V-cycle the paper compares against). */
void orc_cycle(double *u, const double *f, int H, int W, double alpha, int kind, int levels,
               int ncolors, int G, int K, int use_paper, int one_step, int sequential,
               int vcycle, int sides, int coarse_ncolors) {
    if (levels <= 0) levels = orc_auto_levels(H, W, sides);
    int nsteps = vcycle ? 2 * levels - 1 : levels;
    for (int s = 0; s < nsteps; ++s) {
        int j = s < levels ? s + 1 : 2 * levels - 1 - s;
        int b = orc_level_side(j, sides);
        if (sequential) {
            orc_level_sequential(u, f, H, W, alpha, kind, b, G, K, use_paper, one_step);
        } else {
            int nc = orc_level_colours(ncolors, b, coarse_ncolors);
            for (int k = 0; k < nc; ++k)
                orc_phase(u, f, H, W, alpha, kind, b, nc, k, G, K, use_paper, one_step, NULL);
        }
    }
}

/* Outer loop, Alg. 3 with the relative-energy stopping test Eq. (reerr):
 * stop when |F(u_l) - F(u_{l-1})| / |F(u_l)| <= tol (tol > 0), or after
 * `cycles` cycles (exactly `cycles` when tol == 0).  READING: u_0 = f when no
 * initial guess is given.  trace (nullable, length cycles + 1) receives
 * F(u_0), F(u_1), ...  Returns the number of cycles run; *converged is set. */
int orc_solve(const double *f, int H, int W, double alpha, int kind, int levels, int cycles,
              double tol, const double *u0, double *u_out, int ncolors, int G, int K,
              int use_paper, int one_step, int sequential, int vcycle, int sides,
              int coarse_ncolors, double *trace, int *converged) {
    size_t N = (size_t)H * W;
    if (u0) memcpy(u_out, u0, N * sizeof(double));
    else memcpy(u_out, f, N * sizeof(double));
    double Eprev = orc_energy(u_out, f, H, W, alpha, kind);
    if (trace) trace[0] = Eprev;
    int l = 0, conv = 0;
    while (l < cycles) {
        orc_cycle(u_out, f, H, W, alpha, kind, levels, ncolors, G, K, use_paper, one_step,
                  sequential, vcycle, sides, coarse_ncolors);
        ++l;
        double E = orc_energy(u_out, f, H, W, alpha, kind);
        if (trace) trace[l] = E;
        if (tol > 0.0 && fabs(E - Eprev) <= tol * fabs(E)) { conv = 1; Eprev = E; break; }
        Eprev = E;
    }
    if (converged) *converged = conv;
    return l;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing runs; results do not depend
 * on it, every parallel loop writes disjoint outputs). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* E_A at n points (used by the brute-force checks of the block minimiser). */
void orc_local_energy_batch(const double *u, const double *f, int H, int W, int r0, int c0,
                            int bh, int bw, double alpha, int kind, const double *cs, int n,
                            double *out) {
    block_t A = {r0, r0 + bh > H ? H : r0 + bh, c0, c0 + bw > W ? W : c0 + bw};
    double S1 = block_S1(u, f, W, &A);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) out[i] = local_energy(u, H, W, &A, cs[i], alpha, kind, S1);
}
