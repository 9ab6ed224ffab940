"""Pins of the oracle's surface geometry (Sec. 2.1, Sec. 3, Table I).

Each test checks the oracle against something other than itself: the
paper's own closed form of one plane distance, hand-derived worked examples,
analytic curvature of sphere caps and paraboloids, and exact invariances.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

ALL_KINDS = (oracle.MEAN, oracle.GAUSS, oracle.MEAN_EULER, oracle.GAUSS_EULER)
MEAN_KINDS = (oracle.MEAN, oracle.MEAN_EULER)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def test_plane_distance_matches_eq_distance_to_tri():
    """Eq. (distance to tri): for X = W, Y = E, Z = N the generic
    d = XO . n/|n|, n = XZ x XY reduces to
    (u_W + u_E - 2 u_O) / sqrt((u_W + u_E - 2 u_N)^2 + (u_E - u_W)^2 + 4)."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        uW, uE, uN, uO = rng.normal(size=4) * rng.choice([0.01, 1.0, 10.0])
        X = [-1.0, 0.0, uW]
        Y = [1.0, 0.0, uE]
        Z = [0.0, -1.0, uN]
        O = [0.0, 0.0, uO]
        d = oracle.plane_distance(X, Y, Z, O)
        ref = (uW + uE - 2 * uO) / math.sqrt((uW + uE - 2 * uN) ** 2 + (uE - uW) ** 2 + 4)
        assert d == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_plane_distance_is_euclidean_point_plane_distance():
    """|d| equals the textbook point-to-plane distance of O to the plane
    through X, Y, Z, for arbitrary points (not only grid neighbours)."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        X, Y, Z, O = rng.normal(size=(4, 3))
        # plane a.x = b through X, Y, Z via least squares on homogeneous coords
        M = np.array([np.append(P, 1.0) for P in (X, Y, Z)])
        _, _, vt = np.linalg.svd(M)
        p = vt[-1]
        dist = abs(p[:3] @ O + p[3]) / np.linalg.norm(p[:3])
        d = oracle.plane_distance(X, Y, Z, O)
        assert abs(d) == pytest.approx(dist, rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("ex", json.load(open(GOLDEN))["examples"], ids=lambda e: e["name"])
def test_worked_examples(ex):
    u = np.array(ex["u"], dtype=np.float64)
    kbar, d = oracle.direction_curvatures(u, 1, 1)
    np.testing.assert_allclose(d, ex["d"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(kbar, ex["kbar"], rtol=1e-12, atol=1e-14)
    assert oracle.curvature(u, 1, 1, oracle.MEAN) == pytest.approx(ex["H"], rel=1e-12, abs=1e-14)
    assert oracle.curvature(u, 1, 1, oracle.GAUSS) == pytest.approx(ex["K"], rel=1e-12, abs=1e-14)
    f = u.copy()
    f[1, 1] = ex["f_centre"]
    cm = oracle.paper_candidate(u, f, 1, 1, ex["alpha"], oracle.MEAN)
    cg = oracle.paper_candidate(u, f, 1, 1, ex["alpha"], oracle.GAUSS)
    assert cm == pytest.approx(ex["c_paper_mean"], rel=1e-12, abs=1e-14)
    assert cg == pytest.approx(ex["c_paper_gauss"], rel=1e-12, abs=1e-14)
    assert np.mean(d) == pytest.approx(ex["c_half_mean"], rel=1e-12, abs=1e-14)


def test_affine_images_have_zero_curvature():
    """A plane is a minimal, developable surface: every tangent-plane distance
    vanishes and H = K = 0 (Prop. 1 proof, Bernstein).  Dyadic slopes keep the
    arithmetic exact.  With the clamp-to-edge boundary reading the replicated
    border row/column is a kink, so this holds on interior pixels; a constant
    image is flat everywhere and has zero curvature energy."""
    y, x = np.mgrid[0:9, 0:11].astype(np.float64)
    for a, b, c in [(0.25, -0.5, 0.125), (2.0, 0.0, -1.0), (0.0, 0.0, 0.75), (-3.5, 1.25, 8.0)]:
        u = a * x + b * y + c
        for kind in ALL_KINDS:
            cmap = oracle.curvature_map(u, kind)
            assert np.all(cmap[1:-1, 1:-1] == 0.0)
            for r in range(1, 8):
                for cc in range(1, 10):
                    kbar, d = oracle.direction_curvatures(u, r, cc)
                    assert np.all(d == 0.0) and np.all(kbar == 0.0)
    const = np.full((9, 11), 0.625)
    for kind in ALL_KINDS:
        assert np.all(oracle.curvature_map(const, kind) == 0.0)
        assert oracle.energy(const, const, 3.0, kind) == 0.0


def sphere_cap(R, n):
    y, x = np.mgrid[-n:n + 1, -n:n + 1].astype(np.float64)
    return np.sqrt(R * R - x * x - y * y)


@pytest.mark.parametrize("kind", ALL_KINDS)
def test_sphere_cap_closed_form_and_order(kind):
    """Sphere of radius R (umbilic everywhere): |H| = 1/R, |K| = 1/R^2
    (Table I definitions).  The relative error must fall as (h/R)^2."""
    errs = []
    Rs = [10.0, 20.0, 40.0, 80.0]
    for R in Rs:
        n = int(R / 2) + 2
        u = sphere_cap(R, n)
        cmap = oracle.curvature_map(u, kind)
        yy, xx = np.mgrid[0:2 * n + 1, 0:2 * n + 1]
        m = ((yy - n) ** 2 + (xx - n) ** 2 <= (R / 2) ** 2)
        exact = 1.0 / R if kind in MEAN_KINDS else 1.0 / (R * R)
        # a cap bulging upward is concave: the sign convention gives H < 0, K > 0
        if kind in MEAN_KINDS:
            assert np.all(cmap[m] < 0)
        else:
            assert np.all(cmap[m] > 0)
        errs.append(np.max(np.abs(np.abs(cmap[m]) - exact)) / exact)
    assert errs[-1] < 2e-4
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for p in orders:
        assert 1.8 < p < 2.2, orders


def test_paraboloid_vertex():
    """z = (a x^2 + b y^2)/2 at the vertex: principal curvatures a and b along
    the axes.  For a = b (umbilic) the discrete values are exact; for a != b
    the error is second order in the curvature scale."""
    y, x = np.mgrid[-3:4, -3:4].astype(np.float64)
    for a in (0.5, 0.25, -0.75):
        u = 0.5 * a * (x * x + y * y)
        kbar, _ = oracle.direction_curvatures(u, 3, 3)
        np.testing.assert_allclose(kbar, [a] * 4, rtol=1e-13)
        for km, kg in ((oracle.MEAN, oracle.GAUSS), (oracle.MEAN_EULER, oracle.GAUSS_EULER)):
            assert oracle.curvature(u, 3, 3, km) == pytest.approx(a, rel=1e-13)
            assert oracle.curvature(u, 3, 3, kg) == pytest.approx(a * a, rel=1e-13)
    errs = []
    for s in (0.4, 0.2, 0.1, 0.05):
        a, b = 1.5 * s, 0.5 * s
        u = 0.5 * (a * x * x + b * y * y)
        H = oracle.curvature(u, 3, 3, oracle.MEAN)
        K = oracle.curvature(u, 3, 3, oracle.GAUSS)
        errs.append((abs(H - (a + b) / 2) / ((a + b) / 2), abs(K - a * b) / (a * b)))
    for i in range(len(errs) - 1):
        for j in range(2):
            p = math.log2(errs[i][j] / errs[i + 1][j])
            assert 1.8 < p < 2.2


def test_saddle_has_zero_mean_curvature_at_centre():
    """z = a (x^2 - y^2)/2: opposite principal curvatures, H = 0 at the vertex
    by symmetry; K < 0."""
    y, x = np.mgrid[-3:4, -3:4].astype(np.float64)
    u = 0.3 * (x * x - y * y)
    for km, kg in ((oracle.MEAN, oracle.GAUSS), (oracle.MEAN_EULER, oracle.GAUSS_EULER)):
        assert abs(oracle.curvature(u, 3, 3, km)) < 1e-15
        assert oracle.curvature(u, 3, 3, kg) < 0


def rotated_quadric(eps, k1, k2, phi):
    """z = eps (k1 x'^2 + k2 y'^2) with (x', y') the pixel axes rotated by
    phi: a critical point at the centre whose principal curvatures are the
    eigenvalues of the Hessian, 2 eps k1 and 2 eps k2, along axes at angle phi
    to the grid."""
    y, x = np.mgrid[-3:4, -3:4].astype(np.float64)
    xr = x * math.cos(phi) + y * math.sin(phi)
    yr = -x * math.sin(phi) + y * math.cos(phi)
    return eps * (k1 * xr * xr + k2 * yr * yr)


@pytest.mark.parametrize("k1,k2", [(1.0, 0.3), (1.0, -0.5), (0.8, 0.0), (-0.6, -0.2)])
def test_euler_fit_recovers_rotated_principal_curvatures(k1, k2):
    """Kinds MEAN_EULER / GAUSS_EULER: the least-squares fit of Euler's
    formula to the four direction curvatures returns H = eps (k1 + k2) and
    K = 4 eps^2 k1 k2 at the vertex of a quadric for ANY orientation of its
    principal axes, with an error that falls as eps^2 (the direction
    curvatures are normal curvatures, exact up to the slope terms).  The
    extreme sampled directions (kinds MEAN / GAUSS) give the right K only
    when the axes lie along sampled directions: a cylinder turned by 22.5
    degrees gets K != 0 from them, 0 from the fit."""
    for phi in (0.0, math.pi / 8, 0.7, math.pi / 4 + 0.1, 2.0):
        errs = []
        for eps in (1e-2, 1e-3):
            u = rotated_quadric(eps, k1, k2, phi)
            H = oracle.curvature(u, 3, 3, oracle.MEAN_EULER)
            K = oracle.curvature(u, 3, 3, oracle.GAUSS_EULER)
            Hx, Kx = eps * (k1 + k2), 4 * eps * eps * k1 * k2
            errs.append((abs(H - Hx), abs(K - Kx)))
            assert H == pytest.approx(Hx, rel=1e-3, abs=1e-3 * eps * abs(k1))
            assert K == pytest.approx(Kx, rel=1e-3, abs=1e-3 * eps * eps * k1 * k1)
        # second order: a factor 10 in eps is a factor ~1000 in the error of H
        # (relative error ~eps^2) and of K (~eps^4 absolute)
        assert errs[1][0] <= errs[0][0] * 2e-3 + 1e-18
        assert errs[1][1] <= errs[0][1] * 2e-4 + 1e-22
    u = rotated_quadric(1e-3, 1.0, 0.0, math.pi / 8)   # cylinder at 22.5 degrees
    assert abs(oracle.curvature(u, 3, 3, oracle.GAUSS_EULER)) < 1e-11
    # extreme sampled directions: 2 eps cos^2(22.5 deg) and 2 eps sin^2(22.5 deg),
    # product eps^2 / 2
    assert oracle.curvature(u, 3, 3, oracle.GAUSS) == pytest.approx(0.5e-6, rel=1e-3)


def test_translation_and_d4_invariance():
    """F(u) is invariant under adding a constant to u and f (plane distances
    depend on differences only) and under the eight symmetries of the square
    (the plane set is closed under them)."""
    rng = np.random.default_rng(3)
    u = rng.random((13, 17))
    f = rng.random((13, 17))
    for kind in ALL_KINDS:
        E = oracle.energy(u, f, 7.0, kind)
        assert oracle.energy(u + 0.37, f + 0.37, 7.0, kind) == pytest.approx(E, rel=1e-12)
        for k in range(4):
            for flip in (False, True):
                v, g = np.rot90(u, k), np.rot90(f, k)
                if flip:
                    v, g = v[:, ::-1], g[:, ::-1]
                assert oracle.energy(v, g, 7.0, kind) == pytest.approx(E, rel=1e-12)
        # curvature map commutes with a transpose
        np.testing.assert_allclose(oracle.curvature_map(u.T, kind),
                                   oracle.curvature_map(u, kind).T, rtol=1e-12, atol=1e-14)


def test_energy_is_sum_of_pixel_terms():
    """Eq. (MCM)/(GCM): F is the plain sum of |kappa| + alpha/2 (u - f)^2;
    a constant image has zero curvature energy and only the fidelity term."""
    rng = np.random.default_rng(4)
    u = rng.random((6, 7))
    f = rng.random((6, 7))
    for kind in ALL_KINDS:
        cmap = oracle.curvature_map(u, kind)
        ref = np.sum(np.abs(cmap)) + 0.5 * 5.0 * np.sum((u - f) ** 2)
        assert oracle.energy(u, f, 5.0, kind) == pytest.approx(ref, rel=1e-13)
        c = np.full((6, 7), 0.3)
        assert oracle.energy(c, f, 5.0, kind) == pytest.approx(2.5 * np.sum((0.3 - f) ** 2),
                                                             rel=1e-13)


def test_clamped_boundary_reading():
    """Clamp-to-edge: a one-row image sees its N and S neighbours equal to
    itself, so only the W-E line can bend; a 1x1 image is flat."""
    u = np.array([[0.0, 1.0, 0.0, 2.0]])
    kbar, d = oracle.direction_curvatures(u, 0, 1)
    # N = S = O: the N-S line is flat
    assert kbar[1] == 0.0
    # W-E: delta = (0 + 0)/2 - 1 = -1 < 0 (a peak)
    assert kbar[0] < 0
    one = np.array([[0.4]])
    assert oracle.curvature(one, 0, 0, oracle.MEAN) == 0.0


def test_euler_fit_is_the_closed_form_of_the_four_directions():
    """At the sampled angles 0, 90, 45 and 135 degrees the columns
    (1, cos 2theta, sin 2theta) of the least-squares design are orthogonal,
    so the fit of kappa(theta) = a + b cos 2theta + s sin 2theta has the
    closed form a = (k0 + k1 + k2 + k3)/4, b = (k0 - k1)/2, s = (k2 - k3)/2
    (numpy's least squares agrees), and the principal curvatures a -+
    sqrt(b^2 + s^2) give H = a, K = a^2 - b^2 - s^2.  The oracle's kinds 2
    and 3 (normal equations from the lines' angles, Gauss-Jordan) match it
    on every pixel of random images, borders included."""
    X = np.array([[1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1]], dtype=float)
    rng = np.random.default_rng(12)
    for trial in range(3):
        u = rng.random((7, 9)) * (0.2 + trial)
        for r in range(7):
            for c in range(9):
                kbar, _ = oracle.direction_curvatures(u, r, c)
                a, b, s = np.linalg.lstsq(X, kbar, rcond=None)[0]
                assert a == pytest.approx(kbar.sum() / 4, abs=1e-12)
                assert b == pytest.approx((kbar[0] - kbar[1]) / 2, abs=1e-12)
                assert s == pytest.approx((kbar[2] - kbar[3]) / 2, abs=1e-12)
                H = oracle.curvature(u, r, c, oracle.MEAN_EULER)
                K = oracle.curvature(u, r, c, oracle.GAUSS_EULER)
                scale = 1.0 + np.max(np.abs(kbar)) ** 2
                assert abs(H - a) <= 1e-12 * scale
                assert abs(K - (a * a - b * b - s * s)) <= 1e-12 * scale
