"""Property-based pins of the oracle (hypothesis, deterministic draws): the
identities of the fixed-example pins, drawn over random images, blocks,
shifts and all four curvature kinds, and the reconstruction operators'
adjoint identities over random shapes, masks and angle counts."""
import math

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402

KINDS = st.sampled_from([oracle.MEAN, oracle.GAUSS, oracle.MEAN_EULER, oracle.GAUSS_EULER])


@st.composite
def images(draw, min_side=1, max_side=9):
    H = draw(st.integers(min_side, max_side))
    W = draw(st.integers(min_side, max_side))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    return rng.random((H, W)), rng.random((H, W))


@settings(max_examples=60, deadline=None, derandomize=True)
@given(images(), KINDS, st.data())
def test_local_energy_is_the_energy_difference(img, kind, data):
    """E_A(c) - E_A(0) = F(u + c 1_A) - F(u) for any block A and shift c: the
    ring holds every pixel whose stencil sees A (Sec. 2.2)."""
    u, f = img
    H, W = u.shape
    r0 = data.draw(st.integers(0, H - 1))
    c0 = data.draw(st.integers(0, W - 1))
    bh = data.draw(st.integers(1, H - r0))
    bw = data.draw(st.integers(1, W - c0))
    c = data.draw(st.floats(-0.5, 0.5))
    alpha = data.draw(st.floats(0.5, 30.0))
    v = u.copy()
    v[r0:r0 + bh, c0:c0 + bw] += c
    dF = oracle.energy(v, f, alpha, kind) - oracle.energy(u, f, alpha, kind)
    dE = (oracle.local_energy(u, f, r0, c0, bh, bw, c, alpha, kind)
          - oracle.local_energy(u, f, r0, c0, bh, bw, 0.0, alpha, kind))
    scale = 1.0 + abs(oracle.energy(u, f, alpha, kind))
    assert abs(dF - dE) <= 1e-10 * scale


@settings(max_examples=40, deadline=None, derandomize=True)
@given(images(2, 10), KINDS, st.floats(-2.0, 2.0), st.integers(0, 7))
def test_energy_invariances(img, kind, shift, sym):
    """F(u + t, f + t) = F(u, f), and F is unchanged under the eight
    symmetries of the square (the tangent-plane set is closed under them)."""
    u, f = img
    E = oracle.energy(u, f, 7.0, kind)
    assert oracle.energy(u + shift, f + shift, 7.0, kind) == pytest.approx(E, rel=1e-11, abs=1e-12)
    v, g = np.rot90(u, sym % 4), np.rot90(f, sym % 4)
    if sym >= 4:
        v, g = v[:, ::-1], g[:, ::-1]
    assert oracle.energy(v.copy(), g.copy(), 7.0, kind) == pytest.approx(E, rel=1e-11)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(st.floats(-1.0, 1.0), st.floats(-1.0, 1.0), st.floats(0.0, math.pi))
def test_euler_fit_on_random_quadrics(k1, k2, phi):
    """Kinds 2 and 3 recover H = eps (k1 + k2) and K = 4 eps^2 k1 k2 at the
    vertex of a quadric with principal axes at any angle."""
    eps = 1e-3
    y, x = np.mgrid[-3:4, -3:4].astype(np.float64)
    xr = x * math.cos(phi) + y * math.sin(phi)
    yr = -x * math.sin(phi) + y * math.cos(phi)
    u = eps * (k1 * xr * xr + k2 * yr * yr)
    H = oracle.curvature(u, 3, 3, oracle.MEAN_EULER)
    K = oracle.curvature(u, 3, 3, oracle.GAUSS_EULER)
    assert abs(H - eps * (k1 + k2)) <= 1e-5 * eps + 1e-4 * eps * abs(k1 + k2)
    # the direction curvatures carry O(eps^3) slope terms: K is exact to O(eps^4)
    assert abs(K - 4 * eps * eps * k1 * k2) <= 1e-4 * eps * eps


@settings(max_examples=30, deadline=None, derandomize=True)
@given(images(3, 8), KINDS, st.data())
def test_block_search_never_raises_the_local_energy(img, kind, data):
    """The chosen shift's local energy is never above that of c = 0, whatever
    the budget (the c = 0 candidate is always evaluated)."""
    u, f = img
    H, W = u.shape
    b = data.draw(st.sampled_from([1, 2, 3]))
    r0 = data.draw(st.integers(0, H - 1))
    c0 = data.draw(st.integers(0, W - 1))
    bh, bw = min(b, H - r0), min(b, W - c0)
    G = data.draw(st.sampled_from([3, 5, 9]))
    K = data.draw(st.integers(2, 8))
    c, _ = oracle.block_min(u, f, r0, c0, bh, bw, 15.0, kind, G=G, K=K)
    E0 = oracle.local_energy(u, f, r0, c0, bh, bw, 0.0, 15.0, kind)
    Ec = oracle.local_energy(u, f, r0, c0, bh, bw, c, 15.0, kind)
    assert Ec <= E0 + 1e-12 * (1.0 + abs(E0))


@settings(max_examples=40, deadline=None, derandomize=True)
@given(images(1, 12), st.integers(1, 40), st.integers(0, 2 ** 31 - 1))
def test_radon_pair_is_adjoint_and_keeps_mass(img, n, seed):
    """<R u, y> = <u, R^T y>, and every angle's projection sums to the image's
    sum, for any shape and angle count (every p lies inside the detector)."""
    from oracle import recon
    u, _ = img
    H, W = u.shape
    D = recon.radon_geometry(H, W, n)[0]
    y = np.random.default_rng(seed).normal(size=(n, D))
    Ru = recon.radon_forward(u, n)
    assert np.sum(Ru * y) == pytest.approx(np.sum(u * recon.radon_adjoint(y, H, W)),
                                           rel=1e-10, abs=1e-10)
    np.testing.assert_allclose(Ru.sum(axis=1), u.sum(), rtol=1e-12)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(images(1, 12), st.floats(0.05, 1.0), st.integers(0, 2 ** 31 - 1))
def test_mri_operator_is_adjoint_and_contractive(img, frac, seed):
    from oracle import recon
    u, _ = img
    H, W = u.shape
    rng = np.random.default_rng(seed)
    mask = (rng.random((H, W)) < frac).astype(float)
    y = rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))
    Au = recon.forward(u, mask)
    assert np.vdot(y, Au) == pytest.approx(np.vdot(recon.adjoint(y, mask), u), rel=1e-10,
                                           abs=1e-10)
    assert np.linalg.norm(Au) <= np.linalg.norm(u) * (1 + 1e-12)
