"""Pins of the reconstruction oracle (Sec. 5: MRI-like operator A = M F, and
CT with a parallel-beam Radon transform).

The MRI operator is pinned by its adjoint identity and Parseval, the Radon
pair by its adjoint identity, mass per angle, the theta = 0 column sums,
each projection's first moment (the projected centroid, exact) and the
analytic projection of an off-centre Gaussian,
the filtered backprojection by the Ram-Lak kernel's zero DC gain and a
densely sampled phantom; the per-colour
correction by a closed form (full mask: the Gram matrix is diagonal) and by
a dense linear solve of the assembled normal equations; the sweep by
monotone descent of the data term when the regulariser vanishes, and by
descent and denoising on an undersampled case.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import recon


def test_operator_adjoint_and_parseval():
    rng = np.random.default_rng(0)
    H, W = 12, 10
    mask = (rng.random((H, W)) < 0.4).astype(float)
    u = rng.normal(size=(H, W))
    y = rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))
    # <A u, y> = <u, A^H y> (complex inner products; u real)
    lhs = np.vdot(y, recon.forward(u, mask))
    rhs = np.vdot(recon.adjoint(y, mask), u)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # orthonormal DFT: ||F u|| = ||u||; the mask can only shrink it
    full = np.ones((H, W))
    assert np.linalg.norm(recon.forward(u, full)) == pytest.approx(np.linalg.norm(u), rel=1e-12)
    assert np.linalg.norm(recon.forward(u, mask)) < np.linalg.norm(u)
    # the DC entry of F u is sum(u) / sqrt(H W)
    assert recon.forward(u, full)[0, 0] == pytest.approx(u.sum() / np.sqrt(H * W), rel=1e-12)


def test_colour_labels_cover_the_colour():
    H, W, b = 13, 10, 3
    for k in range(4):
        lab, n = recon.colour_labels(H, W, b, 4, k)
        seen = set()
        for r in range(H):
            for c in range(W):
                bi, bj = r // b, c // b
                if oracle.block_colour(bi, bj, 4) == k:
                    assert lab[r, c] >= 0
                    seen.add(int(lab[r, c]))
                else:
                    assert lab[r, c] == -1
        assert seen == set(range(n))


@pytest.mark.parametrize("b", [1, 2, 4])
def test_full_mask_step_is_the_diagonal_closed_form(b):
    """With every k-space entry sampled, A^H A = I, so <A phi_i, A phi_j> =
    s_i delta_ij (disjoint blocks of s_i pixels) and each block's shift is
    c_i = (<b - A u, A phi_i> + 2 alpha d_i) / (s_i + 2 alpha)."""
    case = synth.mri_case(20, 17, 3, accel=1.0, sigma=0.02)
    assert case.mask.all()
    mask = case.mask.astype(float)
    kspace = case.kspace.astype(complex)
    u = np.real(recon.adjoint(kspace, mask)) + 0.05 * np.sin(np.arange(20 * 17)).reshape(20, 17)
    alpha = 0.3
    for k in range(4):
        _, c = recon.colour_step(u, kspace, mask, alpha, oracle.MEAN, b, 4, k, cg_iters=20)
        lab, n = recon.colour_labels(20, 17, b, 4, k)
        g = np.real(recon.adjoint(kspace - recon.forward(u, mask), mask))
        d = oracle.chalf_map(u, oracle.MEAN) if b == 1 else np.zeros_like(u)
        for i in range(n):
            blk = lab == i
            s = blk.sum()
            di = d[blk].sum() if b == 1 else 0.0
            want = (g[blk].sum() + 2 * alpha * di) / (s + 2 * alpha)
            assert c[i] == pytest.approx(want, rel=1e-9, abs=1e-12)


def test_cg_equals_dense_normal_equations():
    """Undersampled mask: assemble the Gram matrix column by column from A
    applied to every block indicator, solve it densely, and compare with the
    colour step's CG run to n iterations (exact in exact arithmetic)."""
    case = synth.mri_case(12, 10, 5, accel=2.5, sigma=0.02)
    mask = case.mask.astype(float)
    kspace = case.kspace.astype(complex)
    u = np.real(recon.adjoint(kspace, mask))
    alpha = 0.05
    b, k = 2, 1
    lab, n = recon.colour_labels(12, 10, b, 4, k)
    G = np.zeros((n, n))
    Aphi = [recon.forward((lab == i).astype(float), mask) for i in range(n)]
    for i in range(n):
        for j in range(n):
            G[i, j] = np.real(np.vdot(Aphi[i], Aphi[j]))
    res = kspace - recon.forward(u, mask)
    rhs = np.array([np.real(np.vdot(Aphi[i], res)) for i in range(n)])
    c_dense = np.linalg.solve(G + 2 * alpha * np.eye(n), rhs)
    _, c = recon.colour_step(u, kspace, mask, alpha, oracle.MEAN, b, 4, k, cg_iters=n)
    np.testing.assert_allclose(c, c_dense, rtol=1e-8, atol=1e-10)


def test_vanishing_regulariser_never_raises_the_data_term():
    """alpha -> 0: each colour step minimises 1/2 ||A u - b||^2 exactly over
    its blocks' span (CG run to convergence), so the data term never rises."""
    case = synth.mri_case(24, 20, 9, accel=3.0, sigma=0.02)
    mask = case.mask.astype(float)
    kspace = case.kspace.astype(complex)
    u = np.real(recon.adjoint(kspace, mask))
    data = lambda v: 0.5 * np.sum(np.abs(recon.forward(v, mask) - kspace) ** 2)
    prev = data(u)
    for j in range(1, 4):
        b = oracle.level_side(j)
        for k in range(4):
            lab, n = recon.colour_labels(24, 20, b, 4, k)
            u, _ = recon.colour_step(u, kspace, mask, 1e-9, oracle.MEAN, b, 4, k,
                                     cg_iters=n + 2)
            cur = data(u)
            assert cur <= prev * (1 + 1e-9) + 1e-15
            prev = cur


def test_reconstruction_descends_and_denoises():
    case = synth.mri_case(64, 64, 7, accel=3.0, sigma=0.01)
    u0 = np.real(recon.adjoint(case.kspace.astype(complex), case.mask.astype(float)))
    u, trace = recon.solve(case.kspace, case.mask, 0.02, oracle.MEAN, cycles=4, cg_iters=8)
    assert np.all(np.diff(trace) < 0)
    assert synth.psnr(u, case.clean) > synth.psnr(u0, case.clean) + 1.0


# ---------------------------------------------------------------------------
# CT: parallel-beam Radon transform with linear-interpolation weights.

def test_radon_pair_adjoint_mass_and_columns():
    rng = np.random.default_rng(2)
    H, W, n = 13, 9, 17
    u = rng.normal(size=(H, W))
    y = rng.normal(size=(n, recon.radon_geometry(H, W, n)[0]))
    Ru = recon.radon_forward(u, n)
    assert np.sum(Ru * y) == pytest.approx(np.sum(u * recon.radon_adjoint(y, H, W)), rel=1e-12)
    # every angle's projection carries the image's sum (weights 1 - w, w)
    np.testing.assert_allclose(Ru.sum(axis=1), u.sum(), rtol=1e-12)
    # theta = 0 with an odd width: each column falls on one bin, at the centre
    D = Ru.shape[1]
    h = (D - 1) // 2
    np.testing.assert_allclose(Ru[0, h - (W - 1) // 2: h + (W - 1) // 2 + 1], u.sum(axis=0),
                               rtol=1e-12)
    assert np.all(Ru[0, :h - (W - 1) // 2] == 0) and np.all(Ru[0, h + (W - 1) // 2 + 1:] == 0)


def test_ramp_filter_and_fbp():
    """The Ram-Lak kernel sums to zero (no DC gain: a constant projection is
    filtered to ~0 away from the detector's ends), and filtered
    backprojection of a densely sampled phantom recovers it."""
    row = np.ones((1, 101))
    f = recon.ramp_filter(row)[0]
    assert np.max(np.abs(f[40:61])) < 0.01
    clean = synth.piecewise_image(32, 32, 5, 6, 0.0).clean.astype(np.float64)
    u = recon.fbp(recon.radon_forward(clean, 90), 32, 32)
    assert synth.psnr(u, clean) > 24.0


def test_ct_step_equals_dense_normal_equations():
    H, W, n = 10, 9, 12
    rng = np.random.default_rng(4)
    clean = synth.piecewise_image(H, W, 3, 3, 0.0).clean.astype(np.float64)
    sino = recon.radon_forward(clean, n) + 0.05 * rng.normal(size=(n, recon.radon_geometry(H, W, n)[0]))
    u = recon.fbp(sino, H, W)
    op = recon.CtOp(H, W, n)
    alpha, b, k = 0.3, 2, 2
    lab, m = recon.colour_labels(H, W, b, 4, k)
    Aphi = [op.fwd((lab == i).astype(float)) for i in range(m)]
    G = np.array([[np.sum(Aphi[i] * Aphi[j]) for j in range(m)] for i in range(m)])
    res = sino - op.fwd(u)
    rhs = np.array([np.sum(Aphi[i] * res) for i in range(m)])
    c_dense = np.linalg.solve(G + 2 * alpha * np.eye(m), rhs)
    _, c = recon.colour_step_op(u, sino, op, alpha, oracle.MEAN, b, 4, k, cg_iters=m)
    np.testing.assert_allclose(c, c_dense, rtol=1e-7, atol=1e-9)


def test_ct_reconstruction_improves_on_fbp():
    clean = synth.piecewise_image(32, 32, 5, 6, 0.0).clean.astype(np.float64)
    n = 45
    rng = np.random.default_rng(1)
    sino = recon.radon_forward(clean, n)
    sino = sino + 0.1 * rng.normal(size=sino.shape)
    u0 = recon.fbp(sino, 32, 32)
    u, trace = recon.solve_ct(sino, 32, 32, 1.0, oracle.MEAN, cycles=4, cg_iters=8)
    assert np.all(np.diff(trace) < 0)
    assert synth.psnr(u, clean) > synth.psnr(u0, clean) + 1.5


@pytest.mark.parametrize("shape,n", [((13, 9), 17), ((8, 15), 12), ((1, 7), 5)])
def test_radon_first_moment_is_the_projected_centroid(shape, n):
    """Linear interpolation keeps the first moment of each pixel's mass
    ((1 - w) f + w (f + 1) = p), so every angle's projection has its centroid
    at t0 + (D - 1)/2 with t0 = x0 cos theta + y0 sin theta, (x0, y0) the
    image's centroid about the centre.  An off-centre mass fixes the sign
    and orientation of both terms at every angle."""
    H, W = shape
    rng = np.random.default_rng(H * 31 + W)
    u = rng.random((H, W)) * np.exp(np.arange(W) / W)[None, :]
    Ru = recon.radon_forward(u, n)
    D = Ru.shape[1]
    y, x = np.mgrid[0:H, 0:W]
    x0 = np.sum(u * (x - (W - 1) / 2.0)) / u.sum()
    y0 = np.sum(u * (y - (H - 1) / 2.0)) / u.sum()
    th = np.pi * np.arange(n) / n
    want = x0 * np.cos(th) + y0 * np.sin(th) + (D - 1) / 2.0
    got = Ru @ np.arange(D) / Ru.sum(axis=1)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


def test_radon_of_a_gaussian_is_the_analytic_projection():
    """The Radon transform of exp(-|z - z0|^2 / (2 s^2)) is
    s sqrt(2 pi) exp(-(t - t0)^2 / (2 s^2)) at every angle.  At theta = 0 and
    pi/2 every pixel lands on a bin (odd W and H), so the bins sample the
    projection: the pixel sum of a Gaussian of s = 3 equals its integral to
    ~1e-7 of the peak.  At other angles the linear-interpolation splat of
    pixel-driven projection ripples: at 45 degrees the pixel positions lie
    1/sqrt(2) apart and the hat weights each bin collects sum to between
    0.914 and 1.121 of their mean, so the bins stay within 13% of the
    analytic projection's peak (a one-bin centring error alone would exceed
    0.2 of it at theta = 0)."""
    H, W, n, s = 41, 45, 12, 3.0
    x0, y0 = 5.3, -4.1
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    u = np.exp(-((x - (W - 1) / 2 - x0) ** 2 + (y - (H - 1) / 2 - y0) ** 2) / (2 * s * s))
    Ru = recon.radon_forward(u, n)
    D = Ru.shape[1]
    t = np.arange(D) - (D - 1) / 2.0
    peak = s * np.sqrt(2 * np.pi)
    for a in range(n):
        th = np.pi * a / n
        t0 = x0 * np.cos(th) + y0 * np.sin(th)
        want = peak * np.exp(-(t - t0) ** 2 / (2 * s * s))
        tol = 1e-6 if a in (0, n // 2) else 0.13
        assert np.max(np.abs(Ru[a] - want)) < tol * peak, a
