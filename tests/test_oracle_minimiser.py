"""Pins of the oracle's block subproblem (Sec. 2.2, Alg. 3) and sweep.

The ring-only local energy is pinned to the full energy difference, the
block search to brute force (and, handed its ring sum by the caller, to
itself on the whole image), the phase to its snapshot definition, and the
whole sweep to monotone descent in sequential (Gauss-Seidel) order.
"""
import numpy as np
import pytest

import oracle
import synth

KINDS = [oracle.MEAN, oracle.GAUSS, oracle.MEAN_EULER, oracle.GAUSS_EULER]


def rand_img(H, W, seed, smooth=True):
    rng = np.random.default_rng(seed)
    u = rng.random((H, W))
    if smooth:
        y, x = np.mgrid[0:H, 0:W]
        u = 0.5 + 0.3 * np.sin(0.7 * x + 0.4 * y) + 0.05 * rng.normal(size=(H, W))
    return u


def blocks_of(H, W, b):
    for bi in range((H + b - 1) // b):
        for bj in range((W + b - 1) // b):
            yield bi, bj, bi * b, bj * b, min(b, H - bi * b), min(b, W - bj * b)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("b", [1, 2, 3, 4, 5])
def test_local_energy_equals_full_energy_difference(kind, b):
    """E_A(c) - E_A(0) = F(u + c phi_A) - F(u): the ring holds every pixel whose
    curvature moves, with the clamped boundary, for blocks clipped at edges."""
    H, W = 11, 13
    u = rand_img(H, W, 10 + b, smooth=False)
    f = rand_img(H, W, 20 + b, smooth=False)
    alpha = 3.0
    F0 = oracle.energy(u, f, alpha, kind)
    for _, _, r0, c0, bh, bw in blocks_of(H, W, b):
        for c in (-0.3, 0.05, 0.7):
            v = u.copy()
            v[r0:r0 + bh, c0:c0 + bw] += c
            dF = oracle.energy(v, f, alpha, kind) - F0
            dE = (oracle.local_energy(u, f, r0, c0, bh, bw, c, alpha, kind)
                  - oracle.local_energy(u, f, r0, c0, bh, bw, 0.0, alpha, kind))
            assert dE == pytest.approx(dF, rel=1e-10, abs=1e-10 * max(1.0, abs(F0)))


def test_ring_sizes():
    """Ring of an interior block: 9 pixels for b = 1, 16 for b = 2, 8b for
    b >= 3 (frame of width one on each side of the block boundary)."""
    H = W = 40
    assert oracle.ring_size(H, W, 10, 10, 1, 1) == 9
    assert oracle.ring_size(H, W, 10, 10, 2, 2) == 16
    for b in (3, 4, 8, 16):
        assert oracle.ring_size(H, W, 8, 8, b, b) == 8 * b
    # corner block b = 4: outside, row 4 (5 px) and column 4 (4 px); inside,
    # row 3 and column 3 (7 px).  Row/column 0 clamp onto themselves, so
    # their pixels stay interior.
    assert oracle.ring_size(H, W, 0, 0, 4, 4) == (4 + 1) + 4 + (2 * 4 - 1)


@pytest.mark.parametrize("kind", KINDS)
def test_bracket_contains_minimiser(kind):
    """Every c outside [c_fid - rho, c_fid + rho] has E_A(c) > E_A(c_fid)."""
    H, W = 10, 10
    u = rand_img(H, W, 5)
    f = u + 0.1 * np.random.default_rng(6).normal(size=(H, W))
    alpha = 4.0
    for b in (1, 2, 4):
        for _, _, r0, c0, bh, bw in list(blocks_of(H, W, b))[:6]:
            c, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind)
            cf, rho = info["c_fid"], info["rho"]
            Ef = oracle.local_energy(u, f, r0, c0, bh, bw, cf, alpha, kind)
            out = np.concatenate([cf - rho * np.linspace(1.001, 6.0, 60),
                                  cf + rho * np.linspace(1.001, 6.0, 60)])
            E = oracle.local_energy_batch(u, f, r0, c0, bh, bw, out, alpha, kind)
            assert np.all(E > Ef)


def _brute_force(u, f, r0, c0, bh, bw, alpha, kind, cf, rho):
    """Global minimum of E_A on the bracket by grid search (20001 points) and
    a 2001-point refinement around the best grid point.  Also returns the
    largest |dE_A/dc| next to the optimum and the number of local minima of
    the sampled curve."""
    grid = np.linspace(cf - rho, cf + rho, 20001)
    E = oracle.local_energy_batch(u, f, r0, c0, bh, bw, grid, alpha, kind)
    i = int(np.argmin(E))
    step = grid[1] - grid[0]
    fine = np.linspace(grid[i] - step, grid[i] + step, 2001)
    Ef = oracle.local_energy_batch(u, f, r0, c0, bh, bw, fine, alpha, kind)
    j = int(np.argmin(Ef))
    slope = np.max(np.abs(np.diff(Ef))) / (fine[1] - fine[0])
    n_min = int(np.sum((E[1:-1] < E[:-2]) & (E[1:-1] < E[2:])))
    if Ef[j] < E[i]:
        return fine[j], Ef[j], slope, n_min
    return grid[i], E[i], slope, n_min


def _bf_cases(kind, side=8, seeds=(77,)):
    for seed in seeds:
        img = synth.piecewise_image(side, side, seed + kind, 3 if side == 8 else 5, 0.08)
        f = img.f.astype(np.float64)
        u = oracle.cycle(f.copy(), f, 20.0, kind, levels=1)   # move away from u = f
        for b in (1, 2, 4):
            for _, _, r0, c0, bh, bw in blocks_of(side, side, b):
                yield u, f, r0, c0, bh, bw


@pytest.mark.parametrize("kind", KINDS)
def test_block_min_against_brute_force_long_search(kind):
    """16x16 images, every block of b = 1, 2, 4, golden search of K = 40
    evaluations.  Where E_A has a single local minimum on the bracket the pick
    equals the brute-force optimum to 1e-6 |E_A| on every block; over all
    blocks it does on >= 97% (the misses are narrow notches of the
    non-smooth |kappa| terms that fall between grid points); it is never
    worse than c = 0."""
    alpha = 20.0
    gaps, uni = [], []
    for u, f, r0, c0, bh, bw in _bf_cases(kind, side=16, seeds=(77, 78)):
        c, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind, G=9, K=40)
        assert info["E_best"] <= info["E_zero"]
        if info["rho"] == 0:
            continue
        _, Ebf, _, n_min = _brute_force(u, f, r0, c0, bh, bw, alpha, kind, info["c_fid"],
                                        info["rho"])
        gaps.append((info["E_best"] - Ebf) / max(abs(Ebf), 1e-12))
        uni.append(n_min == 1)
    gaps, uni = np.array(gaps), np.array(uni)
    assert uni.sum() > 0.5 * len(uni)
    assert np.all(gaps[uni] <= 1e-6), np.sort(gaps[uni])[-3:]
    assert np.mean(gaps <= 1e-6) >= 0.97, np.sort(gaps)[-5:]


@pytest.mark.parametrize("kind", KINDS)
def test_block_min_default_budget_within_resolution(kind):
    """Default budget (G, K): the golden search ends on a bracket of width
    w = 2 D phi^(K-2), D the grid step, which holds the minimiser when E_A is
    unimodal; the best evaluated point is then within w of it, so its energy
    exceeds the brute-force optimum by at most slope * w, slope = the largest
    |dE_A/dc| within w of the optimum.  That holds on every unimodal block
    and on >= 97% of all blocks; c = 0 is never beaten by the pick."""
    alpha = 20.0
    phi = (5 ** 0.5 - 1) / 2
    G, K = oracle.DEFAULT_G, oracle.DEFAULT_K
    ok, uni = [], []
    for u, f, r0, c0, bh, bw in _bf_cases(kind, side=16, seeds=(77,)):
        c, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind)
        assert info["E_best"] <= info["E_zero"]
        if info["rho"] == 0:
            continue
        cbf, Ebf, _, n_min = _brute_force(u, f, r0, c0, bh, bw, alpha, kind,
                                          info["c_fid"], info["rho"])
        w = 2 * (2 * info["rho"] / (G - 1)) * phi ** (K - 2)
        cs = np.linspace(cbf - w, cbf + w, 4001)
        Es = oracle.local_energy_batch(u, f, r0, c0, bh, bw, cs, alpha, kind)
        slope = np.max(np.abs(np.diff(Es))) / (cs[1] - cs[0])
        ok.append(info["E_best"] - Ebf <= slope * w + 1e-12)
        uni.append(n_min == 1)
    ok, uni = np.array(ok), np.array(uni)
    assert np.all(ok[uni])
    assert np.mean(ok) >= 0.97


def test_fidelity_limit_returns_block_mean():
    """alpha -> infinity: the curvature term is negligible and c -> c_fid,
    the block mean of f - u (the paper's f*)."""
    u = rand_img(8, 8, 8)
    f = rand_img(8, 8, 9, smooth=False)
    for kind in KINDS:
        for b in (1, 2, 4):
            c, info = oracle.block_min(u, f, 0, 0, b, b, 1e9, kind)
            assert c == pytest.approx(info["c_fid"], abs=1e-6)
            assert c == pytest.approx(np.mean(f[:b, :b] - u[:b, :b]), abs=1e-6)


def test_constant_image_is_fixed_point():
    """u = f = constant: zero curvature, S1 = 0, bracket of width 0; every
    block returns exactly 0 and the cycle leaves u unchanged."""
    u = np.full((9, 12), 0.4)
    for kind in KINDS:
        v = oracle.cycle(u, u, 10.0, kind, levels=0)
        assert np.array_equal(v, u)


@pytest.mark.parametrize("kind", KINDS)
def test_sequential_updates_never_raise_energy(kind):
    """Gauss-Seidel order (one block at a time): F(u + c phi_A) <= F(u) after
    every single update (Alg. 3 with |I_k| = 1), checked with the full F."""
    img = synth.piecewise_image(12, 12, 31 + kind, 4, 0.1)
    f = img.f.astype(np.float64)
    u = f.copy()
    alpha = 15.0
    F = oracle.energy(u, f, alpha, kind)
    for b in (1, 2, 4, 8):
        for _, _, r0, c0, bh, bw in blocks_of(12, 12, b):
            c, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind)
            u[r0:r0 + bh, c0:c0 + bw] += c
            Fn = oracle.energy(u, f, alpha, kind)
            assert Fn <= F + 1e-12 * abs(F)
            assert Fn - F == pytest.approx(info["E_best"] - info["E_zero"], abs=1e-10 * abs(F))
            F = Fn
    # and the oracle's own sequential level routine does the same thing
    u2 = f.copy()
    for b in (1, 2, 4, 8):
        u2 = oracle.level_sequential(u2, f, alpha, kind, b)
    np.testing.assert_allclose(u2, u, rtol=0, atol=1e-12)


@pytest.mark.parametrize("ncolors", [2, 4])
def test_phase_is_snapshot_of_block_solves(ncolors):
    """A phase = every block of the colour solved from the phase-start state,
    then all applied (Sec. 2.3 read with snapshot semantics); blocks of other
    colours are untouched; each block's own local energy does not rise."""
    img = synth.piecewise_image(10, 14, 5, 4, 0.1)
    f = img.f.astype(np.float64)
    u = oracle.cycle(f, f, 12.0, oracle.MEAN, levels=1)
    for b in (1, 2, 4):
        for k in range(ncolors):
            un, cs = oracle.phase(u, f, 12.0, oracle.MEAN, b, ncolors, k)
            nbj = (14 + b - 1) // b
            for bi, bj, r0, c0, bh, bw in blocks_of(10, 14, b):
                blk = un[r0:r0 + bh, c0:c0 + bw] - u[r0:r0 + bh, c0:c0 + bw]
                if oracle.block_colour(bi, bj, ncolors) != k:
                    assert np.all(blk == 0)
                    continue
                c, info = oracle.block_min(u, f, r0, c0, bh, bw, 12.0, oracle.MEAN)
                assert cs[bi * nbj + bj] == c
                np.testing.assert_allclose(blk, c, rtol=0, atol=1e-15)
                assert info["E_best"] <= info["E_zero"]


def test_colour_assignment():
    """Two colours: checkerboard of blocks; four colours: the paper's 2x2
    parity classes, so 4-neighbouring blocks differ in colour (Sec. 2.3)."""
    for ncolors in (2, 4):
        for bi in range(6):
            for bj in range(6):
                k = oracle.block_colour(bi, bj, ncolors)
                assert 0 <= k < ncolors
                assert oracle.block_colour(bi + 1, bj, ncolors) != k
                assert oracle.block_colour(bi, bj + 1, ncolors) != k
    assert oracle.block_colour(0, 0, 2) == 0 and oracle.block_colour(1, 1, 2) == 0
    assert {oracle.block_colour(i, j, 4) for i in (0, 1) for j in (0, 1)} == {0, 1, 2, 3}


def test_auto_levels():
    """Block sides 1, 2, 4, ... up to the largest power of two <= min(H, W)/2."""
    assert oracle.auto_levels(64, 64) == 6
    assert oracle.auto_levels(512, 512) == 9
    assert oracle.auto_levels(1024, 1024) == 10
    assert oracle.auto_levels(2048, 2048) == 11
    assert oracle.auto_levels(1, 100) == 1
    assert oracle.auto_levels(3, 3) == 1
    assert oracle.auto_levels(4, 9) == 2


# ---------------------------------------------------------------------------
# Single-step mode (one step of Alg. 2 per block, kept if it lowers E_A).

def _fbs_by_brute_force(c_fid, alpha):
    """argmin_c alpha/2 (c - c_fid)^2 + c^2 (the proximal step of Alg. 2 with
    c_1/2 = 0, eta = 1), located on a fine grid, independent of any formula."""
    lo, hi = min(0.0, c_fid) - 1.0, max(0.0, c_fid) + 1.0
    for _ in range(4):
        g = np.linspace(lo, hi, 2001)
        q = 0.5 * alpha * (g - c_fid) ** 2 + g ** 2
        i = int(np.argmin(q))
        step = g[1] - g[0]
        lo, hi = g[max(i - 1, 0)] - step, g[min(i + 1, 2000)] + step
    return g[i]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("b", [1, 2, 4, 8])
def test_one_step_picks_zero_or_the_step_and_never_raises_energy(kind, b):
    H, W = 24, 28
    u = rand_img(H, W, 300 + b)
    f = u + 0.08 * np.random.default_rng(400 + b).normal(size=(H, W))
    alpha = 12.0
    n_step = 0
    for bi, bj, r0, c0, bh, bw in blocks_of(H, W, b):
        c, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind, one_step=True,
                                   finest=(b == 1))
        assert info["n_eval"] == 2
        assert info["E_best"] <= info["E_zero"]
        if b == 1:
            c1 = oracle.paper_candidate(u, f, r0, c0, alpha, kind)
        else:
            c1 = _fbs_by_brute_force(info["c_fid"], alpha)
        E1 = oracle.local_energy(u, f, r0, c0, bh, bw, c1, alpha, kind)
        if c == 0.0:
            assert E1 >= info["E_zero"] - 1e-9 * abs(info["E_zero"])
        else:
            n_step += 1
            assert c == pytest.approx(c1, abs=1e-6)
            assert E1 <= info["E_zero"] + 1e-9 * abs(info["E_zero"])
    assert n_step > 0


def test_one_step_alpha_limits():
    """Large alpha: the step tends to the block's fidelity mean c_fid and is
    taken; small alpha: the step tends to 0."""
    H, W = 16, 16
    u = np.full((H, W), 0.5)
    f = u.copy()
    f[4:8, 4:8] += 0.3
    c_big, info = oracle.block_min(u, f, 4, 4, 4, 4, 1e6, oracle.MEAN, one_step=True)
    assert c_big == pytest.approx(info["c_fid"], rel=1e-5)
    assert info["c_fid"] == pytest.approx(0.3)
    c_small, _ = oracle.block_min(u, f, 4, 4, 4, 4, 1e-6, oracle.MEAN, one_step=True)
    assert abs(c_small) < 1e-6


@pytest.mark.parametrize("kind", KINDS)
def test_one_step_sequential_levels_never_raise_energy(kind):
    H, W = 20, 22
    img = synth.piecewise_image(H, W, 77, 4, 0.08)
    f = img.f.astype(np.float64)
    u = f.copy()
    E = oracle.energy(u, f, 10.0, kind)
    for b in (1, 2, 4, 8, 1, 2):
        u = oracle.level_sequential(u, f, 10.0, kind, b, one_step=True)
        E1 = oracle.energy(u, f, 10.0, kind)
        assert E1 <= E + 1e-9 * abs(E)
        E = E1


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("one_step", [False, True])
def test_search_with_a_supplied_ring_sum_is_block_min(kind, one_step):
    """The search seen only through s, S1 and the ring sum (the form a block
    split over row strips uses, the ring sum assembled by the caller) picks
    the same shift as block_min after the same number of evaluations; the
    ring sum it is handed here is the full energy difference less the
    fidelity part, computed from the whole image."""
    H, W, alpha = 14, 12, 9.0
    u = rand_img(H, W, 40 + kind)
    f = rand_img(H, W, 50 + kind, smooth=False)
    for b in (1, 2, 3, 5):
        for _, _, r0, c0, bh, bw in blocks_of(H, W, b):
            c, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind, one_step=one_step,
                                       finest=(b == 1))
            s = bh * bw
            S1 = float(np.sum(u[r0:r0 + bh, c0:c0 + bw] - f[r0:r0 + bh, c0:c0 + bw]))
            F0 = oracle.energy(u, f, alpha, kind)
            curv0 = F0 - 0.5 * alpha * float(np.sum((u - f) ** 2))
            calls = []

            def ring(cc):
                v = u.copy()
                v[r0:r0 + bh, c0:c0 + bw] += cc
                calls.append(cc)
                ring0 = oracle.local_energy(u, f, r0, c0, bh, bw, 0.0, alpha, kind)
                # sum over ring(A) of |kappa(v)| = (total |kappa(v)|) - (the rest,
                # unchanged by the shift) = curv(v) - (curv0 - ring0 at c = 0)
                curv = np.sum(np.abs(oracle.curvature_map(v, kind)))
                return curv - (curv0 - ring0)

            cand = oracle.paper_candidate(u, f, r0, c0, alpha, kind) if b == 1 else None
            c2, info2 = oracle.block_search(s, S1, alpha, ring, one_step=one_step, cand=cand)
            assert c2 == pytest.approx(c, abs=1e-9), (b, r0, c0)
            assert info2["n_eval"] == info["n_eval"]
            # ring evaluations: E(0), E at every considered point, and (the
            # search) the bracket's ring sum at c_fid
            assert len(calls) == info["n_eval"] + (0 if one_step else 1)
