"""Pins of the oracle's outer loop (Alg. 3, Eq. reerr) and the paper's trends.

The images of Sec. 4 are unavailable, so the tables' numbers cannot be
reproduced; their qualitative findings are checked on the synthetic images:
coarse layers cut the number of outer iterations (Table 1), and the half
V-cycle lowers the energy steadily.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth


def test_energy_trace_and_fixed_cycles():
    img = synth.single_64()
    f = img.f.astype(np.float64)
    u, trace, n, conv = oracle.solve(f, 20.0, oracle.MEAN, levels=0, cycles=5, tol=0.0)
    assert n == 5 and not conv
    assert trace.shape == (6,)
    assert trace[0] == pytest.approx(oracle.energy(f, f, 20.0, oracle.MEAN), rel=1e-14)
    assert trace[-1] == pytest.approx(oracle.energy(u, f, 20.0, oracle.MEAN), rel=1e-14)
    # the colour-parallel sweep is not guaranteed monotone cycle to cycle,
    # but on this image it descends clearly overall
    assert trace[-1] < 0.5 * trace[0]


def test_stopping_rule_eq_reerr():
    """Stop at the first cycle with |F_l - F_{l-1}| <= tol |F_l|."""
    img = synth.single_64()
    f = img.f.astype(np.float64)
    tol = 1e-3
    u, trace, n, conv = oracle.solve(f, 20.0, oracle.MEAN, cycles=200, tol=tol)
    assert conv
    rel = np.abs(np.diff(trace)) / np.abs(trace[1:])
    assert rel[-1] <= tol
    assert np.all(rel[:-1] > tol)


def test_initial_guess_and_resume():
    """Resuming from u after k cycles equals running k + m cycles."""
    img = synth.piecewise_image(24, 20, 5, 4, 0.05)
    f = img.f.astype(np.float64)
    u3, _, _, _ = oracle.solve(f, 20.0, oracle.GAUSS, cycles=3)
    u5a, _, _, _ = oracle.solve(f, 20.0, oracle.GAUSS, cycles=2, u0=u3)
    u5, _, _, _ = oracle.solve(f, 20.0, oracle.GAUSS, cycles=5)
    np.testing.assert_array_equal(u5a, u5)


def test_levels_reduce_iterations():
    """Table 1 trend: more layers need far fewer outer iterations to reach the
    same relative-energy tolerance than the single (pixel) layer."""
    img = synth.piecewise_image(32, 32, 11, 4, 0.08)
    f = img.f.astype(np.float64)
    _, t1, n1, c1 = oracle.solve(f, 10.0, oracle.MEAN, levels=1, cycles=400, tol=1e-5)
    _, tL, nL, cL = oracle.solve(f, 10.0, oracle.MEAN, levels=0, cycles=400, tol=1e-5)
    assert cL
    assert nL < n1
    # and the multilevel energy is at least as low
    assert tL[-1] <= t1[-1] * (1 + 1e-3)


def test_cycle_count_does_not_grow_with_the_image():
    """Table "linear" trend: with every level down to blocks of half the
    image side, the cycles to the relative-energy tolerance stay in a narrow
    band as the pixel count grows 16-fold (32^2 to 128^2, two images of
    each size from the same generator), so the cost grows with the pixels
    alone."""
    counts = {}
    for side in (32, 64, 128):
        counts[side] = []
        for i in (0, 1):
            f = synth.large(side, i).f.astype(np.float64)
            _, _, n, conv = oracle.solve(f, 20.0, oracle.MEAN, cycles=200, tol=1e-4, ncolors=4)
            assert conv
            counts[side].append(n)
    flat = [n for v in counts.values() for n in v]
    assert max(flat) - min(flat) <= 3, counts
    assert max(counts[128]) <= min(counts[32]) + 3, counts


def test_denoising_improves_psnr():
    """The minimiser of the curvature energy removes noise: PSNR against the
    clean synthetic image rises (Sec. 4 measures PSNR)."""
    img = synth.single_64()
    f = img.f.astype(np.float64)
    u, _, _, _ = oracle.solve(f, 20.0, oracle.MEAN, cycles=20)
    assert synth.psnr(u, img.clean) > synth.psnr(f, img.clean) + 3.0


def test_four_colours_at_coarse_levels_is_gauss_seidel():
    """With four colours and b >= 3 same-colour blocks are >= 3 pixels apart,
    so no block's ring touches another same-colour block (Sec. 2.3's
    independence claim holds) and the colour-parallel phase equals solving
    its blocks one after another."""
    img = synth.piecewise_image(24, 24, 13, 5, 0.1)
    f = img.f.astype(np.float64)
    u = oracle.cycle(f, f, 15.0, oracle.MEAN, levels=2)
    b = 4
    for k in range(4):
        par, _ = oracle.phase(u, f, 15.0, oracle.MEAN, b, 4, k)
        seq = u.copy()
        for bi in range(6):
            for bj in range(6):
                if oracle.block_colour(bi, bj, 4) != k:
                    continue
                c, _ = oracle.block_min(seq, f, bi * b, bj * b, b, b, 15.0, oracle.MEAN)
                seq[bi * b:(bi + 1) * b, bj * b:(bj + 1) * b] += c
        np.testing.assert_array_equal(par, seq)


def test_thread_count_does_not_change_result():
    """The phase's snapshot semantics make the block order irrelevant: one
    thread and many threads give bit-identical results."""
    code = (
        "import numpy as np, oracle, synth\n"
        "f = synth.piecewise_image(40, 36, 3, 5, 0.1).f.astype(np.float64)\n"
        "u, _, _, _ = oracle.solve(f, 15.0, 1, cycles=2)\n"
        "import sys; sys.stdout.write(u.tobytes().hex()[:4000] + str(float(u.sum())))\n"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "4"):
        env = dict(os.environ, OMP_NUM_THREADS=nt, PYTHONPATH=root)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, cwd=root,
                                   capture_output=True, text=True, check=True).stdout)
    assert outs[0] == outs[1]


def test_set_num_threads_keeps_results():
    """The timing runs' thread setting: the count takes effect and the solve
    is bit-identical with one thread and with all of them."""
    f = synth.piecewise_image(40, 36, 4, 5, 0.1).f.astype(np.float64)
    n0 = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        assert oracle.num_threads() == 1
        u1, _, _, _ = oracle.solve(f, 20.0, 0, cycles=2, ncolors=4)
    finally:
        oracle.set_num_threads(n0)
    assert oracle.num_threads() == n0
    un, _, _, _ = oracle.solve(f, 20.0, 0, cycles=2, ncolors=4)
    np.testing.assert_array_equal(u1, un)


@pytest.mark.parametrize("shape", [(1, 9), (9, 1), (1, 1), (3, 2), (7, 5)])
def test_degenerate_shapes(shape):
    """Single-row, single-column, single-pixel and tiny images run and never
    raise the energy in sequential order."""
    rng = np.random.default_rng(sum(shape))
    f = rng.random(shape)
    for kind in (oracle.MEAN, oracle.GAUSS):
        u, trace, n, _ = oracle.solve(f, 5.0, kind, cycles=3, sequential=True)
        assert n == 3
        assert np.all(np.diff(trace) <= 1e-12 * np.abs(trace[1:]))
        assert np.all(np.isfinite(u))


# ---------------------------------------------------------------------------
# Decoupled colourings and the full V-cycle.

def test_decoupled_colours_keep_blocks_three_pixels_apart():
    """ncolors = 0: on every level two distinct blocks of one colour are at
    least 3 pixels apart (so no window of a ring pixel of one holds a ring
    pixel of the other)."""
    for b in (1, 2, 4, 8, 16):
        nc = oracle.level_colours(0, b)
        p = int(round(nc ** 0.5))
        assert p * p == nc and (p - 1) * b >= 3 and (p == 2 or (p - 2) * b < 3)
        cols = {}
        for bi in range(2 * p + 1):
            for bj in range(2 * p + 1):
                cols.setdefault(oracle.block_colour(bi, bj, nc), []).append((bi, bj))
        assert sorted(cols) == list(range(nc))
        for members in cols.values():
            for a in members:
                for c in members:
                    if a == c:
                        continue
                    gap_r = max(0, abs(a[0] - c[0]) * b - b)
                    gap_c = max(0, abs(a[1] - c[1]) * b - b)
                    assert max(gap_r, gap_c) >= 3


@pytest.mark.parametrize("kind", [oracle.MEAN, oracle.GAUSS])
@pytest.mark.parametrize("b", [1, 2, 4])
def test_decoupled_phase_equals_one_block_at_a_time(kind, b):
    """A colour's parallel (snapshot) solve equals solving its blocks one after
    another, each applied before the next, when the colouring is decoupled."""
    H, W = 19, 23
    img = synth.piecewise_image(H, W, 90 + b, 4, 0.08)
    f = img.f.astype(np.float64)
    u = oracle.cycle(f, f, 12.0, kind, levels=1)
    nc = oracle.level_colours(0, b)
    nbi, nbj = (H + b - 1) // b, (W + b - 1) // b
    for k in range(nc):
        par, _ = oracle.phase(u, f, 12.0, kind, b, nc, k)
        seq = u.copy()
        for bi in range(nbi):
            for bj in range(nbj):
                if oracle.block_colour(bi, bj, nc) != k:
                    continue
                r0, c0 = bi * b, bj * b
                bh, bw = min(b, H - r0), min(b, W - c0)
                c, _ = oracle.block_min(seq, f, r0, c0, bh, bw, 12.0, kind, finest=(b == 1))
                seq[r0:r0 + bh, c0:c0 + bw] += c
        np.testing.assert_allclose(par, seq, rtol=0, atol=1e-12)
        u = par


@pytest.mark.parametrize("kind", [oracle.MEAN, oracle.GAUSS])
@pytest.mark.parametrize("vcycle", [False, True])
def test_decoupled_solve_is_monotone(kind, vcycle):
    """With decoupled colours every phase is a sequence of block updates that
    never raise F, so the energy trace never rises."""
    img = synth.piecewise_image(40, 44, 5, 6, 0.08)
    u, trace, n, _ = oracle.solve(img.f, 15.0, kind, cycles=6, ncolors=0, vcycle=vcycle)
    assert n == 6
    assert np.all(np.diff(trace) <= 1e-10 * np.abs(trace[1:]))


def test_vcycle_is_half_cycle_then_levels_back_up():
    img = synth.piecewise_image(33, 40, 6, 5, 0.08)
    f = img.f.astype(np.float64)
    L = oracle.auto_levels(33, 40)
    uv = oracle.cycle(f, f, 15.0, oracle.MEAN, ncolors=4, vcycle=True)
    uh = oracle.cycle(f, f, 15.0, oracle.MEAN, ncolors=4)
    for j in range(L - 1, 0, -1):
        for k in range(4):
            uh, _ = oracle.phase(uh, f, 15.0, oracle.MEAN, 1 << (j - 1), 4, k)
    np.testing.assert_array_equal(uv, uh)


def test_paper_block_sides_schedule():
    """Sec. 2.2: level j groups the pixels into patches of (2^j - 1) x (2^j - 1)
    (1, 3, 7, 15, ... pixels a side), ceil(m / (2^j - 1)) x ceil(n / (2^j - 1))
    of them.  One phase of level j on a 40 x 29 image returns a shift for
    exactly the patches of its colour, each constant over its patch."""
    assert [oracle.level_side(j, 1) for j in range(1, 6)] == [1, 3, 7, 15, 31]
    assert [oracle.level_side(j, 0) for j in range(1, 6)] == [1, 2, 4, 8, 16]
    # coarsest side <= half the shorter image side
    assert oracle.auto_levels(64, 64, 1) == 5 and oracle.auto_levels(1024, 1024, 1) == 9
    assert oracle.auto_levels(13, 100, 1) == 2 and oracle.auto_levels(5, 5, 1) == 1
    img = synth.piecewise_image(40, 29, 8, 4, 0.08)
    f = img.f.astype(np.float64)
    u0 = oracle.cycle(f, f, 15.0, oracle.MEAN, levels=1, ncolors=4)
    for j in (2, 3, 4):
        b = oracle.level_side(j, 1)
        mj, nj = -(-40 // b), -(-29 // b)
        moved = 0
        for k in range(4):
            u1, c = oracle.phase(u0, f, 15.0, oracle.MEAN, b, 4, k)
            assert c.shape == (mj * nj,)
            for bi in range(mj):
                for bj in range(nj):
                    blk = (slice(bi * b, (bi + 1) * b), slice(bj * b, (bj + 1) * b))
                    if (2 * (bi % 2) + bj % 2) != k:
                        assert np.all(u1[blk] == u0[blk])   # other colours untouched
                    else:   # one constant per patch
                        assert np.all(u1[blk] == u0[blk] + c[bi * nj + bj])
                        moved += c[bi * nj + bj] != 0.0
        assert moved > 0


def test_paper_block_sides_cycle_is_its_phase_sequence():
    img = synth.piecewise_image(33, 40, 6, 5, 0.08)
    f = img.f.astype(np.float64)
    L = oracle.auto_levels(33, 40, 1)
    assert L == 4   # sides 1, 3, 7, 15
    uc = oracle.cycle(f, f, 15.0, oracle.GAUSS, ncolors=4, sides=1)
    up = f.copy()
    for b in (1, 3, 7, 15):
        for k in range(4):
            up, _ = oracle.phase(up, f, 15.0, oracle.GAUSS, b, 4, k)
    np.testing.assert_array_equal(uc, up)


@pytest.mark.parametrize("kind", [oracle.MEAN, oracle.GAUSS_EULER])
def test_paper_block_sides_monotone_and_denoise(kind):
    """Patches of odd sides keep the defining properties: the sequential
    (Gauss-Seidel) sweep never raises F, the decoupled colouring never raises
    F, and the colour-parallel solve lowers F and denoises."""
    img = synth.piecewise_image(36, 31, 9, 5, 0.08)
    f = img.f.astype(np.float64)
    _, tr, n, _ = oracle.solve(f, 15.0, kind, cycles=4, sequential=True, sides=1)
    assert np.all(np.diff(tr) <= 1e-10 * np.abs(tr[1:]))
    _, tr, n, _ = oracle.solve(f, 15.0, kind, cycles=4, ncolors=0, sides=1)
    assert np.all(np.diff(tr) <= 1e-10 * np.abs(tr[1:]))
    u, tr, n, _ = oracle.solve(f, 15.0, kind, cycles=6, ncolors=4, sides=1)
    assert tr[-1] < 0.7 * tr[0]
    assert synth.psnr(u, img.clean) > synth.psnr(f, img.clean)


def test_coarse_colour_count_schedule():
    """coarse_ncolors sets the colours of the levels with block side >= 64
    only; a cycle is then the phase sequence with 4 colours below 64 and 2
    from 64 on, and the solve still descends and denoises."""
    assert oracle.level_colours(4, 32, 2) == 4
    assert oracle.level_colours(4, 64, 2) == 2 and oracle.level_colours(0, 128, 2) == 2
    assert oracle.level_colours(4, 64, 0) == 4 and oracle.level_colours(0, 64, 0) == 4
    img = synth.piecewise_image(150, 140, 17, 8, 0.08)
    f = img.f.astype(np.float64)
    L = oracle.auto_levels(150, 140)
    assert L == 7   # sides 1 .. 64
    uc = oracle.cycle(f, f, 20.0, oracle.MEAN, ncolors=4, coarse_ncolors=2)
    up = f.copy()
    for j in range(1, L + 1):
        b = oracle.level_side(j)
        nc = 2 if b >= 64 else 4
        for k in range(nc):
            up, _ = oracle.phase(up, f, 20.0, oracle.MEAN, b, nc, k)
    np.testing.assert_array_equal(uc, up)
    u, tr, n, _ = oracle.solve(f, 20.0, oracle.MEAN, cycles=3, ncolors=4, coarse_ncolors=2)
    assert np.all(np.diff(tr) < 0)
    assert synth.psnr(u, img.clean) > synth.psnr(f, img.clean)


def test_one_coarse_colour_is_block_jacobi():
    """coarse_ncolors = 1: every block of a coarse level solves from the same
    state in one phase (a block-Jacobi step): the phase equals each block's
    own minimiser from the input state, applied to all blocks at once; the
    cycle is its phase sequence and the solve descends and denoises."""
    assert oracle.level_colours(4, 64, 1) == 1 and oracle.level_colours(4, 32, 1) == 4
    assert all(oracle.block_colour(bi, bj, 1) == 0 for bi in range(5) for bj in range(7))
    img = synth.piecewise_image(200, 170, 19, 8, 0.08)
    f = img.f.astype(np.float64)
    u = oracle.cycle(f, f, 20.0, oracle.MEAN, levels=6, ncolors=4)
    for b in (64, 128):
        up, cs = oracle.phase(u, f, 20.0, oracle.MEAN, b, 1, 0)
        want = u.copy()
        nbi, nbj = -(-200 // b), -(-170 // b)
        for bi in range(nbi):
            for bj in range(nbj):
                r0, c0 = bi * b, bj * b
                bh, bw = min(b, 200 - r0), min(b, 170 - c0)
                c, _ = oracle.block_min(u, f, r0, c0, bh, bw, 20.0, oracle.MEAN)
                assert cs[bi * nbj + bj] == c
                want[r0:r0 + bh, c0:c0 + bw] += c
        np.testing.assert_array_equal(up, want)
    L = oracle.auto_levels(200, 170)
    uc = oracle.cycle(f, f, 20.0, oracle.MEAN, ncolors=4, coarse_ncolors=1)
    up = f.copy()
    for j in range(1, L + 1):
        b = oracle.level_side(j)
        nc = 1 if b >= 64 else 4
        for k in range(nc):
            up, _ = oracle.phase(up, f, 20.0, oracle.MEAN, b, nc, k)
    np.testing.assert_array_equal(uc, up)
    u, tr, n, _ = oracle.solve(f, 20.0, oracle.MEAN, cycles=3, ncolors=4, coarse_ncolors=1)
    assert np.all(np.diff(tr) < 0)
    assert synth.psnr(u, img.clean) > synth.psnr(f, img.clean)
