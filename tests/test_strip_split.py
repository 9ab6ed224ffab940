"""A single image split into row strips over gloo ranks (CPU) computes the
whole-image sweep: the halo exchange per phase, the all-reduced S1 and ring
sums of the blocks that straddle a strip boundary, and the all-reduced FP64
energy are the only exchanges it needs.  Compared with the oracle's
whole-image solve (Alg. 3) on the same input; the number of collectives each
rank took part in equals the count of `split_rounds`."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from strip_split import split_rounds, split_solve, strip_rows

CYCLES = 2
ALPHA = 15.0

# (H, W, world, solve options); every case has strips of >= 2 rows
CASES = [
    (30, 26, 2, dict(kind=oracle.MEAN, ncolors=4)),
    (30, 26, 2, dict(kind=oracle.GAUSS, ncolors=2)),
    (33, 20, 2, dict(kind=oracle.MEAN_EULER, ncolors=4, one_step=True)),
    (32, 24, 2, dict(kind=oracle.MEAN, ncolors=4)),                      # aligned strips
    (30, 26, 2, dict(kind=oracle.GAUSS_EULER, ncolors=4, sides=1)),      # sides 2^j - 1
    (31, 27, 2, dict(kind=oracle.MEAN, ncolors=0)),                      # decoupled colours
]
CASES3 = [
    (30, 26, 3, dict(kind=oracle.MEAN, ncolors=4)),
    (29, 24, 3, dict(kind=oracle.GAUSS, ncolors=2, coarse_ncolors=0)),
]
# strips of 3, 3, 2 and 2 rows: a block of side 8 spans three strips, and
# the halo of a 2-row strip is its neighbour's whole strip
CASES4 = [
    (10, 24, 4, dict(kind=oracle.MEAN, ncolors=4, levels=4)),
    (10, 24, 4, dict(kind=oracle.GAUSS_EULER, ncolors=2, levels=4)),
]


def _f(H, W, seed):
    return synth.piecewise_image(H, W, 50 + seed, 5, 0.08).f.astype(np.float64)


def _worker(rank, world, port, cases, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=120))
    res = []
    for i, (H, W, _, kw) in enumerate(cases):
        kw = dict(kw)
        kind = kw.pop("kind")
        u, tr, rounds = split_solve(_f(H, W, i), ALPHA, kind, CYCLES, rank, world, **kw)
        res.append((u, tr, rounds))
    out[rank] = res
    dist.destroy_process_group()


def _run(cases, world):
    oracle.build()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, cases, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return [out[r] for r in range(world)]


def _check(cases, results, world):
    for i, (H, W, _, kw) in enumerate(cases):
        kw = dict(kw)
        kind = kw.pop("kind")
        f = _f(H, W, i)
        uo, tro, _, _ = oracle.solve(f, ALPHA, kind, cycles=CYCLES, **kw)
        counts = split_rounds(H, W, world, **{k: v for k, v in kw.items()})
        want_rounds = CYCLES * (counts["halo"] + counts["block_rounds"] + counts["energy"]) + 2
        for r in range(world):
            u, tr, rounds = results[r][i]
            assert u.shape == f.shape
            assert np.max(np.abs(u - uo)) <= 1e-12, (i, r)
            np.testing.assert_allclose(tr, tro, rtol=1e-12)
            assert rounds == want_rounds, (i, r, rounds, want_rounds)
        assert np.array_equal(results[0][i][0], results[-1][i][0])


def test_two_rank_strip_split_equals_the_whole_image_solve():
    results = _run(CASES, 2)
    _check(CASES, results, 2)
    # blocks straddle the boundary at row 15; none straddle row 16 of 32 rows
    assert split_rounds(30, 26, 2)["straddling"] > 0
    assert split_rounds(32, 24, 2)["straddling"] == 0


def test_three_rank_strip_split_equals_the_whole_image_solve():
    results = _run(CASES3, 3)
    _check(CASES3, results, 3)


def test_four_rank_strip_split_with_blocks_over_three_strips():
    R = strip_rows(10, 4)
    assert R == [0, 3, 6, 8, 10]
    assert sum(1 for x in R[1:-1] if 0 < x < 8) == 2      # rows 0 .. 7: three strips
    results = _run(CASES4, 4)
    _check(CASES4, results, 4)


def test_strip_rows_and_round_counts():
    assert strip_rows(10, 3) == [0, 4, 7, 10]
    assert strip_rows(1024, 4) == [0, 256, 512, 768, 1024]
    # 1024^2, blocks 1 .. 512, 4 colours (2 on b >= 64): with two strips the
    # boundary at row 512 is a multiple of every block side, so only the halo
    # exchanges and the energy remain
    two = split_rounds(1024, 1024, 2, ncolors=4, coarse_ncolors=2)
    assert two["straddling"] == 0 and two["lockstep_rounds"] == two["phases"] + 2 == 34
    # with eight strips of 128 rows the blocks of sides 256 and 512 straddle:
    # each such phase adds S1 and the search's 2 + G + K ring evaluations
    eight = split_rounds(1024, 1024, 8, ncolors=4, coarse_ncolors=2)
    assert eight["straddling"] == 20
    assert eight["lockstep_rounds"] == 34 + 4 * (1 + 2 + oracle.DEFAULT_G + oracle.DEFAULT_K)
    with pytest.raises(ValueError):
        from strip_split import _Strip
        _Strip(np.zeros((3, 4)), 1, 2)          # rows [2, 3): one row
