"""The rule by which the solve runs a level in place.

A phase of colour k reads, for every block of that colour, the block and the
pixels up to 2 away from it (the ring and the ring's 3 x 3 curvature
stencils).  One buffer updated in place gives exactly the snapshot state of
the phase (new values on earlier colours, old values elsewhere) when no such
read window contains a pixel of another block of colour k.  The library
decides this with (p - 1) b >= 2 for p x p colours and b >= 2 (two colours:
never); this test checks that criterion against a brute-force search over
the oracle's own colouring.
"""
import numpy as np
import pytest

import oracle


def windows_stay_clear(b, ncolors, H=None, W=None):
    """Brute force: no block's window (block +- 2 px) meets another block of
    the same colour, on an image large enough to hold every neighbourhood."""
    p = {2: 2, 4: 2, 9: 3, 16: 4}[ncolors]
    H = H or (2 * p + 3) * b
    W = W or (2 * p + 3) * b
    nbi, nbj = -(-H // b), -(-W // b)
    col = np.array([[oracle.block_colour(i, j, ncolors) for j in range(nbj)] for i in range(nbi)])
    owner = np.repeat(np.repeat(np.arange(nbi * nbj).reshape(nbi, nbj), b, 0), b, 1)[:H, :W]
    pix_col = np.repeat(np.repeat(col, b, 0), b, 1)[:H, :W]
    for bi in range(nbi):
        for bj in range(nbj):
            r0, c0 = bi * b, bj * b
            win_o = owner[max(0, r0 - 2):r0 + b + 2, max(0, c0 - 2):c0 + b + 2]
            win_c = pix_col[max(0, r0 - 2):r0 + b + 2, max(0, c0 - 2):c0 + b + 2]
            same = (win_c == col[bi, bj]) & (win_o != bi * nbj + bj)
            if same.any():
                return False
    return True


def rule(b, ncolors):
    p = {4: 2, 9: 3, 16: 4}.get(ncolors, 0)
    return b >= 2 and p >= 2 and (p - 1) * b >= 2


@pytest.mark.parametrize("ncolors", [2, 4, 9, 16])
@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 8])
def test_in_place_criterion_matches_brute_force(b, ncolors):
    clear = windows_stay_clear(b, ncolors)
    if b >= 2:
        # the library's rule (levels of b >= 2; the finest level keeps S and R)
        assert rule(b, ncolors) == clear, (b, ncolors, clear)
    else:
        assert not rule(b, ncolors)


def test_decoupled_colourings_are_in_place_on_every_level_of_b_ge_2():
    """The decoupled colouring (ncolors = 0) picks p x p colours with
    (p - 1) b >= 3, so every one of its levels with b >= 2 qualifies."""
    for b in (2, 3, 4, 7, 8, 15, 16, 64):
        nc = oracle.level_colours(0, b)
        assert nc in (4, 9, 16) and rule(b, nc) and windows_stay_clear(b, nc)
