"""Shared helpers of the GPU parity tests (comparison with the FP64 oracle).

Tolerances, derived from FP32 arithmetic:

* Per-pixel curvature: each direction curvature takes ~16 FP32 operations and
  two rsqrt (<= 2 ulp each), so its relative error is a few 1e-7 of the
  largest direction curvature; |Delta kappa| <= 2e-5 (1 + max|kbar|) leaves a
  margin of ~10x on [0, 1] images.
* Energy: FP32 pixel terms (relative error <= ~1e-6) summed in FP64:
  |F_gpu - F_oracle| <= 2e-6 |F_oracle|.
* Block shifts: |c_gpu - c_oracle| <= 1e-4 (the required per-sweep bound on
  u).  Where several shifts are correct -- candidates whose energies agree to
  within FP32 evaluation noise -- the GPU's c is a tie if the oracle's FP64
  E_A at the GPU's c is within tau of the oracle's own optimum, with tau =
  1e-6 times the block's energy scale (ring curvature plus fidelity distance,
  both non-negative).  Derivation: the GPU evaluates E_A(c) in FP32 as a sum
  of non-negative ring terms and the fidelity term, each with relative error
  of about 4 eps32 (two rsqrt of <= 2 ulp and a few roundings per
  direction), so an evaluation is off by at most ~4 eps32 of the scale; a
  comparison of two candidates flips only when their true gap is below
  twice that, 8 eps32, and the search's pick loses at most that gap per
  flipped comparison; two flips in one search give 16 eps32 = 9.5e-7,
  i.e. 1e-6 (the FP64 oracle's own error is far below).  Measured over the
  whole GPU suite: 40 ties, the largest gap 2.9e-7 of the scale.  Ties are
  counted and reported.
"""
import oracle

TIE_REL = 1e-6
C_TOL = 1e-4
# (E_A(c_gpu) - E_A(c_oracle)) / scale of every block whose shifts differ by
# more than C_TOL, collected over a test session for the terminal summary
TIE_LOG = []
# search budget of both sides (the library's and the oracle's default)
G_DEF, K_DEF = oracle.DEFAULT_G, oracle.DEFAULT_K


def blocks_of_colour(H, W, b, ncolors, k):
    nbi, nbj = (H + b - 1) // b, (W + b - 1) // b
    for bi in range(nbi):
        for bj in range(nbj):
            col = oracle.block_colour(bi, bj, ncolors)
            if col == k:
                yield bi, bj, bi * b, bj * b, min(b, H - bi * b), min(b, W - bj * b)


def block_rect(H, W, b, bi, bj):
    r0, c0 = bi * b, bj * b
    return r0, c0, min(b, H - r0), min(b, W - c0)


def sample_blocks(H, W, b, ncolors, k, n, rng):
    """Up to n distinct blocks (bi, bj) of colour k drawn at random; large
    levels are drawn from their colour lattice without walking every block."""
    nbi, nbj = (H + b - 1) // b, (W + b - 1) // b
    if nbi * nbj <= 64 * n:
        blocks = [(bi, bj) for bi, bj, *_ in blocks_of_colour(H, W, b, ncolors, k)]
        idx = rng.choice(len(blocks), size=min(n, len(blocks)), replace=False)
        return {blocks[i] for i in idx}
    out = set()
    p = 1 if ncolors == 2 else int(round(ncolors ** 0.5))
    for _ in range(100 * n):
        if len(out) >= n:
            break
        if ncolors == 2:
            bi, bj = int(rng.integers(nbi)), int(rng.integers(nbj))
            if (bi + bj) % 2 != k:
                continue
        else:
            ni, nj = (nbi - k // p + p - 1) // p, (nbj - k % p + p - 1) // p
            bi, bj = k // p + p * int(rng.integers(ni)), k % p + p * int(rng.integers(nj))
        out.add((bi, bj))
    return out


def energy_scale(u, f, r0, c0, bh, bw, c, alpha, kind, c_fid):
    """Non-negative parts of E_A at c: ring curvature + alpha s/2 (c - c_fid)^2."""
    s = bh * bw
    S1 = -c_fid * s
    e = oracle.local_energy(u, f, r0, c0, bh, bw, c, alpha, kind)
    fid = 0.5 * alpha * (s * c * c + 2 * c * S1)
    ring = e - fid
    return ring + 0.5 * alpha * s * (c - c_fid) ** 2


def compare_phase(u, f, c_gpu_blocks, alpha, kind, b, ncolors, k, c_orc_blocks, sample=None,
                  G=G_DEF, K=K_DEF, use_paper=True, one_step=False):
    """Compare per-block shifts of one phase.  c_*_blocks: dict (bi, bj) -> c.
    Returns (n_blocks, n_match, n_tie, list_of_failures)."""
    H, W = u.shape
    n = match = tie = 0
    fails = []
    if sample is None:
        blocks = blocks_of_colour(H, W, b, ncolors, k)
    else:
        blocks = [(bi, bj, *block_rect(H, W, b, bi, bj)) for bi, bj in sorted(sample)]
        assert all(oracle.block_colour(bi, bj, ncolors) == k for bi, bj in sample)
    for bi, bj, r0, c0, bh, bw in blocks:
        n += 1
        cg = float(c_gpu_blocks[(bi, bj)])
        if (bi, bj) in c_orc_blocks:
            co = float(c_orc_blocks[(bi, bj)])
        else:
            co, _ = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind, G=G, K=K,
                                     use_paper=use_paper, one_step=one_step, finest=(b == 1))
        if abs(cg - co) <= C_TOL:
            match += 1
            continue
        Eg = oracle.local_energy(u, f, r0, c0, bh, bw, cg, alpha, kind)
        Eo = oracle.local_energy(u, f, r0, c0, bh, bw, co, alpha, kind)
        _, info = oracle.block_min(u, f, r0, c0, bh, bw, alpha, kind, G=G, K=K,
                                   use_paper=use_paper, one_step=one_step, finest=(b == 1))
        scale = max(energy_scale(u, f, r0, c0, bh, bw, cg, alpha, kind, info["c_fid"]),
                    energy_scale(u, f, r0, c0, bh, bw, co, alpha, kind, info["c_fid"]))
        TIE_LOG.append((Eg - Eo) / max(scale, 1e-300))
        if Eg - Eo <= TIE_REL * scale:
            tie += 1
        else:
            fails.append(dict(block=(bi, bj), b=b, c_gpu=cg, c_orc=co, E_gpu=Eg, E_orc=Eo,
                              scale=scale, rel=(Eg - Eo) / max(scale, 1e-30)))
    return n, match, tie, fails
