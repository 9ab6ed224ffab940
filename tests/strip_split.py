"""Row-strip split of ONE image over ranks, emulated on the FP64 oracle (CPU,
torch.distributed with gloo).  Test infrastructure: it shows which exchange
steps a single-image split of the sweep would need and that, with them, the
split computes the whole-image result.

Decomposition.  Rank r owns rows [R_r, R_{r+1}) of u and f and keeps a halo
of two rows on each side (one row for the 3x3 stencil of a ring pixel, one
more because a block's ring reaches one row beyond the block).  A phase
(level, colour; snapshot semantics) then runs as:

  1. halo exchange: every rank receives its neighbours' two boundary rows of
     u as they stand at the phase start (one round);
  2. blocks whose rows lie in one strip: the owner runs the oracle's block
     minimiser on its strip and halo alone (no exchange);
  3. blocks whose rows straddle a strip boundary: every rank adds the part
     of S1 = sum_A (u - f) and of the ring sum sum_{q in ring(A)}
     |kappa_q(u + c phi_A)| that lies in its rows, and an all-reduce sums
     them, once for S1 and once per ring evaluation of the block search (the
     search runs the same steps on every rank, so the rounds line up);
  4. every rank adds the shifts to its own rows.

Each cycle ends with one more halo exchange (the energy's stencils read the
neighbours' rows as the last phase left them) and an all-reduce of the
ranks' FP64 energy sums (Eq. MCM / GCM), which feeds the stopping test.

The emulation runs the straddling blocks' searches one after another (one
round per evaluation); a GPU split would run all straddling blocks of a
phase in lockstep, so its dependent rounds per phase are 1 (halo), plus,
when the phase has straddling blocks, 1 (S1) and the search's ring
evaluations (2 + G + K; 2 in the one-step mode).  `split_rounds` counts
both for any shape.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

import oracle


def strip_rows(H, world):
    """Row boundaries R_0 = 0 < R_1 < ... < R_world = H, strips as equal as
    possible (the first H mod world strips one row taller)."""
    q, rem = divmod(H, world)
    R = [0]
    for r in range(world):
        R.append(R[-1] + q + (1 if r < rem else 0))
    return R


def _blocks(H, W, b, nc, k):
    """The blocks (a0, a1, c0, c1) of colour k on the level with side b,
    clipped to the image, in raster order."""
    out = []
    for bi in range((H + b - 1) // b):
        for bj in range((W + b - 1) // b):
            if oracle.block_colour(bi, bj, nc) == k:
                out.append((bi * b, min(H, bi * b + b), bj * b, min(W, bj * b + b)))
    return out


def _straddles(a0, a1, R):
    return any(a0 < x < a1 for x in R[1:-1])


def _ring(H, W, a0, a1, c0, c1):
    """ring(A): in-image pixels within Chebyshev distance 1 of A whose clamped
    3x3 stencil holds pixels inside and outside A (raster order)."""
    def inside(r, c):
        return a0 <= r < a1 and c0 <= c < c1

    out = []
    for r in range(max(a0 - 1, 0), min(a1 + 1, H)):
        for c in range(max(c0 - 1, 0), min(c1 + 1, W)):
            if not inside(r, c) or any(
                    not inside(min(max(r + dr, 0), H - 1), min(max(c + dc, 0), W - 1))
                    for dr in (-1, 0, 1) for dc in (-1, 0, 1)):
                out.append((r, c))
    return out


def _levels(H, W, levels, ncolors, coarse_ncolors, sides):
    L = levels if levels > 0 else oracle.auto_levels(H, W, sides)
    for j in range(1, L + 1):
        b = oracle.level_side(j, sides)
        yield b, oracle.level_colours(ncolors, b, coarse_ncolors)


def split_rounds(H, W, world, levels=0, ncolors=4, coarse_ncolors=0, sides=0, G=oracle.DEFAULT_G,
                 K=oracle.DEFAULT_K, one_step=False):
    """Exchange rounds of one cycle of the strip split.  Returns a dict:
    phases; halo (one per phase and one before the energy); straddling
    (blocks); block_rounds (the emulation's all-reduces: S1 and the ring
    evaluations of every straddling block); lockstep_rounds (dependent
    rounds with the straddling blocks of a phase batched, the energy's two
    included); energy (1)."""
    R = strip_rows(H, world)
    evals = 2 if one_step else 2 + G + K
    phases = straddling = lockstep = 0
    for b, nc in _levels(H, W, levels, ncolors, coarse_ncolors, sides):
        for k in range(nc):
            phases += 1
            n = sum(_straddles(a0, a1, R) for a0, a1, _, _ in _blocks(H, W, b, nc, k))
            straddling += n
            lockstep += 1 + (1 + evals if n else 0)
    return dict(phases=phases, halo=phases + 1, straddling=straddling,
                block_rounds=straddling * (1 + evals), lockstep_rounds=lockstep + 2, energy=1)


class _Strip:
    def __init__(self, f, rank, world):
        H, W = f.shape
        self.H, self.W = H, W
        R = strip_rows(H, world)
        self.R = R
        self.R0, self.R1 = R[rank], R[rank + 1]
        if self.R1 - self.R0 < 2:
            raise ValueError("every strip needs at least two rows")
        self.h0, self.h1 = min(2, self.R0), min(2, H - self.R1)
        self.base = self.R0 - self.h0
        self.rank, self.world = rank, world
        self.f = np.array(f[self.base:self.R1 + self.h1], dtype=np.float64)
        self.u = self.f.copy()            # u0 = f
        self.rounds = 0

    def _allreduce(self, x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t)
        self.rounds += 1
        return float(t.item())

    def halo_exchange(self):
        W, n = self.W, self.R1 - self.R0
        own = self.u[self.h0:self.h0 + n]
        mine = torch.from_numpy(np.concatenate([own[:2], own[-2:]]).copy())
        got = [torch.zeros(4, W, dtype=torch.float64) for _ in range(self.world)]
        dist.all_gather(got, mine)
        self.rounds += 1
        if self.h0:
            self.u[:self.h0] = got[self.rank - 1].numpy()[4 - self.h0:]
        if self.h1:
            self.u[self.h0 + n:] = got[self.rank + 1].numpy()[:self.h1]

    def energy(self, alpha, kind):
        self.halo_exchange()              # own-row stencils read the neighbours' rows
        n = self.R1 - self.R0
        kap = oracle.curvature_map(self.u, kind)[self.h0:self.h0 + n]
        d = self.u[self.h0:self.h0 + n] - self.f[self.h0:self.h0 + n]
        part = float(np.sum(np.abs(kap)) + 0.5 * alpha * np.sum(d * d))
        return self._allreduce(part)

    def _own(self, r):
        return self.R0 <= r < self.R1

    def straddling_block(self, A, alpha, kind, G, K, one_step):
        a0, a1, c0, c1 = A
        lo, hi = max(a0, self.R0), min(a1, self.R1)
        S1 = self._allreduce(float(np.sum(self.u[lo - self.base:hi - self.base, c0:c1]
                                          - self.f[lo - self.base:hi - self.base, c0:c1]))
                             if lo < hi else 0.0)
        ring = [(r, c) for r, c in _ring(self.H, self.W, a0, a1, c0, c1) if self._own(r)]
        top = self.base + self.u.shape[0]
        r_lo, r_hi = max(a0, self.base) - self.base, min(a1, top) - self.base

        def ring_sum(c):
            v = self.u.copy()
            if r_lo < r_hi:
                v[r_lo:r_hi, c0:c1] += c
            kap = oracle.curvature_map(v, kind)
            return self._allreduce(sum(abs(kap[r - self.base, cc]) for r, cc in ring))

        s = (a1 - a0) * (c1 - c0)
        c, _ = oracle.block_search(s, S1, alpha, ring_sum, G, K, one_step)
        return c

    def phase(self, b, nc, k, alpha, kind, G, K, use_paper, one_step):
        self.halo_exchange()
        shifts = []
        for A in _blocks(self.H, self.W, b, nc, k):
            a0, a1, c0, c1 = A
            if _straddles(a0, a1, self.R):
                shifts.append((A, self.straddling_block(A, alpha, kind, G, K, one_step)))
            elif self._own(a0):
                c, _ = oracle.block_min(self.u, self.f, a0 - self.base, c0, a1 - a0, c1 - c0,
                                        alpha, kind, G, K, use_paper, one_step, finest=(b == 1))
                shifts.append((A, c))
        for (a0, a1, c0, c1), c in shifts:
            lo, hi = max(a0, self.R0), min(a1, self.R1)
            if lo < hi:
                self.u[lo - self.base:hi - self.base, c0:c1] += c

    def own_rows(self):
        return self.u[self.h0:self.h0 + self.R1 - self.R0].copy()


def split_solve(f, alpha, kind, cycles, rank, world, levels=0, ncolors=4, coarse_ncolors=0,
                sides=0, G=oracle.DEFAULT_G, K=oracle.DEFAULT_K, use_paper=True, one_step=False):
    """Runs `cycles` cycles (tol = 0) of the strip split as rank `rank` of an
    initialised process group of `world` ranks.  Returns (u, trace, rounds)
    with u the whole image (gathered), trace the energies at u0 and after
    each cycle, and rounds the collectives this rank took part in."""
    st = _Strip(f, rank, world)
    trace = [st.energy(alpha, kind)]
    for _ in range(cycles):
        for b, nc in _levels(st.H, st.W, levels, ncolors, coarse_ncolors, sides):
            for k in range(nc):
                st.phase(b, nc, k, alpha, kind, G, K, use_paper, one_step)
        trace.append(st.energy(alpha, kind))
    parts = [None] * world
    dist.all_gather_object(parts, st.own_rows())
    return np.concatenate(parts), np.array(trace), st.rounds
