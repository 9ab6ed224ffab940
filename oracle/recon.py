"""FP64 oracle of the reconstruction extension (Sec. 5), MRI-like operator.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the product path never
imports it.

Problem (Sec. 5): recover a real image u from data b = A u + noise by
minimising  J(u) = 1/2 ||A u - b||^2 + alpha sum_x |kappa(u(x))|.
Here A = M F: F the orthonormal 2-D DFT (numpy.fft with norm="ortho"), M a
0/1 mask of sampled k-space entries (MRI; the CT operator of Sec. 5 is not
built).  The multigrid sweep of Sec. 2.2 visits the levels fine to coarse and
on each level the colours in order (Alg. 3); the blocks phi_i of one colour
are solved together, because A couples them.  Sec. 5 replaces each block's
curvature term by alpha (c_i - d_i)^2 around the curvature-only estimate d_i
(the Proposition of Sec. 3 on which Eq. c-sol1 rests) and solves the normal
equations of the resulting quadratic problem,

    [<A phi_i, A phi_j> + 2 alpha delta_ij] c = <b - A u, A phi_i> + 2 alpha d_i,

by conjugate gradients.  u is real and A complex, so the inner products are
the real parts (the derivative of 1/2 ||A(u + sum c_i phi_i) - b||^2 in the
real c_i).

READINGS (listed in the design notes): d_i on the finest level is c_{1/2} of
Eq. c-sol1 (Prop. 2 for Gaussian curvature); on coarser levels d_i = 0, as in
the single-step mode (the paper's coarse-layer estimate comes from a figure
that is missing).  CG starts from c = 0 and runs a fixed number of
iterations (stopping early only on an exactly zero residual or a
non-positive p.Ap, which a positive alpha rules out).  The initial
image is the zero-filled reconstruction Re(A^H b).
"""
from __future__ import annotations

import numpy as np

from . import chalf_map, curvature_map, level_colours, level_side, auto_levels, block_colour


def forward(u, mask):
    """A u = M F u."""
    return mask * np.fft.fft2(u, norm="ortho")


def adjoint(y, mask):
    """A^H y = F^H M y (complex)."""
    return np.fft.ifft2(mask * y, norm="ortho")


def objective(u, kspace, mask, alpha, kind):
    """J(u) = 1/2 ||A u - b||^2 + alpha sum |kappa(u)| (Sec. 5)."""
    res = forward(u, mask) - kspace
    return 0.5 * float(np.sum(np.abs(res) ** 2)) + alpha * float(
        np.sum(np.abs(curvature_map(u, kind))))


def colour_labels(H, W, b, ncolors, k):
    """Per pixel the slot (0 .. n-1) of its block among the blocks of colour
    k on the level of side b, -1 elsewhere; and n."""
    nbi, nbj = -(-H // b), -(-W // b)
    slot = -np.ones((nbi, nbj), dtype=np.int64)
    n = 0
    for bi in range(nbi):
        for bj in range(nbj):
            if block_colour(bi, bj, ncolors) == k:
                slot[bi, bj] = n
                n += 1
    lab = np.repeat(np.repeat(slot, b, axis=0), b, axis=1)[:H, :W]
    return lab, n


def cg(apply, rhs, iters):
    """Conjugate gradients from x = 0, a fixed number of iterations."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    p = r.copy()
    rr = float(r @ r)
    for _ in range(iters):
        if rr == 0.0:
            break
        q = apply(p)
        pq = float(p @ q)
        if pq <= 0.0:     # only a singular system (alpha -> 0) gets here
            break
        a = rr / pq
        x = x + a * p
        r = r - a * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def colour_step(u, kspace, mask, alpha, kind, b, ncolors, k, cg_iters):
    """Joint correction of the blocks of colour k on the level of side b.
    Returns (u + sum c_i phi_i, c)."""
    H, W = u.shape
    lab, n = colour_labels(H, W, b, ncolors, k)
    on = lab >= 0
    idx = lab[on]

    def phi(v):           # sum_i v_i phi_i
        z = np.zeros((H, W))
        z[on] = v[idx]
        return z

    def phi_t(y):         # (<y, phi_i>)_i for a real image y
        return np.bincount(idx, weights=y[on], minlength=n)

    if n == 0:
        return u.copy(), np.zeros(0)
    g = np.real(adjoint(kspace - forward(u, mask), mask))
    if b == 1:
        d = phi_t(chalf_map(u, kind))
    else:
        d = np.zeros(n)
    rhs = phi_t(g) + 2.0 * alpha * d

    def apply(v):
        return phi_t(np.real(adjoint(forward(phi(v), mask), mask))) + 2.0 * alpha * v

    c = cg(apply, rhs, cg_iters)
    return u + phi(c), c


def cycle(u, kspace, mask, alpha, kind, levels=0, ncolors=4, cg_iters=8, sides=0):
    """One fine-to-coarse cycle of colour steps (Alg. 3 order)."""
    H, W = u.shape
    L = levels if levels > 0 else auto_levels(H, W, sides)
    u = np.asarray(u, np.float64).copy()
    for j in range(1, L + 1):
        b = level_side(j, sides)
        nc = level_colours(ncolors, b)
        for k in range(nc):
            u, _ = colour_step(u, kspace, mask, alpha, kind, b, nc, k, cg_iters)
    return u


def solve(kspace, mask, alpha, kind, levels=0, cycles=5, ncolors=4, cg_iters=8, sides=0,
          u0=None):
    """Cycles from u0 (default: the zero-filled Re(A^H b)).  Returns (u, trace
    of J: before the first cycle and after each)."""
    kspace = np.asarray(kspace, np.complex128)
    mask = np.asarray(mask, np.float64)
    u = np.real(adjoint(kspace, mask)) if u0 is None else np.asarray(u0, np.float64).copy()
    trace = [objective(u, kspace, mask, alpha, kind)]
    for _ in range(cycles):
        u = cycle(u, kspace, mask, alpha, kind, levels, ncolors, cg_iters, sides)
        trace.append(objective(u, kspace, mask, alpha, kind))
    return u, np.array(trace)
