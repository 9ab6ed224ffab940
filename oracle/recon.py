"""FP64 oracle of the reconstruction extension (Sec. 5), MRI-like operator.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the product path never
imports it.

Problem (Sec. 5): recover a real image u from data b = A u + noise by
minimising  J(u) = 1/2 ||A u - b||^2 + alpha sum_x |kappa(u(x))|.
Two operators of Sec. 5: MRI, A = M F with F the orthonormal 2-D DFT
(numpy.fft with norm="ortho") and M a 0/1 mask of sampled k-space entries;
and CT, A = R, a parallel-beam Radon transform (defined below).  The multigrid sweep of Sec. 2.2 visits the levels fine to coarse and
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
image is the zero-filled reconstruction Re(A^H b) for MRI and, for CT, the filtered
backprojection (pi / n) R^T (h * b) with the Ram-Lak kernel h[0] = 1/4,
h[k] = -1 / (pi k)^2 for odd k, 0 for even k != 0 (Ramachandran and
Lakshminarayanan, 1971), applied to each angle's projection by direct
convolution over the detector.

CT geometry (READING: Sec. 5 names the Radon transform but no discretisation).
n angles theta_a = pi a / n; the centre of pixel (r, c) is at x = c - (W-1)/2,
y = r - (H-1)/2; its projection t = x cos theta + y sin theta falls at the
position p = t + (D-1)/2 of a detector of D = 2 ceil(hypot(H-1, W-1)/2) + 3
unit bins, and the pixel's value is shared between bins floor(p) and
floor(p) + 1 by linear interpolation (weights 1 - frac(p) and frac(p)).  Every
p lies in [1, D-2], so no weight falls off the detector, and each angle's
projection sums to the image's sum.  The adjoint gathers with the same
weights (a matched pair).
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


def radon_geometry(H, W, n_angles):
    """(D, cos theta_a, sin theta_a) of the CT geometry."""
    D = 2 * int(np.ceil(np.hypot(H - 1, W - 1) / 2.0)) + 3
    th = np.pi * np.arange(n_angles) / n_angles
    return D, np.cos(th), np.sin(th)


def _positions(H, W, c, s, D):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    p = (x - (W - 1) / 2.0) * c + (y - (H - 1) / 2.0) * s + (D - 1) / 2.0
    f = np.floor(p).astype(np.int64)
    return f, p - f


def radon_forward(u, n_angles):
    """R u: n_angles x D sinogram (linear-interpolation splat of every pixel)."""
    u = np.asarray(u, np.float64)
    H, W = u.shape
    D, cs, sn = radon_geometry(H, W, n_angles)
    out = np.zeros((n_angles, D))
    for a in range(n_angles):
        f, w = _positions(H, W, cs[a], sn[a], D)
        np.add.at(out[a], f.ravel(), ((1.0 - w) * u).ravel())
        np.add.at(out[a], f.ravel() + 1, (w * u).ravel())
    return out


def radon_adjoint(sino, H, W):
    """R^T y: every pixel gathers its two bins per angle with its weights."""
    sino = np.asarray(sino, np.float64)
    n_angles, D = sino.shape
    D2, cs, sn = radon_geometry(H, W, n_angles)
    assert D == D2
    img = np.zeros((H, W))
    for a in range(n_angles):
        f, w = _positions(H, W, cs[a], sn[a], D)
        img += (1.0 - w) * sino[a][f] + w * sino[a][f + 1]
    return img


def ramp_filter(sino):
    """Each angle's projection convolved with the Ram-Lak kernel (the
    detector's D bins, zero outside)."""
    sino = np.asarray(sino, np.float64)
    D = sino.shape[1]
    k = np.arange(-(D - 1), D)
    h = np.zeros(k.shape)
    h[k == 0] = 0.25
    odd = (k % 2) != 0
    h[odd] = -1.0 / (np.pi * k[odd]) ** 2
    return np.array([np.convolve(row, h)[D - 1:2 * D - 1] for row in sino])


def fbp(sino, H, W):
    """Filtered backprojection (pi / n) R^T (h * b)."""
    n = np.asarray(sino).shape[0]
    return radon_adjoint(ramp_filter(sino), H, W) * (np.pi / n)


class MriOp:
    """A = M F and its adjoint (real part taken by the caller)."""

    def __init__(self, mask):
        self.mask = np.asarray(mask, np.float64)

    def fwd(self, u):
        return forward(u, self.mask)

    def adj(self, y):
        return np.real(adjoint(y, self.mask))


class CtOp:
    """A = R (parallel-beam Radon transform of the CT geometry) and R^T."""

    def __init__(self, H, W, n_angles):
        self.H, self.W, self.n = H, W, n_angles

    def fwd(self, u):
        return radon_forward(u, self.n)

    def adj(self, y):
        return radon_adjoint(y, self.H, self.W)


def objective_op(u, data, op, alpha, kind):
    """J(u) = 1/2 ||A u - b||^2 + alpha sum |kappa(u)| (Sec. 5)."""
    res = op.fwd(u) - data
    return 0.5 * float(np.sum(np.abs(res) ** 2)) + alpha * float(
        np.sum(np.abs(curvature_map(u, kind))))


def objective(u, kspace, mask, alpha, kind):
    """J(u) for the MRI operator."""
    return objective_op(u, np.asarray(kspace, np.complex128), MriOp(mask), alpha, kind)


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
    """Joint correction of the blocks of colour k on the level of side b, MRI
    operator.  Returns (u + sum c_i phi_i, c)."""
    return colour_step_op(u, np.asarray(kspace, np.complex128), MriOp(mask), alpha, kind, b,
                          ncolors, k, cg_iters)


def colour_step_op(u, data, op, alpha, kind, b, ncolors, k, cg_iters):
    """Joint correction of the blocks of colour k on the level of side b for
    the operator op (fwd, adj).  Returns (u + sum c_i phi_i, c)."""
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
    g = op.adj(data - op.fwd(u))
    if b == 1:
        d = phi_t(chalf_map(u, kind))
    else:
        d = np.zeros(n)
    rhs = phi_t(g) + 2.0 * alpha * d

    def apply(v):
        return phi_t(op.adj(op.fwd(phi(v)))) + 2.0 * alpha * v

    c = cg(apply, rhs, cg_iters)
    return u + phi(c), c


def cycle(u, kspace, mask, alpha, kind, levels=0, ncolors=4, cg_iters=8, sides=0):
    """One fine-to-coarse cycle of colour steps (Alg. 3 order), MRI operator."""
    return cycle_op(u, np.asarray(kspace, np.complex128), MriOp(mask), alpha, kind, levels,
                    ncolors, cg_iters, sides)


def cycle_op(u, data, op, alpha, kind, levels=0, ncolors=4, cg_iters=8, sides=0):
    """One fine-to-coarse cycle of colour steps (Alg. 3 order)."""
    H, W = u.shape
    L = levels if levels > 0 else auto_levels(H, W, sides)
    u = np.asarray(u, np.float64).copy()
    for j in range(1, L + 1):
        b = level_side(j, sides)
        nc = level_colours(ncolors, b)
        for k in range(nc):
            u, _ = colour_step_op(u, data, op, alpha, kind, b, nc, k, cg_iters)
    return u


def solve(kspace, mask, alpha, kind, levels=0, cycles=5, ncolors=4, cg_iters=8, sides=0,
          u0=None):
    """Cycles from u0 (default: the zero-filled Re(A^H b)).  Returns (u, trace
    of J: before the first cycle and after each)."""
    kspace = np.asarray(kspace, np.complex128)
    op = MriOp(mask)
    u = op.adj(kspace) if u0 is None else np.asarray(u0, np.float64).copy()
    return _solve(u, kspace, op, alpha, kind, levels, cycles, ncolors, cg_iters, sides)


def solve_ct(sino, H, W, alpha, kind, levels=0, cycles=5, ncolors=4, cg_iters=8, sides=0,
             u0=None):
    """The CT case: sino is the n_angles x D sinogram.  Start: u0, else the
    filtered backprojection."""
    sino = np.asarray(sino, np.float64)
    op = CtOp(H, W, sino.shape[0])
    u = fbp(sino, H, W) if u0 is None else np.asarray(u0, np.float64).copy()
    return _solve(u, sino, op, alpha, kind, levels, cycles, ncolors, cg_iters, sides)


def _solve(u, data, op, alpha, kind, levels, cycles, ncolors, cg_iters, sides):
    trace = [objective_op(u, data, op, alpha, kind)]
    for _ in range(cycles):
        u = cycle_op(u, data, op, alpha, kind, levels, ncolors, cg_iters, sides)
        trace.append(objective_op(u, data, op, alpha, kind))
    return u, np.array(trace)
