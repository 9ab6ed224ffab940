"""FP64 CPU oracle of the multigrid curvature-energy sweep.

TEST INFRASTRUCTURE ONLY: the plain restatement of the paper's method that
the CUDA library is checked against.  Only ``tests/``, the package smoke check
and the benchmark's CPU-baseline leg load it; the product path never does.
It shares no code with the CUDA path.

The numerics live in ``cm_oracle.c`` (plain C, IEEE double, optional OpenMP
over the blocks of one colour, which the phase's snapshot semantics make
order-independent).  This module compiles it with gcc and wraps it with
ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None
# ring(c, ctx) -> sum over the block's ring of |kappa_q(u + c phi_A)|
_RING_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)

MEAN, GAUSS = 0, 1
# Extension: principal curvatures from a least-squares fit of Euler's formula
# to the four direction curvatures (instead of their extremes).
MEAN_EULER, GAUSS_EULER = 2, 3
# Default search budget: the same as the library's default options.
DEFAULT_G, DEFAULT_K = 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            i, d = ctypes.c_int, ctypes.c_double
            sig = {
                "orc_plane_distance": (d, [dp, dp, dp, dp]),
                "orc_direction_curvatures": (None, [dp, i, i, i, i, dp, dp]),
                "orc_curvature": (d, [dp, i, i, i, i, i]),
                "orc_curvature_map": (None, [dp, i, i, i, dp]),
                "orc_energy": (d, [dp, dp, i, i, d, i]),
                "orc_local_energy": (d, [dp, dp, i, i, i, i, i, i, d, d, i]),
                "orc_ring_size": (i, [i, i, i, i, i, i]),
                "orc_paper_candidate": (d, [dp, dp, i, i, i, i, d, i]),
                "orc_block_min": (d, [dp, dp, i, i, i, i, i, i, d, i, i, i, i, i, i, dp]),
                "orc_block_colour": (i, [i, i, i]),
                "orc_auto_levels": (i, [i, i, i]),
                "orc_level_side": (i, [i, i]),
                "orc_phase": (i, [dp, dp, i, i, d, i, i, i, i, i, i, i, i, dp]),
                "orc_level_sequential": (None, [dp, dp, i, i, d, i, i, i, i, i, i]),
                "orc_cycle": (None, [dp, dp, i, i, d, i, i, i, i, i, i, i, i, i, i, i]),
                "orc_solve": (i, [dp, i, i, d, i, i, i, d, dp, dp, i, i, i, i, i, i, i, i, i, dp,
                                  ip]),
                "orc_level_colours": (i, [i, i, i]),
                "orc_chalf_map": (None, [dp, i, i, i, dp]),
                "orc_num_threads": (i, []),
                "orc_set_num_threads": (None, [i]),
                "orc_local_energy_batch": (None, [dp, dp, i, i, i, i, i, i, d, i, dp, i, dp]),
                "orc_block_search": (d, [d, d, d, i, i, i, d, _RING_FN, ctypes.c_void_p, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def plane_distance(X, Y, Z, O) -> float:
    X, Y, Z, O = (_f64(v) for v in (X, Y, Z, O))
    return lib().orc_plane_distance(_dp(X), _dp(Y), _dp(Z), _dp(O))


def direction_curvatures(u, r: int, c: int):
    u = _f64(u)
    H, W = u.shape
    kbar = np.zeros(4)
    d = np.zeros(8)
    lib().orc_direction_curvatures(_dp(u), H, W, r, c, _dp(kbar), _dp(d))
    return kbar, d


def curvature(u, r: int, c: int, kind: int) -> float:
    u = _f64(u)
    H, W = u.shape
    return lib().orc_curvature(_dp(u), H, W, r, c, kind)


def curvature_map(u, kind: int) -> np.ndarray:
    u = _f64(u)
    H, W = u.shape
    out = np.zeros((H, W))
    lib().orc_curvature_map(_dp(u), H, W, kind, _dp(out))
    return out


def energy(u, f, alpha: float, kind: int) -> float:
    u, f = _f64(u), _f64(f)
    H, W = u.shape
    return lib().orc_energy(_dp(u), _dp(f), H, W, float(alpha), kind)


def local_energy(u, f, r0, c0, bh, bw, c, alpha, kind) -> float:
    u, f = _f64(u), _f64(f)
    H, W = u.shape
    return lib().orc_local_energy(_dp(u), _dp(f), H, W, r0, c0, bh, bw, float(c),
                                  float(alpha), kind)


def local_energy_batch(u, f, r0, c0, bh, bw, cs, alpha, kind) -> np.ndarray:
    u, f, cs = _f64(u), _f64(f), _f64(cs)
    H, W = u.shape
    out = np.zeros(cs.size)
    lib().orc_local_energy_batch(_dp(u), _dp(f), H, W, r0, c0, bh, bw, float(alpha), kind,
                                 _dp(cs), cs.size, _dp(out))
    return out


def ring_size(H, W, r0, c0, bh, bw) -> int:
    return lib().orc_ring_size(H, W, r0, c0, bh, bw)


def paper_candidate(u, f, r, c, alpha, kind) -> float:
    u, f = _f64(u), _f64(f)
    H, W = u.shape
    return lib().orc_paper_candidate(_dp(u), _dp(f), H, W, r, c, float(alpha), kind)


def block_min(u, f, r0, c0, bh, bw, alpha, kind, G=DEFAULT_G, K=DEFAULT_K, use_paper=True,
              one_step=False, finest=None):
    """Returns (c, info) with info = dict(E_best, E_zero, c_fid, rho, S1, n_eval).
    one_step: the paper's single step (Alg. 2, t = 0) kept if it lowers E_A;
    finest: the block is on the finest level (default: a 1 x 1 block)."""
    u, f = _f64(u), _f64(f)
    H, W = u.shape
    info = np.zeros(6)
    if finest is None:
        finest = bh == 1 and bw == 1
    c = lib().orc_block_min(_dp(u), _dp(f), H, W, r0, c0, bh, bw, float(alpha), kind, G, K,
                            int(use_paper), int(one_step), int(finest), _dp(info))
    keys = ("E_best", "E_zero", "c_fid", "rho", "S1", "n_eval")
    return c, dict(zip(keys, info.tolist()))


def block_search(s, S1, alpha, ring, G=DEFAULT_G, K=DEFAULT_K, one_step=False, cand=None):
    """The steps of block_min for a block seen only through s = |A|,
    S1 = sum_A (u - f) and ring(c), a callable returning the ring sum
    sum_{q in ring(A)} |kappa_q(u + c phi_A)| (e.g. assembled from the partial
    sums of several row strips); cand: the closed-form candidate (the
    paper's c_1 on the finest level) or None.  ring is called in the search's
    own order, the same on every caller.  Returns (c, info) as block_min."""
    err = []

    def cb(c, _ctx):
        if err:
            return 0.0
        try:
            return float(ring(c))
        except BaseException as e:   # noqa: BLE001 -- re-raised below
            err.append(e)
            return 0.0

    fn = _RING_FN(cb)
    info = np.zeros(6)
    c = lib().orc_block_search(float(s), float(S1), float(alpha), G, K, int(one_step),
                               float("nan") if cand is None else float(cand), fn, None,
                               _dp(info))
    if err:
        raise err[0]
    keys = ("E_best", "E_zero", "c_fid", "rho", "S1", "n_eval")
    return c, dict(zip(keys, info.tolist()))


def block_colour(bi, bj, ncolors) -> int:
    return lib().orc_block_colour(bi, bj, ncolors)


def auto_levels(H, W, sides=0) -> int:
    """Default level count (sides = 1: the paper's block sides 2^j - 1)."""
    return lib().orc_auto_levels(H, W, int(sides))


def level_side(j, sides=0) -> int:
    """Block side of level j = 1, 2, ...: 2^(j-1), or 2^j - 1 with sides = 1."""
    return lib().orc_level_side(j, int(sides))


def phase(u, f, alpha, kind, b, ncolors, k, G=DEFAULT_G, K=DEFAULT_K, use_paper=True,
          one_step=False):
    """One (level, colour) phase from state u; returns (u_new, c_per_block)."""
    u = _f64(u).copy()
    f = _f64(f)
    H, W = u.shape
    nb = ((H + b - 1) // b) * ((W + b - 1) // b)
    cs = np.zeros(nb)
    lib().orc_phase(_dp(u), _dp(f), H, W, float(alpha), kind, b, ncolors, k, G, K,
                    int(use_paper), int(one_step), _dp(cs))
    return u, cs


def level_sequential(u, f, alpha, kind, b, G=DEFAULT_G, K=DEFAULT_K, use_paper=True,
                     one_step=False):
    u = _f64(u).copy()
    f = _f64(f)
    H, W = u.shape
    lib().orc_level_sequential(_dp(u), _dp(f), H, W, float(alpha), kind, b, G, K,
                               int(use_paper), int(one_step))
    return u


def chalf_map(u, kind) -> np.ndarray:
    """c_{1/2} of every pixel: the shift the curvature term alone asks for
    (Eq. c-sol1; Prop. 2 for Gaussian curvature)."""
    u = _f64(u)
    H, W = u.shape
    out = np.zeros((H, W))
    lib().orc_chalf_map(_dp(u), H, W, kind, _dp(out))
    return out


def level_colours(ncolors, b, coarse_ncolors=0) -> int:
    """Colours of the level with block side b (ncolors = 0: decoupled;
    coarse_ncolors, when set, on the levels with b >= 64)."""
    return lib().orc_level_colours(ncolors, b, coarse_ncolors)


def cycle(u, f, alpha, kind, levels=0, ncolors=2, G=DEFAULT_G, K=DEFAULT_K, use_paper=True,
          sequential=False, one_step=False, vcycle=False, sides=0, coarse_ncolors=0):
    u = _f64(u).copy()
    f = _f64(f)
    H, W = u.shape
    lib().orc_cycle(_dp(u), _dp(f), H, W, float(alpha), kind, levels, ncolors, G, K,
                    int(use_paper), int(one_step), int(sequential), int(vcycle), int(sides),
                    int(coarse_ncolors))
    return u


def solve(f, alpha, kind, levels=0, cycles=20, tol=0.0, u0=None, ncolors=2, G=DEFAULT_G,
          K=DEFAULT_K, use_paper=True, sequential=False, one_step=False, vcycle=False,
          sides=0, coarse_ncolors=0):
    """Alg. 3 outer loop.  Returns (u, trace, cycles_run, converged)."""
    f = _f64(f)
    H, W = f.shape
    u = np.zeros_like(f)
    trace = np.zeros(cycles + 1)
    conv = ctypes.c_int(0)
    u0p = None
    if u0 is not None:
        u0a = _f64(u0)
        u0p = _dp(u0a)
    n = lib().orc_solve(_dp(f), H, W, float(alpha), kind, levels, cycles, float(tol), u0p,
                        _dp(u), ncolors, G, K, int(use_paper), int(one_step), int(sequential),
                        int(vcycle), int(sides), int(coarse_ncolors), _dp(trace),
                        ctypes.byref(conv))
    return u, trace[: n + 1], n, bool(conv.value)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """OpenMP threads of the following calls (results do not depend on it)."""
    lib().orc_set_num_threads(int(n))
