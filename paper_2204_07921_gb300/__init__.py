"""GB300 multigrid curvature-energy minimisation (Python binding of libcm).

Thin ctypes binding over the C ABI in ``include/cm.h``: every function here
only checks tensor shapes/dtypes/devices and forwards raw device pointers
and the current CUDA stream.  All arithmetic of the method runs in the CUDA
kernels of ``libcm.so``; there is no CPU fallback, and importing a function
that needs the library raises if it cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, build as build_library

__all__ = [
    "CMError", "Options", "Stats", "Context", "load", "cm_energy", "cm_curvature", "cm_phase",
    "cm_level", "cm_energy_noalloc", "cm_solve_batched", "cm_probe_alu", "cm_recon",
    "cm_recon_ct", "cm_radon", "cm_radon_adjoint", "cm_radon_bins", "cm_radon_entries",
    "cm_fft2d",
    "cm_solve", "cm_auto_levels", "MEAN", "GAUSS", "MEAN_EULER", "GAUSS_EULER",
]

# Curvature kinds: H or K from the extreme direction curvatures (Sec. 3), or
# from a least-squares fit of Euler's formula to the four directions.
MEAN, GAUSS, MEAN_EULER, GAUSS_EULER = 0, 1, 2, 3
CM_OK, CM_ERR_INVALID, CM_ERR_CUDA, CM_ERR_OOM = 0, 1, 2, 3
CM_ERR_TIMEOUT, CM_ERR_NUMERIC, CM_NOT_CONVERGED = 4, 5, 6
STATUS_NAMES = {0: "CM_OK", 1: "CM_ERR_INVALID", 2: "CM_ERR_CUDA", 3: "CM_ERR_OOM",
                4: "CM_ERR_TIMEOUT", 5: "CM_ERR_NUMERIC", 6: "CM_NOT_CONVERGED"}


class CMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("ncolors", ctypes.c_int), ("grid_points", ctypes.c_int),
                ("golden_evals", ctypes.c_int), ("paper_candidate", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("max_trace", ctypes.c_int),
                ("one_step", ctypes.c_int), ("vcycle", ctypes.c_int),
                ("coarse_spec", ctypes.c_int), ("coarse_dmax", ctypes.c_int),
                ("coarse_ncolors", ctypes.c_int), ("block_sides", ctypes.c_int),
                ("shapes", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("cycles_run", ctypes.c_int), ("converged", ctypes.c_int),
                ("monotone_violations", ctypes.c_int), ("levels", ctypes.c_int),
                ("energy_initial", ctypes.c_double), ("energy_final", ctypes.c_double),
                ("trace_len", ctypes.c_int), ("energy_trace", ctypes.c_double * 4097)]

    def trace(self):
        return list(self.energy_trace[: self.trace_len])


_lib = None
_lock = threading.Lock()

_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_D = ctypes.c_double
SIGNATURES = {
    "cm_options_default": (_I, [ctypes.POINTER(Options)]),
    "cm_create": (_I, [ctypes.POINTER(_P), _I]),
    "cm_destroy": (None, [_P]),
    "cm_last_error": (ctypes.c_char_p, [_P]),
    "cm_auto_levels": (_I, [_I, _I]),
    "cm_energy": (_I, [_P, _P, _P, _I, _I, _F, _I, ctypes.POINTER(_D), _P]),
    "cm_curvature": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "cm_phase": (_I, [_P, _P, _P, _P, _I, _I, _F, _I, _I, _I, ctypes.POINTER(Options), _P, _P]),
    "cm_probe_alu": (_I, [_I, _P, _P, _P]),
    "cm_selftest_wait": (_I, [_I, _I, _P, _P]),
    "cm_energy_noalloc": (_I, [_P, _P, _I, _I, _F, _I, _P, _P]),
    "cm_radon_bins": (_I, [_I, _I]),
    "cm_radon_entries": (ctypes.c_longlong, [_I, _I, _I]),
    "cm_radon": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "cm_radon_adjoint": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "cm_recon_ct": (_I, [_P, _P, _I, _I, _I, _F, _I, _I, _I, _I, _P, _P,
                         ctypes.POINTER(Options), _P, _P]),
    "cm_fft2d": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "cm_recon": (_I, [_P, _P, _P, _I, _I, _F, _I, _I, _I, _I, _P, _P, ctypes.POINTER(Options),
                      _P, _P]),
    "cm_level": (_I, [_P, _P, _P, _P, _I, _I, _F, _I, _I, ctypes.POINTER(Options), _P, _P]),
    "cm_solve_batched": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_I),
                              ctypes.POINTER(_F), ctypes.POINTER(_I), _I, _I, _D,
                              ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(Options),
                              ctypes.POINTER(Stats), _P]),
    "cm_solve": (_I, [_P, _P, _I, _I, _F, _I, _I, _I, _D, _P, _P, ctypes.POINTER(Options),
                      ctypes.POINTER(Stats), _P]),
}


def load(path: str | None = None):
    """Load libcm.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or LIB
            if path is None:
                build_library()
            if not os.path.exists(so):
                raise RuntimeError(f"libcm not found at {so}")
            L = ctypes.CDLL(so)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    load().cm_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


def cm_auto_levels(H: int, W: int) -> int:
    return load().cm_auto_levels(H, W)


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _on_gpu(t) -> bool:
    return t.is_cuda


def _img(t, name, shape=None, like=None):
    """Checks that t is a contiguous CUDA float32 matrix (of `shape`, on the
    device of `like`) before its pointer reaches the library, which trusts
    the sizes it is given."""
    import torch
    if not isinstance(t, torch.Tensor) or not _on_gpu(t) or t.dtype != torch.float32:
        raise TypeError(f"{name}: expected a CUDA float32 tensor")
    if t.dim() != 2 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous H x W tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if like is not None and t.device != like.device:
        raise ValueError(f"{name}: on {t.device}, expected {like.device}")
    return t


def _blocks_out(c_out, H, W, b, like):
    """c_out of cm_phase / cm_level: CUDA float32, one entry per block of the
    level (ceil(H / b) x ceil(W / b)); None passes through."""
    import torch
    if c_out is None:
        return None
    if not (isinstance(c_out, torch.Tensor) and _on_gpu(c_out) and c_out.dtype == torch.float32
            and c_out.is_contiguous()):
        raise TypeError("c_out: expected a contiguous CUDA float32 tensor")
    if b < 1:
        raise ValueError("b: expected a block side >= 1")
    nb = ((H + b - 1) // b) * ((W + b - 1) // b)
    if c_out.numel() < nb:
        raise ValueError(f"c_out: {c_out.numel()} entries, the level has {nb} blocks")
    if c_out.device != like.device:
        raise ValueError(f"c_out: on {c_out.device}, expected {like.device}")
    return c_out.data_ptr()


class Context:
    """Owns a cm_ctx (scratch memory and cached CUDA graphs) on one device."""

    def __init__(self, device: int | None = None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        self._h = _P()
        rc = load().cm_create(ctypes.byref(self._h), device)
        if rc != CM_OK:
            raise CMError(rc, "cm_create failed")

    def close(self):
        if self._h:
            load().cm_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, ok=(CM_OK,)):
        if rc not in ok:
            raise CMError(rc, load().cm_last_error(self._h).decode())
        return rc

    @property
    def handle(self):
        return self._h


_default_ctx = {}


def _ctx(ctx: Context | None, t) -> Context:
    if ctx is not None:
        return ctx
    dev = t.device.index if t.device.index is not None else 0
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


def cm_energy(u, f, alpha: float, kind: int, ctx: Context | None = None, stream=None) -> float:
    """F(u) of Eq. (MCM)/(GCM), FP64 device reduction."""
    _img(u, "u")
    _img(f, "f", u.shape, u)
    c = _ctx(ctx, u)
    H, W = u.shape
    E = ctypes.c_double(0.0)
    c._check(load().cm_energy(c.handle, u.data_ptr(), f.data_ptr(), H, W, float(alpha), kind,
                              ctypes.byref(E), _stream_ptr(stream)))
    return E.value


def cm_selftest_wait(device: int = 0, limit: int = 1024) -> dict:
    """Bounded-wait self-test: a wait that nothing completes must time out,
    and the same wait after one arrival must complete."""
    t, c = ctypes.c_int(-1), ctypes.c_int(-1)
    rc = load().cm_selftest_wait(device, limit, ctypes.byref(t), ctypes.byref(c))
    if rc != CM_OK:
        raise CMError(rc, "cm_selftest_wait failed")
    return {"timed_out": t.value, "completed": c.value}


def cm_probe_alu(device: int = 0, stream=None) -> dict:
    """Measured FP32 FMA and rsqrtf rates of the GPU (operations per second)."""
    fma, rsq = ctypes.c_double(), ctypes.c_double()
    rc = load().cm_probe_alu(device, ctypes.byref(fma), ctypes.byref(rsq), _stream_ptr(stream))
    if rc != CM_OK:
        raise CMError(rc, "cm_probe_alu failed")
    return {"fma_per_s": fma.value, "rsqrt_per_s": rsq.value}


def cm_energy_noalloc(u, f, alpha: float, kind: int, E_out, stream=None):
    """F(u) into the one-element float64 CUDA tensor E_out, without any
    device allocation (the library's fixed scratch array; see include/cm.h)."""
    import torch
    _img(u, "u")
    _img(f, "f", u.shape, u)
    if not (isinstance(E_out, torch.Tensor) and _on_gpu(E_out) and
            E_out.dtype == torch.float64 and E_out.numel() >= 1):
        raise TypeError("E_out: expected a CUDA float64 tensor")
    if E_out.device != u.device:
        raise ValueError(f"E_out: on {E_out.device}, expected {u.device}")
    H, W = u.shape
    rc = load().cm_energy_noalloc(u.data_ptr(), f.data_ptr(), H, W, float(alpha), kind,
                                  E_out.data_ptr(), _stream_ptr(stream))
    if rc != CM_OK:
        raise CMError(rc, "cm_energy_noalloc failed")
    return E_out


def cm_curvature(u, kind: int, out=None, ctx: Context | None = None, stream=None):
    import torch
    _img(u, "u")
    out = torch.empty_like(u) if out is None else _img(out, "out", u.shape, u)
    c = _ctx(ctx, u)
    H, W = u.shape
    c._check(load().cm_curvature(c.handle, u.data_ptr(), H, W, kind, out.data_ptr(),
                                 _stream_ptr(stream)))
    return out


def cm_phase(S, R, f, alpha: float, kind: int, b: int, colour: int, options: Options | None = None,
             c_out=None, ctx: Context | None = None, stream=None):
    """One (level, colour) phase: writes R on the colour's blocks."""
    _img(S, "S")
    H, W = S.shape
    _img(R, "R", S.shape, S)
    _img(f, "f", S.shape, S)
    cp = _blocks_out(c_out, H, W, b, S)
    c = _ctx(ctx, S)
    opts = options or default_options()
    c._check(load().cm_phase(c.handle, S.data_ptr(), R.data_ptr(), f.data_ptr(), H, W,
                             float(alpha), kind, b, colour, ctypes.byref(opts), cp,
                             _stream_ptr(stream)))
    return R


def cm_level(S, R, f, alpha: float, kind: int, b: int, options: Options | None = None,
             c_out=None, ctx: Context | None = None, stream=None):
    """One whole level (every colour) from state S; R receives the new state."""
    _img(S, "S")
    H, W = S.shape
    _img(R, "R", S.shape, S)
    _img(f, "f", S.shape, S)
    cp = _blocks_out(c_out, H, W, b, S)
    c = _ctx(ctx, S)
    opts = options or default_options()
    c._check(load().cm_level(c.handle, S.data_ptr(), R.data_ptr(), f.data_ptr(), H, W,
                             float(alpha), kind, b, ctypes.byref(opts), cp,
                             _stream_ptr(stream)))
    return R


def cm_solve(f, alpha: float, kind: int, levels: int = 0, cycles: int = 20, tol: float = 0.0,
             u0=None, u_out=None, options: Options | None = None, ctx: Context | None = None,
             stream=None):
    """Alg. 3 solve on the device.  Returns (u_out, Stats)."""
    import torch
    _img(f, "f")
    H, W = f.shape
    if u_out is None:
        u_out = torch.empty_like(f)
    _img(u_out, "u_out", f.shape, f)
    if u0 is not None:
        _img(u0, "u0", f.shape, f)
    c = _ctx(ctx, f)
    opts = options or default_options()
    st = Stats()
    c._check(load().cm_solve(c.handle, f.data_ptr(), H, W, float(alpha), kind, levels, cycles,
                             float(tol), u0.data_ptr() if u0 is not None else None,
                             u_out.data_ptr(), ctypes.byref(opts), ctypes.byref(st),
                             _stream_ptr(stream)),
             ok=(CM_OK, CM_NOT_CONVERGED))
    return u_out, st


def cm_fft2d(x, inverse: bool = False, out=None, ctx: Context | None = None, stream=None):
    """Unnormalised 2-D DFT of a CUDA complex64 H x W tensor (the library's
    own transform of the MRI-like operator; exp(-2 pi i ...) forward,
    exp(+2 pi i ...) inverse).  Returns out (may be x: in place)."""
    import torch
    if not (isinstance(x, torch.Tensor) and _on_gpu(x) and x.dtype == torch.complex64 and
            x.dim() == 2 and x.is_contiguous()):
        raise TypeError("x: expected a contiguous CUDA complex64 H x W tensor")
    H, W = x.shape
    if out is None:
        out = torch.empty_like(x)
    elif not (isinstance(out, torch.Tensor) and out.dtype == torch.complex64 and
              out.shape == x.shape and out.is_contiguous() and out.device == x.device):
        raise TypeError("out: expected a contiguous complex64 tensor of x's shape and device")
    c = _ctx(ctx, x)
    c._check(load().cm_fft2d(c.handle, x.data_ptr(), out.data_ptr(), H, W, int(bool(inverse)),
                             _stream_ptr(stream)))
    return out


def cm_recon(kspace, mask, alpha: float, kind: int = MEAN, levels: int = 0, cycles: int = 5,
             cg_iters: int = 8, u0=None, u_out=None, options: Options | None = None,
             ctx: Context | None = None, stream=None):
    """Reconstruction (Sec. 5) from k-space data of A = M F.  kspace: CUDA
    complex64 H x W (zero off the mask); mask: CUDA uint8 H x W.  Returns
    (u_out, trace of J: before the first cycle and after each)."""
    import numpy as np
    import torch
    if not (isinstance(kspace, torch.Tensor) and _on_gpu(kspace) and
            kspace.dtype == torch.complex64 and kspace.dim() == 2 and kspace.is_contiguous()):
        raise TypeError("kspace: expected a contiguous CUDA complex64 H x W tensor")
    if not (isinstance(mask, torch.Tensor) and _on_gpu(mask) and mask.dtype == torch.uint8 and
            mask.shape == kspace.shape and mask.is_contiguous() and
            mask.device == kspace.device):
        raise TypeError("mask: expected a contiguous CUDA uint8 tensor of the data's shape "
                        "and device")
    H, W = kspace.shape
    if u_out is None:
        u_out = torch.empty((H, W), dtype=torch.float32, device=kspace.device)
    _img(u_out, "u_out", (H, W), kspace)
    if u0 is not None:
        _img(u0, "u0", (H, W), kspace)
    if cycles < 0:
        raise ValueError("cycles: expected >= 0")
    c = _ctx(ctx, kspace)
    opts = options or default_options()
    trace = np.zeros(cycles + 1)
    c._check(load().cm_recon(c.handle, kspace.data_ptr(), mask.data_ptr(), H, W, float(alpha),
                             kind, levels, cycles, cg_iters,
                             u0.data_ptr() if u0 is not None else None, u_out.data_ptr(),
                             ctypes.byref(opts), trace.ctypes.data_as(ctypes.c_void_p),
                             _stream_ptr(stream)))
    return u_out, trace


def cm_radon_bins(H: int, W: int) -> int:
    """Detector bins of the CT geometry."""
    D = load().cm_radon_bins(H, W)
    if D < 0:
        raise ValueError(f"image size {H} x {W} out of range")
    return D


def cm_radon_entries(H: int, W: int, n_angles: int) -> int:
    """Entries of the n_angles x D sinogram of an H x W image; ValueError
    where the library's limits reject the case."""
    m = load().cm_radon_entries(H, W, n_angles)
    if m < 0:
        raise ValueError(f"CT case {H} x {W} with {n_angles} angles out of range")
    return m


def _sinogram(sino, H, W):
    """sino: n_angles x cm_radon_bins(H, W), n_angles >= 1."""
    _img(sino, "sino")
    if H < 1 or W < 1:
        raise ValueError("H, W: expected >= 1")
    D = cm_radon_bins(H, W)
    if sino.shape[0] < 1 or sino.shape[1] != D:
        raise ValueError(f"sino: expected n_angles x {D} for a {H} x {W} image, "
                         f"got {tuple(sino.shape)}")
    cm_radon_entries(H, W, sino.shape[0])


def cm_radon(u, n_angles: int, ctx: Context | None = None, stream=None):
    """sino = R u (n_angles x cm_radon_bins(H, W))."""
    import torch
    _img(u, "u")
    if n_angles < 1:
        raise ValueError("n_angles: expected >= 1")
    c = _ctx(ctx, u)
    H, W = u.shape
    cm_radon_entries(H, W, n_angles)
    sino = torch.empty((n_angles, cm_radon_bins(H, W)), dtype=torch.float32, device=u.device)
    c._check(load().cm_radon(c.handle, u.data_ptr(), H, W, n_angles, sino.data_ptr(),
                             _stream_ptr(stream)))
    return sino


def cm_radon_adjoint(sino, H: int, W: int, ctx: Context | None = None, stream=None):
    """u = R^T sino."""
    import torch
    _sinogram(sino, H, W)
    c = _ctx(ctx, sino)
    u = torch.empty((H, W), dtype=torch.float32, device=sino.device)
    c._check(load().cm_radon_adjoint(c.handle, sino.data_ptr(), sino.shape[0], H, W,
                                     u.data_ptr(), _stream_ptr(stream)))
    return u


def cm_recon_ct(sino, H: int, W: int, alpha: float, kind: int = MEAN, levels: int = 0,
                cycles: int = 5, cg_iters: int = 8, u0=None, u_out=None,
                options: Options | None = None, ctx: Context | None = None, stream=None):
    """CT reconstruction (Sec. 5, A = R) from the n_angles x D sinogram.
    Returns (u_out, trace of J)."""
    import numpy as np
    import torch
    _sinogram(sino, H, W)
    if u_out is None:
        u_out = torch.empty((H, W), dtype=torch.float32, device=sino.device)
    _img(u_out, "u_out", (H, W), sino)
    if u0 is not None:
        _img(u0, "u0", (H, W), sino)
    if cycles < 0:
        raise ValueError("cycles: expected >= 0")
    c = _ctx(ctx, sino)
    opts = options or default_options()
    trace = np.zeros(cycles + 1)
    c._check(load().cm_recon_ct(c.handle, sino.data_ptr(), sino.shape[0], H, W, float(alpha),
                                kind, levels, cycles, cg_iters,
                                u0.data_ptr() if u0 is not None else None, u_out.data_ptr(),
                                ctypes.byref(opts), trace.ctypes.data_as(ctypes.c_void_p),
                                _stream_ptr(stream)))
    return u_out, trace


def cm_solve_batched(fs, alphas, kinds, levels: int = 0, cycles: int = 2000, tol: float = 1e-4,
                     u0s=None, u_outs=None, options: Options | None = None,
                     ctx: Context | None = None, stream=None):
    """Solve many images (lists of CUDA float32 H x W tensors) together.
    Returns (u_outs, [Stats])."""
    import torch
    n = len(fs)
    if n == 0:
        return [], []
    if len(alphas) != n or len(kinds) != n:
        raise ValueError(f"alphas, kinds: expected {n} entries each, got {len(alphas)} and "
                         f"{len(kinds)}")
    for i, t in enumerate(fs):
        _img(t, f"f[{i}]", like=fs[0])
    if u_outs is None:
        u_outs = [torch.empty_like(t) for t in fs]
    if len(u_outs) != n or (u0s is not None and len(u0s) != n):
        raise ValueError(f"u_outs, u0s: expected {n} entries")
    for i in range(n):
        _img(u_outs[i], f"u_outs[{i}]", fs[i].shape, fs[0])
        if u0s is not None and u0s[i] is not None:
            _img(u0s[i], f"u0s[{i}]", fs[i].shape, fs[0])
    c = _ctx(ctx, fs[0])
    PA = _P * n
    f_arr = PA(*[t.data_ptr() for t in fs])
    u_arr = PA(*[t.data_ptr() for t in u_outs])
    u0_arr = PA(*[(t.data_ptr() if t is not None else None) for t in u0s]) if u0s else None
    H = (_I * n)(*[t.shape[0] for t in fs])
    W = (_I * n)(*[t.shape[1] for t in fs])
    al = (_F * n)(*[float(a) for a in alphas])
    kd = (_I * n)(*[int(k) for k in kinds])
    opts = options or default_options()
    stats = (Stats * n)()
    c._check(load().cm_solve_batched(c.handle, n, f_arr, H, W, al, kd, levels, cycles, float(tol),
                                     u0_arr, u_arr, ctypes.byref(opts), stats,
                                     _stream_ptr(stream)),
             ok=(CM_OK, CM_NOT_CONVERGED))
    return u_outs, list(stats)
