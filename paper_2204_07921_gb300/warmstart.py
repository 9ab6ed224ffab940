"""Learned warm start: a small CNN maps f to an initial u for the sweep.

Binding of the cm_net_* / cm_warmstart entry points of libcm plus the
training driver.  Every forward, backward and Adam step runs in the CUDA
kernels of the library; this module only generates the seeded training
pairs (the plain solver computes u*), batches them and calls the library.

Network (see include/cm.h): six 3x3 convolutions, 32 channels, ReLU,
residual output u0 = f + conv6(...), BF16 weights and activations, FP32
accumulation.
"""
from __future__ import annotations

import ctypes
import os
import time

import numpy as np

from . import (CM_OK, CMError, Context, _P, _I, _F, _D, _ctx, _stream_ptr, load,
               cm_solve_batched)

N_PARAMS = 37601


class TrainOpts(ctypes.Structure):
    """cm_train_opts of include/cm.h."""
    _fields_ = [("steps", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_float),
                ("lr_final", ctypes.c_float), ("total_steps", ctypes.c_int),
                ("start_step", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("log_every", ctypes.c_int)]


class TrainLog(ctypes.Structure):
    """cm_train_log of include/cm.h."""
    _fields_ = [("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double),
                ("n_logged", ctypes.c_int), ("losses_cap", ctypes.c_int),
                ("losses", ctypes.POINTER(ctypes.c_double)),
                ("logged_steps", ctypes.POINTER(ctypes.c_int))]


_SIGS = {
    "cm_net_num_params": (_I, []),
    "cm_net_create": (_I, [_P, ctypes.POINTER(_P)]),
    "cm_net_destroy": (None, [_P]),
    "cm_net_last_error": (ctypes.c_char_p, [_P]),
    "cm_net_set_params": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "cm_net_get_params": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
    "cm_net_forward": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "cm_net_gradients": (_I, [_P, _P, _P, _I, _I, _I, ctypes.POINTER(ctypes.c_float),
                              ctypes.POINTER(_D), _P]),
    "cm_net_train_step": (_I, [_P, _P, _P, _I, _I, _I, _F, ctypes.POINTER(_D), _P]),
    "cm_warmstart": (_I, [_P, _P, _P, _I, _I, _I, _P, _I, _F, _I, ctypes.POINTER(_I), _P]),
    "cm_net_save": (_I, [_P, ctypes.c_char_p]),
    "cm_net_load": (_I, [_P, ctypes.c_char_p]),
    "cm_net_train": (_I, [_P, _P, _P, _P, _I, _I, _I, ctypes.POINTER(TrainOpts),
                          ctypes.POINTER(TrainLog), _P]),
}
_bound = False


def _lib():
    global _bound
    L = load()
    if not _bound:
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _bound = True
    return L


def init_params(seed: int, zero_last: bool = True) -> np.ndarray:
    """He-normal weights for the ReLU layers (std sqrt(2 / fan_in)), zero
    biases, and (by default) a zero last layer so that the untrained network
    returns f exactly."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 9), 9 * 32), np.zeros(32)]
    for _ in range(4):
        parts += [rng.normal(0, np.sqrt(2 / (9 * 32)), 9 * 32 * 32), np.zeros(32)]
    parts += [np.zeros(9 * 32) if zero_last else rng.normal(0, np.sqrt(1 / (9 * 32)), 9 * 32),
              np.zeros(1)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == N_PARAMS
    return p


def _batch(t, name="f", shape=None, like=None):
    """(t, N, H, W) of a contiguous CUDA float32 batch, (H, W) or (N, H, W),
    checked against `shape` and the device of `like` when given, before its
    pointer reaches the library, which trusts the sizes it is given."""
    import torch
    from . import _on_gpu
    if not (isinstance(t, torch.Tensor) and _on_gpu(t) and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError(f"{name}: expected a contiguous CUDA float32 tensor")
    if t.dim() not in (2, 3):
        raise ValueError(f"{name}: expected (H, W) or (N, H, W)")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if like is not None and t.device != like.device:
        raise ValueError(f"{name}: on {t.device}, expected {like.device}")
    if t.dim() == 2:
        return t, 1, t.shape[0], t.shape[1]
    return t, t.shape[0], t.shape[1], t.shape[2]


class Net:
    """A cm_net: FP32 master parameters, Adam moments, BF16 copies, buffers."""

    def __init__(self, params: np.ndarray | None = None, ctx: Context | None = None):
        import torch
        self.ctx = ctx or _ctx(None, torch.empty(1, device="cuda"))
        self._h = _P()
        rc = _lib().cm_net_create(self.ctx.handle, ctypes.byref(self._h))
        if rc != CM_OK:
            raise CMError(rc, "cm_net_create failed")
        if params is not None:
            self.set_params(params)

    def _check(self, rc):
        if rc != CM_OK:
            raise CMError(rc, _lib().cm_net_last_error(self._h).decode())

    def close(self):
        if self._h:
            _lib().cm_net_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != N_PARAMS:
            raise ValueError(f"expected {N_PARAMS} parameters")
        self._check(_lib().cm_net_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self) -> np.ndarray:
        p = np.zeros(N_PARAMS, np.float32)
        self._check(_lib().cm_net_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    def forward(self, f, out=None, stream=None):
        import torch
        f, N, H, W = _batch(f)
        out = torch.empty_like(f) if out is None else _batch(out, "out", f.shape, f)[0]
        self._check(_lib().cm_net_forward(self._h, f.data_ptr(), N, H, W, out.data_ptr(),
                                          _stream_ptr(stream)))
        return out

    def gradients(self, f, ustar, stream=None):
        f, N, H, W = _batch(f)
        _batch(ustar, "ustar", f.shape, f)
        g = np.zeros(N_PARAMS, np.float32)
        loss = ctypes.c_double()
        self._check(_lib().cm_net_gradients(self._h, f.data_ptr(), ustar.data_ptr(), N, H, W,
                                            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value, g

    def train_step(self, f, ustar, lr: float, want_loss: bool = True, stream=None):
        f, N, H, W = _batch(f)
        _batch(ustar, "ustar", f.shape, f)
        loss = ctypes.c_double()
        self._check(_lib().cm_net_train_step(self._h, f.data_ptr(), ustar.data_ptr(), N, H, W,
                                             float(lr), ctypes.byref(loss) if want_loss else None,
                                             _stream_ptr(stream)))
        return loss.value if want_loss else None

    def train_native(self, F, U, steps: int, batch: int, lr: float, lr_final: float,
                     seed: int = 0, total_steps: int = 0, start_step: int = 0,
                     log_every: int = 100, stream=None) -> dict:
        """The library's training loop (cm_net_train) on the pairs F, U
        (N x H x W); returns the log (losses with their schedule steps)."""
        F, N, H, W = _batch(F, "F")
        U, _, _, _ = _batch(U, "U", F.shape, F)
        o = TrainOpts(steps=steps, batch=batch, lr=lr, lr_final=lr_final, total_steps=total_steps,
                      start_step=start_step, seed=seed, log_every=log_every)
        cap = steps // log_every + 2
        losses = (ctypes.c_double * cap)()
        at = (ctypes.c_int * cap)()
        lg = TrainLog(losses_cap=cap, losses=losses, logged_steps=at)
        self._check(_lib().cm_net_train(self.ctx.handle, self._h, F.data_ptr(), U.data_ptr(), N,
                                        H, W, ctypes.byref(o), ctypes.byref(lg),
                                        _stream_ptr(stream)))
        n = lg.n_logged
        return {"loss_first": lg.loss_first, "loss_last": lg.loss_last,
                "steps": [at[i] for i in range(n)], "losses": [losses[i] for i in range(n)]}

    def save_checkpoint(self, path: str):
        """Parameters, Adam moments and step (cm_net_save)."""
        self._check(_lib().cm_net_save(self._h, os.fsencode(path)))

    def load_checkpoint(self, path: str):
        self._check(_lib().cm_net_load(self._h, os.fsencode(path)))

    def save(self, path: str, meta: dict | None = None):
        np.savez(path, params=self.get_params(), meta=np.array(repr(meta or {})))

    @classmethod
    def load(cls, path: str, ctx: Context | None = None):
        d = np.load(path)
        return cls(d["params"], ctx=ctx)


def warmstart(net: Net, f, alpha: float, kind: int, check_energy: bool = True, out=None,
              stream=None):
    """u0 = f + net(f) for a batch; with check_energy an image keeps u0 only
    if F(u0) <= F(f).  Returns (u0, used flags)."""
    import torch
    f, N, H, W = _batch(f)
    out = torch.empty_like(f) if out is None else _batch(out, "out", f.shape, f)[0]
    used = (_I * N)()
    rc = _lib().cm_warmstart(net.ctx.handle, net._h, f.data_ptr(), N, H, W, out.data_ptr(),
                             int(check_energy), float(alpha), int(kind), used,
                             _stream_ptr(stream))
    net.ctx._check(rc)
    return out, [int(v) for v in used]


def make_pairs(n: int, side: int, alpha: float = 20.0, kind: int = 0, tol: float = 1e-5,
               split: str = "train", first: int = 0, ctx: Context | None = None,
               batch: int = 64):
    """Seeded (f, u*) pairs: f from the synthetic generator, u* the plain
    method's result at relative-energy tolerance `tol`.  Returns two CUDA
    tensors (n, side, side) and the clean images (numpy)."""
    import torch
    import synth
    F = torch.empty((n, side, side), dtype=torch.float32, device="cuda")
    U = torch.empty_like(F)
    clean = np.empty((n, side, side), np.float32)
    for s in range(0, n, batch):
        imgs = [synth.warmstart_image(split, first + i, side) for i in range(s, min(n, s + batch))]
        for j, im in enumerate(imgs):
            F[s + j].copy_(torch.from_numpy(im.f))
            clean[s + j] = im.clean
        fs = [F[s + j] for j in range(len(imgs))]
        us = [U[s + j] for j in range(len(imgs))]
        cm_solve_batched(fs, [alpha] * len(fs), [kind] * len(fs), tol=tol, cycles=5000,
                         u_outs=us, ctx=ctx)
    return F, U, clean


def train(net: Net, F, U, steps: int, batch: int, lr: float, seed: int = 0, log_every: int = 100,
          lr_final: float | None = None):
    """Adam on mean((u0 - u*)^2) over random mini-batches of the pairs
    (cosine decay of the learning rate to lr_final)."""
    import torch
    rng = np.random.default_rng(seed)
    n = F.shape[0]
    hist = []
    lr_final = lr if lr_final is None else lr_final
    t0 = time.time()
    for it in range(steps):
        idx = torch.from_numpy(rng.choice(n, size=batch, replace=False)).to(F.device)
        fb = F.index_select(0, idx).contiguous()
        ub = U.index_select(0, idx).contiguous()
        a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * it / max(1, steps - 1)))
        want = (it % log_every == 0) or it == steps - 1
        loss = net.train_step(fb, ub, a, want_loss=want)
        if want:
            hist.append((it, loss, time.time() - t0))
    return hist


def evaluate(net: Net, n: int = 16, side: int = 1024, alpha: float = 20.0, kind: int = 0,
             tol: float = 1e-4, ctx: Context | None = None):
    """Time to tolerance and PSNR on fresh test images: the plain sweep from
    f against the warm start (network inference with the energy check, then
    the sweep from u0), both as one batched solve of the n images and as n
    single solves.  Times are CUDA-event times of the whole call."""
    import torch
    import synth
    imgs = [synth.warmstart_image("test", i, side) for i in range(n)]
    F = torch.stack([torch.from_numpy(im.f) for im in imgs]).cuda().contiguous()
    outs = [torch.empty_like(F[0]) for _ in range(n)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    fs = [F[i] for i in range(n)]

    def plain_batched():
        return cm_solve_batched(fs, [alpha] * n, [kind] * n, tol=tol, cycles=5000, u_outs=outs,
                                ctx=ctx)[1]

    U0 = torch.empty_like(F)

    def warm_batched():
        _, used = warmstart(net, F, alpha, kind, check_energy=True, out=U0)
        st = cm_solve_batched(fs, [alpha] * n, [kind] * n, tol=tol, cycles=5000,
                              u0s=[U0[i] for i in range(n)], u_outs=outs, ctx=ctx)[1]
        return st, used

    t_plain, st_plain = timed(plain_batched)
    psnr_plain = [synth.psnr(outs[i].cpu().numpy(), imgs[i].clean) for i in range(n)]
    t_warm, (st_warm, used) = timed(warm_batched)
    psnr_warm = [synth.psnr(outs[i].cpu().numpy(), imgs[i].clean) for i in range(n)]
    t_inf, _ = timed(lambda: warmstart(net, F, alpha, kind, check_energy=True, out=U0))
    return {
        "images": n, "side": side, "alpha": alpha, "kind": kind, "tol": tol,
        "plain_s": t_plain, "warm_s": t_warm, "inference_s": t_inf,
        "speedup": t_plain / t_warm,
        "cycles_plain": [s.cycles_run for s in st_plain],
        "cycles_warm": [s.cycles_run for s in st_warm],
        "used": used,
        "psnr_plain": float(np.mean(psnr_plain)), "psnr_warm": float(np.mean(psnr_warm)),
        "psnr_diff_db": float(np.mean(np.array(psnr_warm) - np.array(psnr_plain))),
        "psnr_diff_min_db": float(np.min(np.array(psnr_warm) - np.array(psnr_plain))),
        "psnr_noisy": float(np.mean([synth.psnr(im.f, im.clean) for im in imgs])),
        "energy_plain": [s.energy_final for s in st_plain],
        "energy_warm": [s.energy_final for s in st_warm],
    }


def evaluate_equal_energy(net: Net, n: int = 16, side: int = 1024, alpha: float = 20.0,
                          kind: int = 0, tol: float = 1e-4, ctx: Context | None = None,
                          images=None):
    """Time to the plain method's final energy and to its PSNR.  For each test
    image the plain sweep from f runs to the tolerance (energy E_p, PSNR
    P_p); the warm-started sweep then runs exactly as many cycles as it needs
    to reach E_p (counted on its energy trace), and, separately, as few cycles
    as it needs to come within 0.05 dB of P_p; each is timed with its
    inference.  Times are CUDA-event times of one image's call each, summed."""
    import torch
    import synth
    from . import cm_solve
    imgs = images if images is not None else [synth.warmstart_image("test", i, side)
                                              for i in range(n)]
    u = None

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    rows = []
    for im in imgs:
        f = torch.from_numpy(im.f).cuda().contiguous()
        u = torch.empty_like(f)
        U0 = torch.empty_like(f)
        tp, sp = timed(lambda: cm_solve(f, alpha, kind, cycles=5000, tol=tol, u_out=u, ctx=ctx)[1])
        psnr_p = synth.psnr(u.cpu().numpy(), im.clean)
        warmstart(net, f, alpha, kind, check_energy=True, out=U0)
        _, sw = cm_solve(f, alpha, kind, cycles=sp.cycles_run, tol=0.0, u0=U0, u_out=u, ctx=ctx)
        tr = sw.trace()
        hit = next((j for j, E in enumerate(tr) if E <= sp.energy_final), None)
        cyc = hit if hit is not None else sp.cycles_run

        def warm_to_energy():
            warmstart(net, f, alpha, kind, check_energy=True, out=U0)
            return cm_solve(f, alpha, kind, cycles=cyc, tol=0.0, u0=U0, u_out=u, ctx=ctx)[1]

        tw, stw = timed(warm_to_energy)
        psnr_w = synth.psnr(u.cpu().numpy(), im.clean)
        # equal PSNR: the fewest warm-started cycles whose result is within
        # 0.05 dB of the plain solve's PSNR (the clean image is known here)
        cq = 0
        while True:
            cm_solve(f, alpha, kind, cycles=cq, tol=0.0, u0=U0, u_out=u, ctx=ctx)
            if synth.psnr(u.cpu().numpy(), im.clean) >= psnr_p - 0.05 or cq >= sp.cycles_run:
                break
            cq += 1

        def warm_to_psnr():
            warmstart(net, f, alpha, kind, check_energy=True, out=U0)
            return cm_solve(f, alpha, kind, cycles=cq, tol=0.0, u0=U0, u_out=u, ctx=ctx)[1]

        tq, _ = timed(warm_to_psnr)
        rows.append({"plain_s": tp, "plain_cycles": sp.cycles_run, "plain_energy": sp.energy_final,
                     "plain_psnr": psnr_p, "warm_s": tw, "warm_cycles": cyc,
                     "warm_reached": hit is not None, "warm_energy": stw.energy_final,
                     "warm_psnr": psnr_w, "psnr_cycles": cq, "psnr_s": tq,
                     "psnr_at_cycles": synth.psnr(u.cpu().numpy(), im.clean)})
    tp = sum(r["plain_s"] for r in rows)
    tw = sum(r["warm_s"] for r in rows)
    d = [r["warm_psnr"] - r["plain_psnr"] for r in rows]
    return {"images": len(rows), "side": imgs[0].f.shape[0], "alpha": alpha, "kind": kind,
            "tol": tol, "plain_s": tp, "warm_s": tw, "speedup": tp / tw,
            "plain_cycles": [r["plain_cycles"] for r in rows],
            "warm_cycles": [r["warm_cycles"] for r in rows],
            "all_reached": all(r["warm_reached"] for r in rows),
            "psnr_diff_db_mean": float(np.mean(d)), "psnr_diff_db_max_abs": float(np.max(np.abs(d))),
            "psnr_plain": float(np.mean([r["plain_psnr"] for r in rows])),
            "psnr_warm": float(np.mean([r["warm_psnr"] for r in rows])),
            "equal_psnr": {"warm_s": sum(r["psnr_s"] for r in rows),
                           "speedup": tp / sum(r["psnr_s"] for r in rows),
                           "warm_cycles": [r["psnr_cycles"] for r in rows],
                           "psnr_diff_db": [r["psnr_at_cycles"] - r["plain_psnr"] for r in rows]}}
