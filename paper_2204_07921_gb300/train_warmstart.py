"""Train the warm-start CNN on the GPU and save its parameters.

    python -m paper_2204_07921_gb300.train_warmstart [--kind mean|gauss] [--alpha A]
        [--pairs 8192] [--side 256] [--steps 12000] [--batch 16] [--lr 2e-3] [--out PATH]

Training pairs: seeded synthetic 256 x 256 images (20 shapes, sigma ~
U(0.03, 0.12)) and the plain method's result u* at relative-energy tolerance
1e-5 (mean curvature with alpha 20 by default; Gaussian curvature with alpha
15 for --kind gauss).  Loss: mean((f + net(f) - u*)^2), Adam with
cosine learning-rate decay.  Every step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
DEFAULT_OUT = os.path.join(DATA, "warmstart_mean_a20.npz")


def default_path(kind: str, alpha: float) -> str:
    return os.path.join(DATA, f"warmstart_{kind}_a{alpha:g}.npz")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=8192)
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--steps", type=int, default=12000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--kind", choices=["mean", "gauss"], default="mean")
    ap.add_argument("--alpha", type=float, default=None,
                    help="fidelity weight (default 20 for mean, 15 for gauss)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--eval", type=int, default=0,
                    help="also evaluate on this many fresh 1024 x 1024 test images")
    a = ap.parse_args(argv)
    import torch
    from paper_2204_07921_gb300 import warmstart as ws

    kind = 0 if a.kind == "mean" else 1
    alpha = a.alpha if a.alpha is not None else (20.0 if kind == 0 else 15.0)
    out = a.out or default_path(a.kind, alpha)
    t0 = time.time()
    F, U, _ = ws.make_pairs(a.pairs, a.side, alpha=alpha, kind=kind, tol=1e-5)
    torch.cuda.synchronize()
    t1 = time.time()
    net = ws.Net(ws.init_params(a.seed, zero_last=True))
    hist = ws.train(net, F, U, a.steps, a.batch, a.lr, seed=a.seed, lr_final=a.lr_final)
    torch.cuda.synchronize()
    t2 = time.time()
    meta = {"pairs": a.pairs, "side": a.side, "steps": a.steps, "batch": a.batch, "lr": a.lr,
            "lr_final": a.lr_final, "seed": a.seed, "kind": a.kind, "alpha": alpha,
            "ustar_tol": 1e-5, "data_s": t1 - t0, "train_s": t2 - t1,
            "loss_first": hist[0][1], "loss_last": hist[-1][1]}
    os.makedirs(os.path.dirname(out), exist_ok=True)
    net.save(out, meta)
    res = {"saved": os.path.relpath(out, ROOT), **meta, "history": hist[:: max(1, len(hist) // 20)]}
    if a.eval:
        res["eval"] = ws.evaluate(net, n=a.eval, alpha=alpha, kind=kind)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
