"""Autotuner of the block-search budget.

The budget of the block search -- G grid points on the bracket and K
golden-section evaluations -- is a parameter of the method (the oracle takes
the same two numbers).  It trades the cost of a cycle against how far each
block's subproblem is minimised, and on this non-convex energy a very precise
per-block search can also settle in worse local minima than a coarser one.
The tuner times a solve to tolerance on a calibration image of the requested
shape class (a seeded image that is not one of the measured workloads) for
each candidate budget, and picks the fastest whose final energy is within
`ENERGY_SLACK` of the lowest final energy any candidate reached.  Results are
cached per GPU model in a JSON file ($CM_AUTOTUNE_CACHE, else
~/.cache/cm_autotune.json).
"""
from __future__ import annotations

import json
import os

CANDIDATES = ((9, 16), (7, 10), (5, 8), (5, 6), (5, 4), (3, 4))
ENERGY_SLACK = 2e-3


def choose(results, slack: float = ENERGY_SLACK):
    """results: list of dicts with G, K, seconds, energy.  The fastest entry
    whose energy is within `slack` (relative) of the lowest energy."""
    if not results:
        raise ValueError("no results")
    e_best = min(r["energy"] for r in results)
    ok = [r for r in results if r["energy"] <= e_best + slack * abs(e_best)]
    return min(ok, key=lambda r: (r["seconds"], -r["G"], -r["K"]))


def _cache_path():
    return os.environ.get("CM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cm_autotune.json"))


def _load_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(H: int, W: int, kind: int, alpha: float, tol: float = 1e-4, ncolors: int = 4,
         candidates=CANDIDATES, ctx=None, use_cache: bool = True, repeats: int = 2):
    """Returns (options, record).  record holds every candidate's time, cycles
    and final energy, and the choice."""
    import torch
    import synth
    import paper_2204_07921_gb300 as cm
    gpu = torch.cuda.get_device_name()
    key = f"{gpu}|{H}x{W}|kind={kind}|alpha={alpha:g}|tol={tol:g}|ncolors={ncolors}"
    path = _cache_path()
    cache = _load_cache(path) if use_cache else {}
    if key in cache:
        rec = cache[key]
        return cm.default_options(ncolors=ncolors, grid_points=rec["G"], golden_evals=rec["K"]), rec
    img = synth.piecewise_image(H, W, synth.BASE_SEED + 900000 + 7 * H + W, 20, 0.08)
    f = torch.from_numpy(img.f).cuda()
    u = torch.empty_like(f)
    results = []
    for G, K in candidates:
        o = cm.default_options(ncolors=ncolors, grid_points=G, golden_evals=K)
        cm.cm_solve(f, alpha, kind, cycles=5000, tol=tol, u_out=u, options=o, ctx=ctx)
        best = None
        for _ in range(repeats):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = cm.cm_solve(f, alpha, kind, cycles=5000, tol=tol, u_out=u, options=o, ctx=ctx)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        results.append({"G": G, "K": K, "seconds": best, "cycles": st.cycles_run,
                        "energy": st.energy_final})
    pick = choose(results)
    rec = {"G": pick["G"], "K": pick["K"], "results": results, "image": f"{H}x{W}",
           "calibration_seed": synth.BASE_SEED + 900000 + 7 * H + W}
    if use_cache:
        cache = _load_cache(path)
        cache[key] = rec
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return cm.default_options(ncolors=ncolors, grid_points=pick["G"], golden_evals=pick["K"]), rec
