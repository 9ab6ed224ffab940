"""Autotuner of the solve's schedule.

It tunes, in stages, on a calibration image of the requested shape class (a
seeded image that is not one of the measured workloads):

1. the block-search budget -- G grid points on the bracket and K golden-
   section evaluations, a parameter of the method (the oracle takes the same
   two numbers): it trades the cost of a cycle against how far each block's
   subproblem is minimised, and on this non-convex energy a very precise
   search can also settle in worse local minima than a coarser one;
2. the colour schedule -- four colours, the checkerboard, or the decoupled
   colouring (more colours on the finest levels, no shared stencils);
3. the colour count of the coarse levels (block side >= 64): the fine
   levels' rule, two colours (same-colour blocks then share only corner
   pixels of their rings) or one (every block from the same state, a
   block-Jacobi step) -- fewer sequential phases on the latency-bound coarse
   levels;
4. the coarse levels' kernel shape -- how many candidates share one cluster
   reduction (first-pair speculation, golden steps per round), which changes
   the number of barriers and not the decisions;
5. the kernel shapes of the levels b = 2 .. 32 (cm_options.shapes: threads
   per block and ring pixels per thread), one level at a time: the level's
   alternative shape is kept only if the solve is faster by more than
   `SHAPE_MARGIN` at an energy within the slack (the shapes differ only in
   the FP32 order of the ring sums, so their energies agree to rounding).

Each stage times a solve to tolerance for every candidate and keeps the
fastest whose final energy is within `ENERGY_SLACK` of the lowest final
energy any candidate of the stage reached.  Results are cached per GPU model
in a JSON file ($CM_AUTOTUNE_CACHE, else ~/.cache/cm_autotune.json).
"""
from __future__ import annotations

import json
import os

CANDIDATES = ((9, 16), (7, 10), (5, 8), (5, 6), (5, 4), (3, 4))
COLOURS = (4, 2, 0)
COARSE_COLOURS = (0, 2, 1)
COARSE = ((-1, 0), (0, 4), (1, 4), (0, 2), (0, 1))   # (coarse_spec, coarse_dmax)
ENERGY_SLACK = 2e-3
SHAPE_MARGIN = 0.01
SHAPE_LEVELS = 5          # cm_options.shapes: bits for b = 2, 4, 8, 16, 32
CACHE_VERSION = 4


def choose(results, slack: float = ENERGY_SLACK):
    """results: list of dicts with G, K, seconds, energy.  The fastest entry
    whose energy is within `slack` (relative) of the lowest energy."""
    if not results:
        raise ValueError("no results")
    e_best = min(r["energy"] for r in results)
    ok = [r for r in results if r["energy"] <= e_best + slack * abs(e_best)]
    return min(ok, key=lambda r: (r["seconds"], -r.get("G", 0), -r.get("K", 0)))


def choose_shape(base, alt, slack: float = ENERGY_SLACK, margin: float = SHAPE_MARGIN):
    """base, alt: results of the solve with a level's default and alternative
    kernel shape.  The alternative wins only if it is faster by more than
    `margin` (relative) and its energy is within `slack` of base's."""
    if alt["energy"] > base["energy"] + slack * abs(base["energy"]):
        return base
    return alt if alt["seconds"] < (1.0 - margin) * base["seconds"] else base


def shape_bits(levels: int):
    """Bits of cm_options.shapes that concern a solve with `levels` levels
    (block sides 1 .. 2^(levels - 1)): bit lb - 1 for b = 2^lb, lb = 1 .. 5."""
    return [lb - 1 for lb in range(1, min(SHAPE_LEVELS, levels - 1) + 1)]


def _cache_path():
    return os.environ.get("CM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cm_autotune.json"))


def _load_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def tune(H: int, W: int, kind: int, alpha: float, tol: float = 1e-4, ncolors=None,
         candidates=CANDIDATES, ctx=None, use_cache: bool = True, repeats: int = 2):
    """Returns (options, record).  record holds every stage's candidates
    (time, cycles, final energy) and the choices.  ncolors fixes the colour
    schedule instead of tuning it."""
    import torch
    import synth
    import paper_2204_07921_gb300 as cm
    gpu = torch.cuda.get_device_name()
    key = (f"v{CACHE_VERSION}|{gpu}|{H}x{W}|kind={kind}|alpha={alpha:g}|tol={tol:g}"
           f"|ncolors={'tuned' if ncolors is None else ncolors}")
    path = _cache_path()
    cache = _load_cache(path) if use_cache else {}

    def options(rec):
        return cm.default_options(ncolors=rec["ncolors"], grid_points=rec["G"],
                                  golden_evals=rec["K"], coarse_spec=rec["coarse_spec"],
                                  coarse_dmax=rec["coarse_dmax"],
                                  coarse_ncolors=rec.get("coarse_ncolors", 0),
                                  shapes=rec.get("shapes", 0))

    if key in cache:
        return options(cache[key]), cache[key]
    seed = synth.BASE_SEED + 900000 + 7 * H + W
    img = synth.piecewise_image(H, W, seed, 20, 0.08)
    f = torch.from_numpy(img.f).cuda()
    u = torch.empty_like(f)

    def run(cfg):
        o = options(cfg)
        cm.cm_solve(f, alpha, kind, cycles=5000, tol=tol, u_out=u, options=o, ctx=ctx)
        best = None
        for _ in range(repeats):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = cm.cm_solve(f, alpha, kind, cycles=5000, tol=tol, u_out=u, options=o,
                                ctx=ctx)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return {**cfg, "seconds": best, "cycles": st.cycles_run, "energy": st.energy_final}

    cfg = {"G": 5, "K": 6, "ncolors": 4 if ncolors is None else ncolors, "coarse_spec": -1,
           "coarse_dmax": 0, "coarse_ncolors": 0, "shapes": 0}
    stages = {}
    stages["budget"] = [run({**cfg, "G": G, "K": K}) for G, K in candidates]
    pick = choose(stages["budget"])
    cfg.update(G=pick["G"], K=pick["K"])
    if ncolors is None:
        stages["colours"] = [run({**cfg, "ncolors": nc}) for nc in COLOURS]
        cfg["ncolors"] = choose(stages["colours"])["ncolors"]
    stages["coarse_colours"] = [run({**cfg, "coarse_ncolors": cn}) for cn in COARSE_COLOURS]
    cfg["coarse_ncolors"] = choose(stages["coarse_colours"])["coarse_ncolors"]
    stages["coarse"] = [run({**cfg, "coarse_spec": sp, "coarse_dmax": dm}) for sp, dm in COARSE]
    pick = choose(stages["coarse"])
    cfg.update(coarse_spec=pick["coarse_spec"], coarse_dmax=pick["coarse_dmax"])
    base = run(cfg)
    stages["shapes"] = [base]
    for bit in shape_bits(cm.cm_auto_levels(H, W)):
        alt = run({**cfg, "shapes": cfg["shapes"] ^ (1 << bit)})
        stages["shapes"].append(alt)
        base = choose_shape(base, alt)
        cfg["shapes"] = base["shapes"]
    rec = {**cfg, "stages": stages, "image": f"{H}x{W}", "calibration_seed": seed}
    if use_cache:
        cache = _load_cache(path)
        cache[key] = rec
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return options(rec), rec
