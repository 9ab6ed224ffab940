"""Benchmark: seconds to relative-energy tolerance 1e-4 on a 1024x1024 image.

One step = the learned warm start (CNN inference and its energy check) and
one full solve of the hot path from its output (Alg. 3 half V-cycles of the
coloured block sweep, every level and colour, with the FP64 energy and
stopping test after each cycle) on the seeded 1024^2 mean-curvature image
(20 shapes, sigma 0.08, alpha 20, levels 1..512), inputs already resident
in HBM.  The plain sweep from f is timed the same way and reported next to
it, with the 16-image warm-start evaluation and the 64-image batched solve.
Prints one JSON line (see --help).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SIDE = 1024
ALPHA = 20.0
KIND = 0
TOL = 1e-4
NCOLORS = 4
COARSE_LB = 6          # levels with block side >= 64 run the coarse path
MAX_CYCLES = 2000
METRIC = ("s to rel-energy tol 1e-4 at 1024^2 (learned warm start + FP32 sweep with FP64 "
          "stopping test; plain sweep reported alongside)")
WARMSTART_PARAMS = os.path.join(ROOT, "paper_2204_07921_gb300", "data", "warmstart_mean_a20.npz")
WARMSTART_PARAMS_GAUSS = os.path.join(ROOT, "paper_2204_07921_gb300", "data", "warmstart_gauss_a15.npz")
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
B1_TRAFFIC_BYTES = 7.41e6     # ncu DRAM bytes of one finest-level phase at 1024^2 (mean of 4)
F_KAPPA = 130.0               # FP32 operations per ring-pixel curvature evaluation


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--side", type=int, default=SIDE)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-warmstart-eval", action="store_true",
                   help="skip the 16-image warm-start evaluation")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the 64-image batched measurement")
    p.add_argument("--no-recon", action="store_true",
                   help="skip the reconstruction (Sec. 5) measurement")
    p.add_argument("--recon-only", action="store_true",
                   help="only run 2 reconstruction cycles at --side (for profiling)")
    p.add_argument("--ct-only", action="store_true",
                   help="only run 2 CT reconstruction cycles at --side, 180 angles (profiling)")
    p.add_argument("--cnn-only", action="store_true",
                   help="profiling aid: warm-start inference on --cnn-images 1024^2 images "
                        "(two passes) and exit")
    p.add_argument("--cnn-images", type=int, default=16,
                   help="images of the --cnn-only inference (default 16)")
    p.add_argument("--phases-only", action="store_true",
                   help="profiling aid: two warm-up cycles, then one launch of every "
                        "(level, colour) phase on the image and exit")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 20 ms with
    timestamps; summary() keeps the samples taken inside the marked window
    (mark_start / mark_end around the timed region)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            t_end = time.time() + 5.0          # wait for the first sample
            while time.time() < t_end and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), float(parts[4]), parts[6:10]))
            except ValueError:
                continue
        os.unlink(self.path)
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if self.t0 - 0.02 <= r[0] <= self.t1 + 0.02]
        else:
            inside = rows
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in the window"],
                    "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[4]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "reasons": reasons,
                "samples": len(inside), "window_s": round(self.t1 - self.t0, 3)
                if self.t0 is not None and self.t1 is not None else None,
                "power_w_median": statistics.median(r[3] for r in inside)}


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# oracle (CPU) timing: shared by the cpu_baseline field and --impl reference


# The schedule the autotuner picks for the 1024^2 workload on the GB300
# (search budget (5, 6), four colours, one on the coarse levels b >= 64): the
# CPU legs run the oracle with it, since they have no GPU to tune on.
REF_SCHEDULE = {"G": 5, "K": 6, "ncolors": 4, "coarse_ncolors": 1}


def oracle_cycle_seconds(u0, f64, n_cycles: int, sched=None):
    """Wall seconds per cycle of the FP64 oracle from state u0 (as it stands,
    OpenMP over the blocks of a colour on the host cores it is given)."""
    import oracle
    sc = sched or REF_SCHEDULE
    u = u0.copy()
    t0 = time.perf_counter()
    for _ in range(n_cycles):
        u = oracle.cycle(u, f64, ALPHA, KIND, ncolors=sc["ncolors"], G=sc["G"], K=sc["K"],
                         coarse_ncolors=sc["coarse_ncolors"])
        oracle.energy(u, f64, ALPHA, KIND)
    return (time.perf_counter() - t0) / n_cycles, oracle.num_threads()


def oracle_warmstart(f64):
    """The learned warm start in FP64 on the host: the network's forward pass
    (oracle/cnn.py, the shipped weights) and the energy check that keeps u0
    only if F(u0) <= F(f).  Returns (u0, seconds, kept)."""
    import numpy as np
    import oracle
    from oracle import cnn as ocnn
    params = np.load(WARMSTART_PARAMS)["params"].astype(np.float64)
    t0 = time.perf_counter()
    u0, _ = ocnn.forward(params, f64[None])
    u0 = u0[0]
    kept = oracle.energy(u0, f64, ALPHA, KIND) <= oracle.energy(f64, f64, ALPHA, KIND)
    if not kept:
        u0 = f64
    return u0, time.perf_counter() - t0, bool(kept)


def run_reference(args):
    """The reference arm is the FP64 oracle, run as it stands on the host
    cores, on the same workload as the GPU line: the learned warm start (the
    network's forward pass in FP64 and the energy check), then the sweep from
    its output with the same schedule to tol 1e-4 (one full solve: its own
    cycle count), then warm-up and timed single-cycle samples.  value = warm
    start time + mean cycle time x the oracle's cycle count."""
    rank, world, _ = dist_setup(args)
    if rank != 0:
        return
    import numpy as np
    import oracle
    import synth
    img = synth.large(args.side)
    f64 = img.f.astype(np.float64)
    u0, t_ws, kept = oracle_warmstart(f64)
    sc = REF_SCHEDULE
    t0 = time.perf_counter()
    u, trace, cycles, conv = oracle.solve(f64, ALPHA, KIND, cycles=MAX_CYCLES, tol=TOL, u0=u0,
                                          ncolors=sc["ncolors"], G=sc["G"], K=sc["K"],
                                          coarse_ncolors=sc["coarse_ncolors"])
    full_s = time.perf_counter() - t0
    times = []
    threads = 1
    for i in range(args.warmup + args.steps):
        per_cycle, threads = oracle_cycle_seconds(u0, f64, 1)
        if i >= args.warmup:
            times.append(per_cycle)
    per_cycle = statistics.mean(times)
    value = t_ws + per_cycle * cycles
    sample = (f"oracle: warm start {t_ws:.1f} s, one full solve from it to tol ({cycles} "
              f"cycles, {full_s:.1f} s), then {args.steps} timed single-cycle samples; "
              f"value = warm start + mean cycle x {cycles}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.side, L=_auto_levels(args.side), sched=sc),
            "oracle_cycles": cycles, "oracle_converged": bool(conv),
            "oracle_full_solve_s": full_s, "oracle_warmstart_s": t_ws,
            "oracle_warmstart_kept": kept, "oracle_final_energy": float(trace[-1]),
            "psnr_db": synth.psnr(u.astype(np.float32), img.clean),
            "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
                             "sample": sample, "per_cycle_s": per_cycle},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _auto_levels(side):
    """Levels of the sides 1, 2, 4, .. up to the largest <= side / 2."""
    L, b = 0, 1
    while 2 * b <= side:
        L += 1
        b *= 2
    return L


def workload_config(side, L, sched):
    """The workload both arms run (same keys and values when the autotuner
    picks the schedule the CPU legs use)."""
    return {"workload": f"denoise {side}^2 mean curv., learned warm start + sweep to tol 1e-4",
            "image": f"{side}x{side}", "shapes": 20, "sigma": 0.08, "kind": "mean",
            "alpha": ALPHA, "tol": TOL, "levels": L, "block_sides": f"1..{1 << (L - 1)}",
            "grid_points": sched["G"], "golden_evals": sched["K"], "ncolors": sched["ncolors"],
            "coarse_ncolors": sched["coarse_ncolors"],
            "warm_start": "6 conv3x3, 32 ch, residual (shipped weights), energy check",
            "l2": "flushed between steps (512 MB write)"}


def cpu_legs(img, cycles_warm, opts, cm, torch, ctx, dev):
    """The oracle on the host cores (as it stands):
    * value: the same workload as the GPU line -- the FP64 warm start, then
      two timed oracle cycles from its output, extrapolated to the GPU's
      cycle count (a bounded sample);
    * single_thread: one oracle cycle with one thread on the 512 x 512
      top-left corner of the image, x 4 for the full image (a sample);
    * parity_vs_gpu: the plain solve from f with the oracle's own schedule
      (four colours on every level, (G, K) = (5, 6)) by the oracle and by the
      GPU: final energies, their relative difference and max |u_gpu - u_orc|
      (both FP32-vs-FP64 trajectories; energy ties separate them)."""
    import numpy as np
    import oracle
    f64 = img.f.astype(np.float64)
    u0, t_ws, kept = oracle_warmstart(f64)
    n_s = 2
    per_cycle, threads = oracle_cycle_seconds(u0, f64, n_s)
    mean_cycles = statistics.mean(cycles_warm)
    res = {"value": t_ws + per_cycle * mean_cycles, "unit": "s", "cores": threads,
           "kind": "oracle",
           "sample": f"FP64 warm start ({t_ws:.1f} s) + {n_s} oracle cycles from it on the "
                     f"{img.f.shape[0]}^2 image, extrapolated x {mean_cycles:g} cycles (the "
                     f"GPU's count)", "per_cycle_s": per_cycle, "warmstart_s": t_ws}
    crop = f64[:512, :512].copy()
    try:
        oracle.set_num_threads(1)
        pc1, _ = oracle_cycle_seconds(crop, crop, 1)
    finally:
        oracle.set_num_threads(threads)
    scale = f64.size / crop.size
    res["single_thread"] = {"value": t_ws + pc1 * scale * mean_cycles, "per_cycle_s": pc1 * scale,
                            "cores": 1, "sample": "one cycle, 1 thread, 512^2 corner x 4 "
                                                  "(the warm start as timed above)"}
    t0 = time.perf_counter()
    uo, trace, n_o, conv = oracle.solve(f64, ALPHA, KIND, cycles=MAX_CYCLES, tol=TOL,
                                        ncolors=4, G=5, K=6)
    t_full = time.perf_counter() - t0
    o4 = cm.default_options(ncolors=4, grid_points=5, golden_evals=6)
    fd = torch.from_numpy(img.f).to(dev)
    ug, st = cm.cm_solve(fd, ALPHA, KIND, cycles=MAX_CYCLES, tol=TOL, options=o4, ctx=ctx)
    ugh = ug.cpu().numpy()
    Eg = oracle.energy(ugh.astype(np.float64), f64, ALPHA, KIND)
    res["parity_vs_gpu"] = {
        "schedule": "plain from f, 4 colours on every level, (G, K) = (5, 6), tol 1e-4",
        "oracle_cycles": n_o, "gpu_cycles": st.cycles_run, "oracle_s": t_full,
        "oracle_final_energy": float(trace[-1]), "gpu_final_energy": Eg,
        "gpu_reported_energy": st.energy_final,
        "rel_energy_diff": (Eg - float(trace[-1])) / float(trace[-1]),
        "max_abs_du": float(np.abs(ugh - uo).max()),
        "mean_abs_du": float(np.abs(ugh - uo).mean())}
    return res


def batched_measurement(cm, torch, synth, ctx, dev, rank=0, world=1):
    """64 images of uneven sizes (sides from {128, ..., 1024}, half mean and
    half Gaussian curvature, sigma ~ U(0.03, 0.12), alpha in {10, 20}) solved
    to tol 1e-4: one batched call vs one cm_solve call per image.  Metric:
    aggregate Mpixel-sweeps/s = sum(H W cycles) / time.  With several ranks
    the images are sharded by the LPT rule (no collective on the data path);
    the job time is the maximum over ranks."""
    from paper_2204_07921_gb300 import shard
    all_items = synth.uneven_batch(64)
    costs = [shard.image_cost(*it.image.f.shape) for it in all_items]
    items = [all_items[i] for i in shard.my_share(costs, rank, world)]
    fs = [torch.from_numpy(it.image.f).to(dev) for it in items]
    outs = [torch.empty_like(t) for t in fs]
    al = [it.alpha for it in items]
    kd = [it.kind for it in items]
    # one schedule for the whole batch, tuned on a median-sized Gaussian-curvature
    # calibration image (the batch mixes the kinds, so the colours stay at four)
    from paper_2204_07921_gb300 import autotune
    opts, brec = autotune.tune(576, 576, 1, 15.0, tol=TOL, ncolors=4, ctx=ctx)

    def batched():
        _, st = cm.cm_solve_batched(fs, al, kd, tol=TOL, cycles=MAX_CYCLES, u_outs=outs,
                                    options=opts, ctx=ctx)
        return st

    def sequential():
        sts = []
        for i in range(len(fs)):
            _, st = cm.cm_solve(fs[i], al[i], kd[i], cycles=MAX_CYCLES, tol=TOL, u_out=outs[i],
                                options=opts, ctx=ctx)
            sts.append(st)
        return sts

    res = {"schedule": {k: brec[k] for k in ("G", "K", "ncolors", "coarse_ncolors", "coarse_spec",
                                             "coarse_dmax", "shapes")}}
    for name, fn in (("batched", batched), ("one_at_a_time", sequential)):
        fn()   # warm-up (graph capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sts = fn()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        mpx = sum(it.image.f.size * st.cycles_run for it, st in zip(items, sts)) / 1e6
        cyc = float(sum(st.cycles_run for st in sts))
        if world > 1:
            import torch.distributed as dist
            v = torch.tensor([t, mpx, cyc], dtype=torch.float64, device=dev)
            tmax = v[:1].clone()
            dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
            dist.all_reduce(v, op=dist.ReduceOp.SUM)
            t, mpx, cyc = float(tmax.item()), float(v[1].item()), float(v[2].item())
        res[name] = {"s": t, "mpixel_sweeps_per_s": mpx / t, "cycles_total": int(cyc)}
    res["speedup"] = res["batched"]["mpixel_sweeps_per_s"] / res["one_at_a_time"]["mpixel_sweeps_per_s"]
    res["workload"] = "64 images, sides U{128..1024} x U{128..1024}, half mean / half Gaussian, tol 1e-4"
    res["pixels"] = int(sum(it.image.f.size for it in all_items))
    res["ranks"] = world
    return res


def measured_hbm_peak():
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json), else the
    fallback figure of one earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def hbm_measurement(cm, torch, synth, ctx, dev, stream, opts, flush, b1_ms, N, nc):
    """GB/s of algorithmic bytes for the finest-level phase and the energy
    kernel (CUDA events on the launching stream), against the HBM peak."""
    peak, src = measured_hbm_peak()
    out = {"peak_gbs": peak, "peak_source": src}
    b1_bytes = 12.0 / nc * N
    out["phase_b1_1024"] = {"bytes_per_launch": b1_bytes, "ms": b1_ms,
                            "gbs": b1_bytes / (b1_ms / 1e3) / 1e9,
                            "frac": b1_bytes / (b1_ms / 1e3) / 1e9 / peak,
                            "note": "working set in L2 (1024^2)"}
    side = 4096
    im = synth.large(side)
    u4 = torch.from_numpy(im.f).to(dev)
    f4 = torch.from_numpy(im.clean).to(dev)
    R4 = u4.clone()
    E_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    n4 = side * side
    reps = 6

    def timed(fn):
        fn(0)
        torch.cuda.synchronize()
        tot = 0.0
        for i in range(reps):
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(i)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    ms = timed(lambda i: cm.cm_phase(u4, R4, f4, ALPHA, KIND, 1, i % nc, options=opts, ctx=ctx))
    by = 12.0 / nc * n4
    out["phase_b1_4096"] = {"bytes_per_launch": by, "ms": ms, "gbs": by / (ms / 1e3) / 1e9,
                            "frac": by / (ms / 1e3) / 1e9 / peak, "note": "L2 flushed"}
    ms = timed(lambda i: cm.cm_energy_noalloc(u4, f4, ALPHA, KIND, E_dev))
    by = 8.0 * n4
    out["energy_4096"] = {"bytes_per_launch": by, "ms": ms, "gbs": by / (ms / 1e3) / 1e9,
                          "frac": by / (ms / 1e3) / 1e9 / peak, "note": "L2 flushed"}
    del u4, f4, R4
    return out


# HBM bytes per pixel of one pass of the warm-start network: the first layer
# reads f (4 B) and writes 32 BF16 channels (64 B); each of the four 32 -> 32
# layers reads and writes 64 B; the output layer reads 64 B and f (4 B) and
# writes u0 (4 B).
CNN_BYTES_PER_PIXEL = 4 + 64 + 4 * 128 + 64 + 4 + 4


def cnn_measurement(torch, synth, net, dev, stream, n=16, side=1024, reps=10):
    """Inference of the warm-start network on n test images of side^2 (every
    activation far above the L2), timed with CUDA events on the launching
    stream after warm-up: algorithmic HBM bytes / device time against the
    HBM peak."""
    peak, src = measured_hbm_peak()
    F = torch.stack([torch.from_numpy(synth.warmstart_image("test", i, side).f)
                     for i in range(n)]).to(dev).contiguous()
    out = torch.empty_like(F)
    for _ in range(3):
        net.forward(F, out=out, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        net.forward(F, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    by = float(CNN_BYTES_PER_PIXEL) * n * side * side
    del F, out
    return {"images": n, "side": side, "ms": ms, "bytes_per_pass": by,
            "gbs": by / (ms / 1e3) / 1e9, "peak_gbs": peak, "peak_source": src,
            "frac": by / (ms / 1e3) / 1e9 / peak,
            "note": "whole forward (first layer on CUDA cores, four 32 -> 32 layers and the "
                    "output layer on tcgen05); per-layer counters: "
                    "profiles/cnn_forward_kernels_1024.md"}


def kernels_per_cycle(opts, L):
    """Kernels of one solve cycle over levels b = 1, 2, .. 2^(L-1): one per
    colour on the levels below the coarse threshold (b < 64); one per colour
    and the apply on the coarse levels, plus the tile sums before the first;
    the energy; the device stopping test."""
    return 2 + sum(level_colours(opts, 1 << j) +
                   (0 if j < COARSE_LB else (2 if j == COARSE_LB else 1))
                   for j in range(L))


def level_colours(opts, b):
    """Colours of the level of block side b under the options (the library's
    rule: coarse_ncolors on b >= 64 when set, the decoupled count for
    ncolors = 0)."""
    if opts.coarse_ncolors != 0 and b >= 64:
        return opts.coarse_ncolors
    if opts.ncolors != 0:
        return opts.ncolors
    p = 2
    while (p - 1) * b < 3:
        p += 1
    return p * p


def recon_measurement(cm, torch, synth, ctx, dev, stream, with_oracle=True):
    """Reconstruction extension (Sec. 5, A = M F): MRI-like cases (phantom of
    12 shapes, Cartesian rows at 1/3 sampling with the central 8% kept,
    complex noise sigma 0.01), alpha 0.02, mean curvature, every level, four
    colours, 8 CG iterations per colour.  Device time per cycle (CUDA events,
    the captured cycle already built), PSNR of the zero-filled start and
    after 5 cycles; the FP64 oracle's time for one cycle at 512^2 beside it."""
    import time
    import numpy as np
    res = {"alpha": 0.02, "kind": "mean", "cg_iters": 8, "accel": 3.0, "sigma": 0.01}
    for side in (512, 1024):
        case = synth.mri_case(side, side, synth.workload_seed(6, side), accel=3.0, sigma=0.01)
        kd = torch.from_numpy(case.kspace).to(dev)
        md = torch.from_numpy(case.mask).to(dev)
        u0, tr0 = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=0, ctx=ctx)
        psnr0 = synth.psnr(u0.cpu().numpy(), case.clean)
        cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=1, ctx=ctx)      # builds the cycle graph
        torch.cuda.synchronize()
        n = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, tr = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=n, ctx=ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"{side}x{side}"] = {
            "s_per_cycle": e0.elapsed_time(e1) / 1e3 / n, "cycles": n,
            "psnr_zero_filled_db": psnr0, "psnr_db": synth.psnr(u.cpu().numpy(), case.clean),
            "objective_trace": [float(x) for x in tr], "sampled_fraction": float(case.mask.mean())}
    # CT (A = R): the phantom's sinogram from the library's own Radon
    # transform plus seeded noise, 180 angles, the filtered backprojection as
    # the start, alpha 1
    side, n_ang = 256, 180
    clean = synth.piecewise_image(side, side, synth.workload_seed(6, 7 * side), 12, 0.0).clean
    cd = torch.from_numpy(clean).to(dev)
    sino = cm.cm_radon(cd, n_ang, ctx=ctx)
    rng = np.random.default_rng(side)
    sino += torch.from_numpy((0.1 * rng.normal(size=tuple(sino.shape))).astype(np.float32)).to(dev)
    u0, _ = cm.cm_recon_ct(sino, side, side, 1.0, cm.MEAN, cycles=0, ctx=ctx)
    psnr0 = synth.psnr(u0.cpu().numpy(), clean)
    cm.cm_recon_ct(sino, side, side, 1.0, cm.MEAN, cycles=1, ctx=ctx)   # builds the graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    u, tr = cm.cm_recon_ct(sino, side, side, 1.0, cm.MEAN, cycles=3, ctx=ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    res["ct_256x256"] = {"angles": n_ang, "bins": int(sino.shape[1]), "alpha": 1.0,
                         "noise_sigma": 0.1, "s_per_cycle": e0.elapsed_time(e1) / 1e3 / 3,
                         "cycles": 3, "psnr_fbp_db": psnr0,
                         "psnr_db": synth.psnr(u.cpu().numpy(), clean),
                         "objective_trace": [float(x) for x in tr]}
    if with_oracle:
        import oracle
        from oracle import recon as orc
        case = synth.mri_case(512, 512, synth.workload_seed(6, 512), accel=3.0, sigma=0.01)
        t = time.perf_counter()
        orc.solve(case.kspace, case.mask, 0.02, cm.MEAN, cycles=1, cg_iters=8)
        res["cpu_baseline"] = {"value": time.perf_counter() - t, "unit": "s per cycle",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": "one cycle of the 512^2 case (FP64, numpy FFT)"}
        # CT oracle: one cycle of a 48^2 case with 45 angles (the 256^2 case
        # would take tens of minutes in numpy); the GPU on the same case
        cl48 = synth.piecewise_image(48, 48, 21, 6, 0.0).clean.astype(np.float64)
        s48 = orc.radon_forward(cl48, 45)
        t = time.perf_counter()
        orc.solve_ct(s48, 48, 48, 1.0, cm.MEAN, cycles=1, cg_iters=8)
        t_orc = time.perf_counter() - t
        s48d = torch.from_numpy(s48.astype(np.float32)).to(dev)
        cm.cm_recon_ct(s48d, 48, 48, 1.0, cm.MEAN, cycles=1, ctx=ctx)
        torch.cuda.synchronize()
        e0.record(stream)
        cm.cm_recon_ct(s48d, 48, 48, 1.0, cm.MEAN, cycles=3, ctx=ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        res["ct_48x48_cpu_baseline"] = {"value": t_orc, "unit": "s per cycle",
                                        "cores": oracle.num_threads(), "kind": "oracle",
                                        "sample": "one cycle, 48^2, 45 angles",
                                        "gpu_s_per_cycle": e0.elapsed_time(e1) / 1e3 / 3}
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2204_07921_gb300 as cm
    import synth

    rank, world, local = dist_setup(args)
    # the autotuner's cache: a file this script writes itself (in the build
    # folder of the package) unless the caller names one
    os.environ.setdefault("CM_AUTOTUNE_CACHE", os.path.join(
        ROOT, "paper_2204_07921_gb300", "_build", f"autotune_rank{rank}.json"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cm.load()
    ctx = cm.Context(local)
    if args.ct_only:
        clean = synth.piecewise_image(args.side, args.side, synth.workload_seed(6, 7 * args.side),
                                      12, 0.0).clean
        sino = cm.cm_radon(torch.from_numpy(clean).to(dev), 180, ctx=ctx)
        u, tr = cm.cm_recon_ct(sino, args.side, args.side, 1.0, cm.MEAN, cycles=2, ctx=ctx)
        torch.cuda.synchronize()
        print(json.dumps({"ct_only": True, "side": args.side, "trace": list(tr)}))
        return
    if args.recon_only:
        case = synth.mri_case(args.side, args.side, synth.workload_seed(6, args.side),
                              accel=3.0, sigma=0.01)
        kd = torch.from_numpy(case.kspace).to(dev)
        md = torch.from_numpy(case.mask).to(dev)
        u, tr = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=2, ctx=ctx)
        torch.cuda.synchronize()
        print(json.dumps({"recon_only": True, "side": args.side, "trace": list(tr)}))
        return
    img = synth.large(args.side)
    f_host = torch.from_numpy(img.f).pin_memory()
    f = f_host.to(dev)
    u = torch.empty_like(f)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    from paper_2204_07921_gb300 import autotune
    opts, tune_rec = autotune.tune(args.side, args.side, KIND, ALPHA, tol=TOL, ncolors=None,
                                   ctx=ctx)
    L = cm.cm_auto_levels(args.side, args.side)

    if args.cnn_only:
        from paper_2204_07921_gb300 import warmstart as ws
        net = ws.Net.load(WARMSTART_PARAMS, ctx=ctx)
        F = torch.stack([torch.from_numpy(synth.warmstart_image("test", i, 1024).f)
                         for i in range(args.cnn_images)]).to(dev).contiguous()
        net.forward(F)
        net.forward(F)
        torch.cuda.synchronize()
        print(json.dumps({"cnn_only": True, "images": args.cnn_images}))
        return

    if args.phases_only:
        _, st = cm.cm_solve(f, ALPHA, KIND, cycles=2, u_out=u, options=opts, ctx=ctx)
        R = u.clone()
        for j in range(L):
            for k in range(level_colours(opts, 1 << j)):
                cm.cm_phase(u, R, f, ALPHA, KIND, 1 << j, k, options=opts, ctx=ctx)
        # the coarse levels as the solve runs them (tile sums, rounds, apply)
        for j in range(COARSE_LB, L):
            cm.cm_level(u, R, f, ALPHA, KIND, 1 << j, options=opts, ctx=ctx)
        cm.cm_energy(u, f, ALPHA, KIND, ctx=ctx)
        # one cycle of the solve outside a graph (profilers do not look inside
        # the conditional loop of the graph): the solve's own kernel sequence
        oh = cm.Options.from_buffer_copy(opts)
        oh.use_graph = 0
        cm.cm_solve(f, ALPHA, KIND, cycles=1, u_out=u, options=oh, ctx=ctx)
        torch.cuda.synchronize()
        print(json.dumps({"phases_only": True, "levels": L, "ncolors": opts.ncolors}))
        return

    from paper_2204_07921_gb300 import warmstart as ws
    net = ws.Net.load(WARMSTART_PARAMS, ctx=ctx)
    U0 = torch.empty_like(f)

    def plain_step(fin, out):
        _, st = cm.cm_solve(fin, ALPHA, KIND, levels=0, cycles=MAX_CYCLES, tol=TOL, u_out=out,
                            options=opts, ctx=ctx)
        return st

    def warm_step(fin, out):
        # learned warm start (inference + the energy check) then the sweep from u0
        ws.warmstart(net, fin, ALPHA, KIND, check_energy=True, out=U0)
        _, st = cm.cm_solve(fin, ALPHA, KIND, levels=0, cycles=MAX_CYCLES, tol=TOL, u0=U0,
                            u_out=out, options=opts, ctx=ctx)
        return st

    for _ in range(args.warmup):
        warm_step(f, u)
        plain_step(f, u)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_steps(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        sts = []
        barrier()
        for i in range(args.steps):
            flush.fill_(float(i))       # L2 flush outside the timed events
            ev[i][0].record(stream)
            sts.append(fn(f, u))
            ev[i][1].record(stream)
        barrier()
        t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        if world > 1:
            tt = torch.tensor([t], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t / args.steps, sts

    with ClockSampler(local) as clk:
        clk.mark_start()
        sec_warm, st_warm = timed_steps(warm_step)
        clk.mark_end()
        psnr_warm = synth.psnr(u.cpu().numpy(), img.clean)
        sec_plain, st_plain = timed_steps(plain_step)
        psnr_plain = synth.psnr(u.cpu().numpy(), img.clean)
    clocks = clk.summary()
    cycles = [s.cycles_run for s in st_warm]
    cycles_plain = [s.cycles_run for s in st_plain]
    sec_per_solve = sec_warm
    final_E = st_warm[-1].energy_final

    # e2e: the warm-start solve through the C ABI with host buffers (pinned):
    # the H2D copy of f and the D2H copy of u inside the timed region.
    u_host = torch.empty_like(f_host).pin_memory()
    fd = torch.empty_like(f)     # persistent device input buffer of the e2e leg
    e2e_t = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fd.copy_(f_host, non_blocking=True)
        warm_step(fd, u)
        u_host.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e = statistics.mean(e2e_t)

    # the bench image at equal final energy (the warm-started sweep stops at the
    # plain solve's energy instead of at the tolerance)
    warm_eq_image = ws.evaluate_equal_energy(net, alpha=ALPHA, kind=KIND, tol=TOL, ctx=ctx,
                                             images=[img])

    # single-step mode (one step of Alg. 2 per block, kept if it lowers E_A):
    # the plain solve to the same tolerance, timed the same way
    opts1 = cm.Options.from_buffer_copy(opts)   # the tuned schedule, one step per block
    opts1.one_step = 1

    def one_step_solve(fin, out):
        _, st = cm.cm_solve(fin, ALPHA, KIND, levels=0, cycles=MAX_CYCLES, tol=TOL, u_out=out,
                            options=opts1, ctx=ctx)
        return st

    one_step_solve(f, u)
    torch.cuda.synchronize()
    sec_one, st_one = timed_steps(one_step_solve)
    one_step_res = {"s": sec_one, "cycles_to_tol": [s.cycles_run for s in st_one],
                    "psnr_db": synth.psnr(u.cpu().numpy(), img.clean),
                    "final_energy": st_one[-1].energy_final,
                    "converged": bool(st_one[-1].converged),
                    "vs_search_plain_time": sec_one / sec_plain}
    # the single-step relative-change test stops far above the search's energy:
    # also the cycles (and time) it needs to reach the searched solve's energy
    n_long = 400
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):   # the first call captures this solve's graph
        e0.record(stream)
        _, st_long = cm.cm_solve(f, ALPHA, KIND, levels=0, cycles=n_long, tol=0.0, u_out=u,
                                 options=opts1, ctx=ctx)
        e1.record(stream)
    torch.cuda.synchronize()
    per_cycle = e0.elapsed_time(e1) / 1e3 / n_long
    target = st_plain[-1].energy_final
    trace = st_long.trace()
    hit = next((i for i, E in enumerate(trace) if E <= target), None)
    one_step_res["to_search_energy"] = {
        "target_energy": target, "cycles_run": n_long, "per_cycle_s": per_cycle,
        "cycles_to_target": hit, "s_to_target": None if hit is None else hit * per_cycle,
        "energy_after_run": trace[-1], "psnr_after_run_db": synth.psnr(u.cpu().numpy(), img.clean)}

    # the colouring / cycle variants of the method (plain solve from f to the
    # same tolerance): the full V-cycle (Sec. 2.2, compared in Sec. 4.1) and
    # the decoupled colouring (blocks of one colour share no stencil)
    def to_energy(ov, lv, target, n=60):
        """Cycles (and time) a variant needs to reach the default schedule's
        final energy: n cycles at tol 0, the first cycle at or below target."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for rep in range(2):   # the first call captures this solve's graph
            e0.record(stream)
            _, st = cm.cm_solve(f, ALPHA, KIND, levels=lv, cycles=n, tol=0.0, u_out=u,
                                options=ov, ctx=ctx)
            e1.record(stream)
        torch.cuda.synchronize()
        per = e0.elapsed_time(e1) / 1e3 / n
        hit = next((i for i, E in enumerate(st.trace()) if E <= target), None)
        return {"cycles": hit, "s": None if hit is None else hit * per, "per_cycle_s": per,
                "energy_after": st.trace()[-1], "cycles_run": n}

    # and the paper's block sides 2^j - 1 (Sec. 2.2), with the default level
    # count (sides up to 511) and with the paper's J = 3 (sides 1, 3, 7)
    variants = {}
    for name, kw in (("vcycle", dict(vcycle=1)), ("decoupled", dict(ncolors=0)),
                     ("decoupled_vcycle", dict(ncolors=0, vcycle=1)),
                     ("paper_sides", dict(block_sides=1)),
                     ("paper_sides_J3", dict(block_sides=1, levels=3)),
                     ("J3", dict(levels=3))):
        # the tuned schedule with the variant's changes; the decoupled
        # colouring keeps its own colours on every level
        ov = cm.Options.from_buffer_copy(opts)
        ov.ncolors = kw.get("ncolors", opts.ncolors)
        ov.vcycle = kw.get("vcycle", 0)
        ov.block_sides = kw.get("block_sides", 0)
        if ov.ncolors == 0:
            ov.coarse_ncolors = 0

        def vsolve(fin, out, ov=ov, lv=kw.get("levels", 0)):
            _, st = cm.cm_solve(fin, ALPHA, KIND, levels=lv, cycles=MAX_CYCLES, tol=TOL,
                                u_out=out, options=ov, ctx=ctx)
            return st

        vsolve(f, u)
        torch.cuda.synchronize()
        sec_v, st_v = timed_steps(vsolve)
        variants[name] = {"s": sec_v, "cycles_to_tol": st_v[-1].cycles_run,
                          "levels": st_v[-1].levels,
                          "psnr_db": synth.psnr(u.cpu().numpy(), img.clean),
                          "final_energy": st_v[-1].energy_final,
                          "monotone_violations": st_v[-1].monotone_violations,
                          "vs_default_schedule_time": sec_v / sec_plain,
                          "to_default_energy": to_energy(ov, kw.get("levels", 0),
                                                         st_plain[-1].energy_final)}
    variants["default_schedule"] = {"s": sec_plain, "cycles_to_tol": cycles_plain[-1],
                                        "psnr_db": psnr_plain,
                                        "final_energy": st_plain[-1].energy_final,
                                        "monotone_violations": st_plain[-1].monotone_violations}

    # complexity (the paper's linear-complexity study, Sec. 4): the plain
    # solve from f to the same tolerance on the same generator's images of
    # 256^2 .. 4096^2 (all levels, the tuned schedule): cycles, time, and
    # device time per pixel and cycle
    complexity = {}
    for side in (256, 512, 1024, 2048, 4096):
        im = synth.large(side)
        fs = torch.from_numpy(im.f).to(dev)
        us = torch.empty_like(fs)
        cm.cm_solve(fs, ALPHA, KIND, levels=0, cycles=MAX_CYCLES, tol=TOL, u_out=us,
                    options=opts, ctx=ctx)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, sts = cm.cm_solve(fs, ALPHA, KIND, levels=0, cycles=MAX_CYCLES, tol=TOL, u_out=us,
                             options=opts, ctx=ctx)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        complexity[f"{side}x{side}"] = {
            "levels": sts.levels, "cycles_to_tol": sts.cycles_run, "s": sec,
            "ns_per_pixel_cycle": 1e9 * sec / (side * side * max(1, sts.cycles_run)),
            "psnr_db": synth.psnr(us.cpu().numpy(), im.clean)}
        del fs, us

    # curvature kinds (plain solve from f to the same tolerance, the same
    # schedule): H and K from the extreme direction curvatures (the paper's
    # kinds) and from the least-squares Euler fit; Gaussian kinds at alpha 15
    kinds_res = {}
    for name, kd, al in (("mean", cm.MEAN, ALPHA), ("gauss", cm.GAUSS, 15.0),
                         ("mean_euler", cm.MEAN_EULER, ALPHA),
                         ("gauss_euler", cm.GAUSS_EULER, 15.0)):
        def ksolve(fin, out, kd=kd, al=al):
            _, st = cm.cm_solve(fin, al, kd, levels=0, cycles=MAX_CYCLES, tol=TOL, u_out=out,
                                options=opts, ctx=ctx)
            return st

        ksolve(f, u)
        torch.cuda.synchronize()
        sec_k, st_k = timed_steps(ksolve)
        kinds_res[name] = {"kind": kd, "alpha": al, "s": sec_k,
                           "cycles_to_tol": st_k[-1].cycles_run,
                           "psnr_db": synth.psnr(u.cpu().numpy(), img.clean),
                           "final_energy": st_k[-1].energy_final,
                           "monotone_violations": st_k[-1].monotone_violations}

    # dominant kernel: finest-level phase (b = 1), launched on the same stream
    state = u.clone()
    R = state.clone()
    n_launch = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nc = level_colours(opts, 1)   # colours of the finest level
    for k in range(nc):
        cm.cm_phase(state, R, f, ALPHA, KIND, 1, k, options=opts, ctx=ctx)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(n_launch):
        cm.cm_phase(state, R, f, ALPHA, KIND, 1, i % nc, options=opts, ctx=ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    b1_ms = e0.elapsed_time(e1) / n_launch
    N = args.side * args.side
    n_active = N // nc
    evals_per_block = 3 + (opts.grid_points - 1) + opts.golden_evals   # 0, paper, c_fid, grid, golden
    curv_evals = n_active * evals_per_block * 9
    evals_per_s = curv_evals / (b1_ms / 1e3)
    # Algorithmic FP32 work: F_KAPPA operations per ring-pixel curvature
    # evaluation (the per-unit figure of the hot-path scope: 8 plane distances,
    # 4 direction curvatures, their extremes, |kappa|) x the evaluations of the
    # launch; the peak is this GPU's measured FP32 rate (cm_probe_alu: FFMA/s
    # x 2 operations).  The kernel is issue-bound on the FP32 and ALU pipes
    # (ncu: 64% issue-active), not on the MUFU pipe.
    alu = cm.cm_probe_alu(local)
    fp32_peak = 2.0 * alu["fma_per_s"] / 1e12
    achieved = evals_per_s * F_KAPPA / 1e12
    mufu_peak = alu["rsqrt_per_s"] / 8 / 1e9
    roofline = {"bound": "alu", "kernel": "phase_b1_kernel (b=1)", "achieved": achieved,
                "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                "peak_source": "measured (cm_probe_alu: FFMA rate x 2)",
                "flop_per_eval": F_KAPPA, "evals_per_launch": curv_evals,
                "launch_ms": b1_ms,
                "issue_active": {"value": 0.64, "source": "profiles/phase_b1_kernel_1024.md"},
                "rsqrt_view": {"achieved_geval_s": evals_per_s / 1e9, "peak_geval_s": mufu_peak,
                               "frac": evals_per_s / 1e9 / mufu_peak,
                               "note": "peak = measured rsqrtf rate / 8 rsqrt per generic "
                                       "evaluation"},
                "measured_rsqrt_per_s": alu["rsqrt_per_s"],
                "measured_fma_per_s": alu["fma_per_s"],
                # dram__bytes_read.sum + dram__bytes_write.sum of one launch of this
                # kernel at 1024^2: the mean of four launches of one ncu capture
                "traffic": B1_TRAFFIC_BYTES if args.side == 1024 else None,
                "traffic_unit": "B per launch"}

    # HBM side of the roofline: algorithmic bytes per launch / device time.
    # The sweep's algorithmic bytes are 12 B per pixel and level (read u and
    # f, write u), so one phase of nc colours moves 12 / nc B per image pixel;
    # the energy reads u and f (8 B per pixel).  At 1024^2 the working set
    # stays in the 129 MB L2; at 4096^2 (134 MB of u and f) the L2 is flushed
    # (512 MB write) before every timed launch, so the bytes come from HBM.
    roofline["hbm"] = hbm_measurement(cm, torch, synth, ctx, dev, stream, opts, flush,
                                      b1_ms, N, nc)
    roofline["cnn_forward"] = cnn_measurement(torch, synth, net, dev, stream)
    roofline["solve"] = {"warm_s": sec_warm, "warm_cycles": cycles, "plain_s": sec_plain,
                         "plain_cycles": cycles_plain, "warm_vs_plain": sec_plain / sec_warm,
                         "psnr_warm_db": psnr_warm, "psnr_plain_db": psnr_plain}

    warm_eval = warm_eval_gauss = None
    if not args.no_warmstart_eval:
        warm_eval = ws.evaluate(net, n=16, side=1024, alpha=ALPHA, kind=KIND, tol=TOL, ctx=ctx)
        # at equal final energy: the warm-started sweep runs the cycles it needs to
        # reach the plain solve's energy (single images, inference included)
        warm_eval["equal_energy"] = ws.evaluate_equal_energy(net, n=16, side=1024, alpha=ALPHA,
                                                             kind=KIND, tol=TOL, ctx=ctx)
        # the Gaussian-curvature network (alpha 15) on the same test set
        net_g = ws.Net.load(WARMSTART_PARAMS_GAUSS, ctx=ctx)
        warm_eval_gauss = ws.evaluate(net_g, n=16, side=1024, alpha=15.0, kind=1, tol=TOL,
                                      ctx=ctx)

    batched_res = None
    if not args.no_batched:
        batched_res = batched_measurement(cm, torch, synth, ctx, dev, rank, world)
    recon_res = None
    if not args.no_recon and rank == 0:
        recon_res = recon_measurement(cm, torch, synth, ctx, dev, stream,
                                      with_oracle=not args.no_cpu_baseline)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_legs(img, cycles, opts, cm, torch, ctx, dev)

    # per warm step: 6 network kernels, 2 energy checks, then the solve graph
    # (initial energy, state initialisation, the cycles)
    per_cycle = kernels_per_cycle(opts, L)
    launches_per_solve = [8 + 2 + c * per_cycle for c in cycles]
    line = {"metric": METRIC, "value": sec_per_solve, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_solve * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args.side, L, {"G": opts.grid_points,
                                                     "K": opts.golden_evals,
                                                     "ncolors": opts.ncolors,
                                                     "coarse_ncolors": opts.coarse_ncolors}),
            "cycles_to_tol": cycles, "sweeps_per_s": statistics.mean(cycles) / sec_per_solve,
            "plain": {"s": sec_plain, "cycles_to_tol": cycles_plain, "psnr_db": psnr_plain,
                      "final_energy": st_plain[-1].energy_final},
            "warm_vs_plain_speedup": sec_plain / sec_warm,
            "warm_at_equal_energy": warm_eq_image,
            "psnr_db": psnr_warm, "psnr_noisy_db": synth.psnr(img.f, img.clean),
            "warmstart_eval_16x1024": warm_eval,
            "warmstart_eval_gauss_16x1024": warm_eval_gauss,
            "final_energy": final_E,
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": 4 * N,
                    "d2h_bytes_per_step": 4 * N},
            "gpu_launches": int(sum(launches_per_solve)),
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "b1_phase_ms": b1_ms, "batched": batched_res, "one_step": one_step_res,
            "reconstruction": recon_res,
            "cycle_variants": variants, "curvature_kinds": kinds_res,
            "complexity": complexity}
    line["autotune"] = tune_rec
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
