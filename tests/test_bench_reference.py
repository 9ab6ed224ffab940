"""The benchmark's reference arm (the FP64 oracle on the host cores: the
warm start in FP64, then the sweep with the same schedule) keeps the
one-JSON-line contract on CPU: the keys and their types, value =
cpu_baseline.value = e2e.value, the GPU line's config, and under several
ranks only rank 0 runs and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--side", "64",
                           "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_line_contract():
    p = _run()
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is False and d["unit"] == "s" and d["value"] > 0
    assert d["config"]["workload"].startswith("denoise 64^2")
    # the GPU line's config when the autotuner picks the CPU legs' schedule
    import bench
    assert d["config"] == bench.workload_config(64, bench._auto_levels(64), bench.REF_SCHEDULE)
    assert d["oracle_warmstart_s"] > 0 and isinstance(d["oracle_warmstart_kept"], bool)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["oracle_converged"] is True and d["oracle_cycles"] >= 1


def test_reference_other_ranks_exit_without_work():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_launch_count_follows_the_schedule():
    """gpu_launches counts the solve's kernels from the level schedule: the
    bench's colour rule equals the oracle's for every option, and a 1024^2
    cycle of the tuned schedule (4 colours, 2 on the coarse levels) is the
    39 kernels of its ncu launch list (32 phases, 4 coarse applies, the tile
    sums, the energy, the stopping test)."""
    import bench
    import oracle
    import paper_2204_07921_gb300 as cm
    for nc in (0, 2, 4, 9, 16):
        for cn in (0, 1, 2, 4):
            o = cm.default_options(ncolors=nc, coarse_ncolors=cn)
            for j in range(12):
                b = 1 << j
                assert bench.level_colours(o, b) == oracle.level_colours(nc, b, cn), (nc, cn, b)
    assert bench.kernels_per_cycle(cm.default_options(ncolors=4, coarse_ncolors=2), 10) == 39
    # one coarse colour: 24 fine phases, 4 coarse phases and 4 applies, the tile
    # sums, the energy, the stopping test
    assert bench.kernels_per_cycle(cm.default_options(ncolors=4, coarse_ncolors=1), 10) == 35
    assert bench.kernels_per_cycle(cm.default_options(ncolors=4), 10) == 47
    assert bench.kernels_per_cycle(cm.default_options(ncolors=4), 6) == 2 + 6 * 4
