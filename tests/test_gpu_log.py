"""Logging (CM_LOG) of the library's solves, in a child process (the level
is read once per process)."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = """
import torch, synth, paper_2204_07921_gb300 as cm
f = torch.from_numpy(synth.piecewise_image(64, 48, 5, 5, 0.08).f).cuda()
u, st = cm.cm_solve(f, 20.0, cm.MEAN, cycles=3, tol=0.0)
cm.cm_solve_batched([f, f.clone()], [20.0, 15.0], [cm.MEAN, cm.GAUSS], cycles=2, tol=0.0)
print("E", repr(st.energy_final), st.cycles_run)
"""


def _run(level):
    env = dict(os.environ, PYTHONPATH=ROOT)
    env.pop("CM_LOG", None)
    if level is not None:
        env["CM_LOG"] = str(level)
    return subprocess.run([sys.executable, "-c", CODE], cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=300, check=True)


def test_log_levels():
    quiet = _run(None)
    assert "[cm]" not in quiet.stderr
    one = _run(1)
    lines = [l for l in one.stderr.splitlines() if l.startswith("[cm]")]
    assert any(l.startswith("[cm] cm_solve 64x48 kind=0") and "cycles=3" in l for l in lines)
    assert sum("cm_solve_batched image" in l for l in lines) == 2
    assert not any("cycle 0 E" in l for l in lines)
    two = _run(2)
    cyc = [l for l in two.stderr.splitlines() if l.startswith("[cm]   cycle")]
    assert len(cyc) == 4 + 2 * 3        # the solve's E0..E3, each batched image's E0..E2
    # logging changes nothing: the same final energy with and without it
    assert quiet.stdout == one.stdout == two.stdout
