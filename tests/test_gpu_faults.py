"""Failure detection without a GPU fault: a bounded device wait that runs out
returns a status the host reads (the context stays usable), and an injected
allocation failure (host side) returns CM_ERR_OOM."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

import paper_2204_07921_gb300 as cm  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_completes():
    r = cm.cm_selftest_wait(0, limit=1000)
    assert r == {"timed_out": 1, "completed": 1}
    # the context is still usable: a solve runs normally afterwards
    f = torch.rand(40, 36, device="cuda")
    u, st = cm.cm_solve(f, 20.0, cm.MEAN, cycles=2)
    torch.cuda.synchronize()
    assert st.cycles_run == 2 and st.energy_final < st.energy_initial


def test_selftest_rejects_bad_limits():
    for limit in (0, (1 << 22) + 1):
        with pytest.raises(cm.CMError) as e:
            cm.cm_selftest_wait(0, limit=limit)
        assert e.value.code == cm.CM_ERR_INVALID


def test_injected_allocation_failure_is_reported():
    """A child process with CM_FAULT_ALLOC_LIMIT=4096: a 64 x 64 solve needs a
    16 KiB scratch image and fails with CM_ERR_OOM; an energy (a few bytes of
    scratch) on the same context still succeeds."""
    code = r'''
import torch, paper_2204_07921_gb300 as cm
f = torch.rand(64, 64, device="cuda")
ctx = cm.Context(0)
try:
    cm.cm_solve(f, 20.0, cm.MEAN, cycles=1, ctx=ctx)
    print("no error")
except cm.CMError as e:
    print("code", e.code)
E = cm.cm_energy(f, f, 20.0, cm.MEAN, ctx=ctx)
print("energy", E)
'''
    env = dict(os.environ, CM_FAULT_ALLOC_LIMIT="4096", PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.split("\n")
    assert f"code {cm.CM_ERR_OOM}" in lines
    assert any(l.startswith("energy ") and float(l.split()[1]) >= 0.0 for l in lines)
