import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_terminal_summary(terminalreporter):
    """The energy gaps of the blocks where the GPU and the oracle picked
    shifts more than 1e-4 apart (ties), relative to the block energy scale."""
    mod = sys.modules.get("gpu_helpers")
    log = getattr(mod, "TIE_LOG", None) if mod else None
    if log:
        import numpy as np
        a = np.asarray(log)
        terminalreporter.write_line(
            f"tie gaps (E_A(c_gpu) - E_A(c_oracle)) / scale: n={a.size} max={a.max():.3e} "
            f"p99={np.quantile(a, 0.99):.3e} p50={np.quantile(a, 0.5):.3e} min={a.min():.3e}")
