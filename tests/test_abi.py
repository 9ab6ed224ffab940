"""The C ABI library builds, loads and exports every function include/cm.h
declares (no compute: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cm_create", "cm_destroy", "cm_energy", "cm_solve", "cm_phase",
                     "cm_last_error", "cm_options_default", "cm_auto_levels"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2204_07921_gb300 import build
    so = build.build()
    lib = ctypes.CDLL(so)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    """Entry points that touch no device: defaults, auto levels, argument
    checks before any CUDA call."""
    import paper_2204_07921_gb300 as cm
    lib = cm.load()
    o = cm.Options()
    assert lib.cm_options_default(ctypes.byref(o)) == 0
    assert (o.ncolors, o.grid_points, o.golden_evals, o.paper_candidate) == (4, 5, 6, 1)
    assert (o.use_graph, o.max_trace, o.one_step, o.vcycle) == (1, 4096, 0, 0)
    assert (o.coarse_spec, o.coarse_dmax, o.block_sides) == (-1, 0, 0)
    assert lib.cm_options_default(None) == cm.CM_ERR_INVALID
    assert lib.cm_auto_levels(64, 64) == 6
    assert lib.cm_auto_levels(1024, 1024) == 10
    assert lib.cm_auto_levels(2048, 2048) == 11
    assert lib.cm_auto_levels(1, 5) == 1
    # null context is rejected without touching the device
    E = ctypes.c_double()
    assert lib.cm_energy(None, None, None, 4, 4, 1.0, 0, ctypes.byref(E), None) == cm.CM_ERR_INVALID
    assert lib.cm_solve(None, None, 4, 4, 1.0, 0, 0, 1, 0.0, None, None, None, None, None) \
        == cm.CM_ERR_INVALID
    assert lib.cm_create(None, 0) == cm.CM_ERR_INVALID
    assert lib.cm_last_error(None) == b"null context"


def test_image_size_limits():
    """Images of 1 .. CM_MAX_SIDE rows and columns and at most CM_MAX_PIXELS
    pixels are accepted; the host-only cm_radon_bins shows the same rule
    the entry points apply before any CUDA call."""
    import numpy as np
    import paper_2204_07921_gb300 as cm
    text = open(os.path.join(HEADER_DIR, "cm.h")).read()
    assert re.search(r"#define CM_MAX_SIDE 524280", text)
    assert re.search(r"#define CM_MAX_PIXELS 2147483647LL", text)
    lib = cm.load()
    # 65535 row tiles of 8 rows: the y-dimension limit of a launch grid
    side, pixels = 65535 * 8, 2 ** 31 - 1
    for H, W in ((1, 1), (side, 1), (1, side), (side, 4096), (46340, 46340)):
        assert H * W <= pixels
        assert lib.cm_radon_bins(H, W) == 2 * int(np.ceil(np.hypot(H - 1, W - 1) / 2)) + 3
    for H, W in ((0, 5), (5, 0), (-1, 5), (side + 1, 1), (1, side + 1), (side, 4097),
                 (1 << 20, 1), (46341, 46341), (50000, 50000)):
        assert lib.cm_radon_bins(H, W) == -1, (H, W)
    with pytest.raises(ValueError):
        cm.cm_radon_bins(50000, 50000)


def test_sinogram_entry_limit():
    """The CT entry points index the n_angles x D sinogram with int: the
    host-only cm_radon_entries (the check cm_radon, cm_radon_adjoint and
    cm_recon_ct apply before any CUDA call) gives n_angles x D, and -1 once
    that count passes CM_MAX_SINO = 2^31 - 1, for image sizes that are
    themselves within the limits."""
    import numpy as np
    import paper_2204_07921_gb300 as cm
    text = open(os.path.join(HEADER_DIR, "cm.h")).read()
    assert re.search(r"#define CM_MAX_SINO 2147483647LL", text)
    lib = cm.load()
    for H, W, n in ((32, 32, 1), (256, 256, 180), (32768, 32768, 100), (46340, 46340, 1)):
        D = 2 * int(np.ceil(np.hypot(H - 1, W - 1) / 2)) + 3
        assert n * D <= 2 ** 31 - 1
        assert lib.cm_radon_entries(H, W, n) == n * D
    # 32768^2 (D = 46343): 46339 angles fit, 50000 (2.3e9 entries) do not
    D = lib.cm_radon_bins(32768, 32768)
    assert D == 46343
    n_fit = (2 ** 31 - 1) // D
    assert lib.cm_radon_entries(32768, 32768, n_fit) == n_fit * D
    for H, W, n in ((32768, 32768, n_fit + 1), (32768, 32768, 50000), (32, 32, 0),
                    (32, 32, 100001), (0, 32, 5), (600000, 1, 5)):
        assert lib.cm_radon_entries(H, W, n) == -1, (H, W, n)
    with pytest.raises(ValueError):
        cm.cm_radon_entries(32768, 32768, 50000)


def test_default_budget_agrees_with_oracle():
    """Parity tests rely on the library and the oracle using the same
    default search budget."""
    import oracle
    import paper_2204_07921_gb300 as cm
    o = cm.default_options()
    assert (o.grid_points, o.golden_evals) == (oracle.DEFAULT_G, oracle.DEFAULT_K)


def test_auto_levels_agree_with_oracle():
    import oracle
    import paper_2204_07921_gb300 as cm
    for H, W in [(64, 64), (512, 512), (1024, 1024), (67, 45), (1, 1), (3, 100), (130, 97)]:
        assert cm.cm_auto_levels(H, W) == oracle.auto_levels(H, W)


def test_header_is_plain_c(tmp_path):
    """include/cm.h compiles as C99 with warnings as errors (a C ABI, not a
    C++ one)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_cm.c"
    src.write_text('#include "cm.h"\nint main(void) { cm_options o; '
                   'return cm_options_default(&o); }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", HEADER_DIR, str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
