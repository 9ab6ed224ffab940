"""The allocation-free energy entry point (cm_energy_noalloc).

It serves callers that cannot let a library allocate device memory -- for
example a process whose caching allocator already holds the GPU's memory, or
code that must avoid the implicit synchronisation of cudaMalloc/cudaFree --
by keeping its scratch in a fixed array inside the library.  This file runs
last so that a stop at its first failure has already run every other test.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_07921_gb300 as cm  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _call(lib, u, f, alpha, kind, E_dev):
    return lib.cm_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                 u.shape[0], u.shape[1], ctypes.c_float(alpha), kind,
                                 ctypes.c_void_p(E_dev.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_energy_matches_context_energy_twice():
    """Two calls in a row through the C ABI agree with cm_energy (same
    tolerance as the energy parity tests: 2e-6 relative); the second call
    reuses the scratch the first left behind."""
    lib = cm.load()
    lib.cm_energy_noalloc.restype = ctypes.c_int
    cases = [(synth.piecewise_image(512, 384, 71, 10, 0.08), 20.0, cm.MEAN),
             (synth.piecewise_image(67, 45, 72, 5, 0.1), 15.0, cm.GAUSS)]
    for img, alpha, kind in cases:
        u = torch.from_numpy(img.f).cuda()
        f = torch.from_numpy(img.clean).cuda()
        E_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, u, f, alpha, kind, E_dev) == cm.CM_OK
        torch.cuda.synchronize()
        E_ref = cm.cm_energy(u, f, alpha, kind)
        assert float(E_dev.item()) == pytest.approx(E_ref, rel=2e-6)


def test_noalloc_rejects_oversize_and_bad_arguments():
    lib = cm.load()
    lib.cm_energy_noalloc.restype = ctypes.c_int
    u = torch.zeros((8, 8), device="cuda")
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 4097 x 4097 needs 129 x 129 tiles > 16384: rejected before any device access
    rc = lib.cm_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                               4097, 4097, ctypes.c_float(1.0), 0,
                               ctypes.c_void_p(E_dev.data_ptr()), stream)
    assert rc == cm.CM_ERR_INVALID
    # sizes beyond the image limits of every entry point (W = INT_MAX would
    # overflow the int tile count) are rejected before the tile count is formed
    for H, W in ((1, 2 ** 31 - 1), (2 ** 31 - 1, 1), (1, 524281)):
        rc = lib.cm_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                   H, W, ctypes.c_float(1.0), 0,
                                   ctypes.c_void_p(E_dev.data_ptr()), stream)
        assert rc == cm.CM_ERR_INVALID, (H, W)
    rc = lib.cm_energy_noalloc(None, ctypes.c_void_p(u.data_ptr()), 8, 8, ctypes.c_float(1.0), 0,
                               ctypes.c_void_p(E_dev.data_ptr()), stream)
    assert rc == cm.CM_ERR_INVALID
    rc = lib.cm_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(u.data_ptr()), 8, 8,
                               ctypes.c_float(-1.0), 0, ctypes.c_void_p(E_dev.data_ptr()), stream)
    assert rc == cm.CM_ERR_INVALID
