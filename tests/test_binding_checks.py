"""The binding checks every tensor before its pointer reaches the library,
which trusts the sizes it is given: shapes against the input image, the
block count of c_out, the sinogram's bin count, list lengths of the batched
call, and devices.  Run on CPU with the GPU-residency test stubbed, so each
rejection must happen before any library or CUDA call."""
import numpy as np
import pytest
import torch

import paper_2204_07921_gb300 as cm
from paper_2204_07921_gb300 import warmstart as ws


@pytest.fixture(autouse=True)
def on_gpu(monkeypatch):
    monkeypatch.setattr(cm, "_on_gpu", lambda t: True)


def img(H, W, dtype=torch.float32):
    return torch.zeros((H, W), dtype=dtype)


def test_energy_and_curvature():
    with pytest.raises(ValueError, match="shape"):
        cm.cm_energy(img(8, 8), img(8, 9), 1.0, cm.MEAN)
    with pytest.raises(TypeError):
        cm.cm_energy(img(8, 8), img(8, 8, torch.float64), 1.0, cm.MEAN)
    with pytest.raises(ValueError, match="contiguous"):
        cm.cm_energy(img(8, 8), img(8, 8).t(), 1.0, cm.MEAN)
    with pytest.raises(ValueError, match="shape"):
        cm.cm_curvature(img(8, 8), cm.MEAN, out=img(7, 8))
    with pytest.raises(ValueError, match="shape"):
        cm.cm_energy_noalloc(img(8, 8), img(9, 8), 1.0, cm.MEAN, torch.zeros(1, dtype=torch.float64))
    with pytest.raises(TypeError):
        cm.cm_energy_noalloc(img(8, 8), img(8, 8), 1.0, cm.MEAN, torch.zeros(1))


def test_phase_and_level():
    S = img(10, 13)
    for fn in (lambda **k: cm.cm_phase(S, k.get("R", img(10, 13)), k.get("f", img(10, 13)),
                                       1.0, cm.MEAN, 4, 0, c_out=k.get("c_out")),
               lambda **k: cm.cm_level(S, k.get("R", img(10, 13)), k.get("f", img(10, 13)),
                                       1.0, cm.MEAN, 4, c_out=k.get("c_out"))):
        with pytest.raises(ValueError, match="R"):
            fn(R=img(10, 12))
        with pytest.raises(ValueError, match="f"):
            fn(f=img(13, 10))
        # 3 x 4 blocks of side 4
        with pytest.raises(ValueError, match="12 blocks"):
            fn(c_out=torch.zeros(11))
        with pytest.raises(TypeError):
            fn(c_out=torch.zeros(12, dtype=torch.float64))
        with pytest.raises(TypeError):
            fn(c_out=torch.zeros(24)[::2])


def test_solve():
    f = img(16, 12)
    with pytest.raises(ValueError, match="u_out"):
        cm.cm_solve(f, 1.0, cm.MEAN, u_out=img(12, 16))
    with pytest.raises(ValueError, match="u0"):
        cm.cm_solve(f, 1.0, cm.MEAN, u0=img(16, 11))


def test_recon():
    k = torch.zeros((16, 12), dtype=torch.complex64)
    m = torch.zeros((16, 12), dtype=torch.uint8)
    with pytest.raises(TypeError, match="mask"):
        cm.cm_recon(k, torch.zeros((16, 13), dtype=torch.uint8), 0.1)
    with pytest.raises(TypeError, match="kspace"):
        cm.cm_recon(k.real.contiguous(), m, 0.1)
    with pytest.raises(ValueError, match="u0"):
        cm.cm_recon(k, m, 0.1, u0=img(12, 16))
    with pytest.raises(ValueError, match="u_out"):
        cm.cm_recon(k, m, 0.1, u_out=img(16, 11))
    with pytest.raises(ValueError, match="cycles"):
        cm.cm_recon(k, m, 0.1, cycles=-1)


def test_ct():
    H, W = 20, 17
    D = cm.cm_radon_bins(H, W)
    assert D == 2 * int(np.ceil(np.hypot(H - 1, W - 1) / 2)) + 3
    with pytest.raises(ValueError, match="sino"):
        cm.cm_radon_adjoint(img(30, D - 1), H, W)
    with pytest.raises(ValueError, match="sino"):
        cm.cm_recon_ct(img(30, D + 2), H, W, 1.0)
    with pytest.raises(ValueError, match="u0"):
        cm.cm_recon_ct(img(30, D), H, W, 1.0, u0=img(W, H))
    with pytest.raises(ValueError, match="cycles"):
        cm.cm_recon_ct(img(30, D), H, W, 1.0, cycles=-2)
    with pytest.raises(ValueError, match="n_angles"):
        cm.cm_radon(img(H, W), 0)


def test_batched():
    fs = [img(8, 8), img(12, 10)]
    with pytest.raises(ValueError, match="alphas"):
        cm.cm_solve_batched(fs, [1.0], [0, 0])
    with pytest.raises(ValueError, match="alphas"):
        cm.cm_solve_batched(fs, [1.0, 1.0], [0])
    with pytest.raises(ValueError, match="u_outs"):
        cm.cm_solve_batched(fs, [1.0, 1.0], [0, 0], u_outs=[img(8, 8)])
    with pytest.raises(ValueError, match=r"u_outs\[1\]"):
        cm.cm_solve_batched(fs, [1.0, 1.0], [0, 0], u_outs=[img(8, 8), img(10, 12)])
    with pytest.raises(ValueError, match=r"u0s\[0\]"):
        cm.cm_solve_batched(fs, [1.0, 1.0], [0, 0], u0s=[img(8, 7), None])
    assert cm.cm_solve_batched([], [], []) == ([], [])


def test_network_batches():
    f = torch.zeros((3, 8, 8))
    assert ws._batch(f)[1:] == (3, 8, 8)
    assert ws._batch(img(5, 6))[1:] == (1, 5, 6)
    with pytest.raises(ValueError, match="ustar"):
        ws._batch(torch.zeros((3, 8, 7)), "ustar", f.shape, f)
    with pytest.raises(ValueError):
        ws._batch(torch.zeros((2, 3, 8, 8)))
    with pytest.raises(TypeError):
        ws._batch(torch.zeros((3, 8, 8), dtype=torch.float16))
