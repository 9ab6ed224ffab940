"""Warm-start CNN kernels (BF16 tensor cores) against the FP64 oracle.

Tolerances: activations and weights are BF16 (8-bit significand, relative
rounding 2^-9 ~ 0.2%) through five layers with FP32 accumulation, so the
network output agrees with the FP64 oracle to a few percent of its scale;
gradients likewise per layer (relative L2 error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_07921_gb300 as cm  # noqa: E402
from paper_2204_07921_gb300 import warmstart as ws  # noqa: E402
from oracle import cnn as ocnn  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_zero_net_returns_f_exactly():
    net = ws.Net(ws.init_params(1, zero_last=True))
    f = dev(np.random.default_rng(0).random((2, 19, 33)))
    u0 = net.forward(f)
    torch.cuda.synchronize()
    assert torch.equal(u0, f)


@pytest.mark.parametrize("shape", [(2, 19, 33), (1, 8, 16), (3, 17, 5), (1, 1, 7)])
def test_forward_parity(shape):
    rng = np.random.default_rng(sum(shape))
    p = ws.init_params(7, zero_last=False)
    f = rng.random(shape).astype(np.float32)
    net = ws.Net(p)
    out_g = (net.forward(dev(f)) - dev(f)).cpu().numpy().astype(np.float64)
    u0_o, _ = ocnn.forward(p.astype(np.float64), f.astype(np.float64))
    out_o = u0_o - f
    scale = np.max(np.abs(out_o))
    assert scale > 1e-3
    assert np.max(np.abs(out_g - out_o)) <= 3e-2 * scale


def test_gradient_parity():
    rng = np.random.default_rng(3)
    shape = (2, 21, 34)
    p = ws.init_params(11, zero_last=False)
    p[-289:] *= 3.0   # a livelier last layer
    f = rng.random(shape).astype(np.float32)
    us = (f + 0.05 * rng.normal(size=shape)).astype(np.float32)
    net = ws.Net(p)
    Lg, gg = net.gradients(dev(f), dev(us))
    Lo, go = ocnn.gradients(p.astype(np.float64), f.astype(np.float64), us.astype(np.float64))
    assert Lg == pytest.approx(Lo, rel=3e-2)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in ocnn.SHAPES])
    for (name, _), a, b in zip(ocnn.SHAPES, offs[:-1], offs[1:]):
        ref = go[a:b]
        err = np.linalg.norm(gg[a:b] - ref) / max(np.linalg.norm(ref), 1e-12)
        assert err <= 5e-2, (name, err)


def test_train_step_follows_adam_and_lowers_loss():
    """The first Adam step moves every parameter with a clear gradient by
    ~lr * sign(g); a few steps on one batch lower the loss."""
    rng = np.random.default_rng(5)
    shape = (4, 32, 32)
    f = rng.random(shape).astype(np.float32)
    us = (f + 0.03 * rng.normal(size=shape)).astype(np.float32)
    p = ws.init_params(2, zero_last=False)
    net = ws.Net(p)
    L0, g = net.gradients(dev(f), dev(us))
    net.train_step(dev(f), dev(us), 1e-3)
    p1 = net.get_params()
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    step = p - p1
    np.testing.assert_allclose(step[big], 1e-3 * np.sign(g[big]), rtol=2e-2, atol=2e-5)
    losses = [net.train_step(dev(f), dev(us), 1e-3) for _ in range(30)]
    assert losses[-1] < 0.8 * L0


def test_warmstart_energy_fallback():
    """A network whose output raises the energy is rejected by the sweep's
    energy: u0 = f for that image."""
    img = synth.piecewise_image(64, 64, 5, 6, 0.05)
    f = dev(img.f[None])
    p = ws.init_params(9, zero_last=False)
    p[-289:-1] = 5.0           # a wild last layer
    net = ws.Net(p)
    u0, used = ws.warmstart(net, f, 20.0, cm.MEAN, check_energy=True)
    torch.cuda.synchronize()
    assert used == [0]
    assert torch.equal(u0, f)
    net0 = ws.Net(ws.init_params(9, zero_last=True))
    u0, used = ws.warmstart(net0, f, 20.0, cm.MEAN, check_energy=True)
    assert used == [1] and torch.equal(u0, f)


@pytest.mark.parametrize("name,kind,alpha", [("warmstart_mean_a20.npz", cm.MEAN, 20.0),
                                             ("warmstart_gauss_a15.npz", cm.GAUSS, 15.0)])
def test_shipped_warmstart_saves_cycles(name, kind, alpha):
    """The shipped networks (mean curvature, alpha 20; Gaussian curvature,
    alpha 15) pass the energy check on fresh test images and the solve from
    their output needs no more cycles than the solve from f."""
    import os
    path = os.path.join(os.path.dirname(ws.__file__), "data", name)
    net = ws.Net.load(path)
    saved = 0
    for i in range(2):
        im = synth.warmstart_image("test", 100 + i, 512)
        f = dev(im.f)
        u0, used = ws.warmstart(net, f[None], alpha, kind, check_energy=True)
        assert used == [1]
        _, sp = cm.cm_solve(f, alpha, kind, cycles=200, tol=1e-4)
        _, sw = cm.cm_solve(f, alpha, kind, cycles=200, tol=1e-4, u0=u0[0].contiguous())
        assert sw.cycles_run <= sp.cycles_run
        saved += sp.cycles_run - sw.cycles_run
    assert saved > 0
