"""Warm-start CNN kernels (BF16 tensor cores) against the FP64 oracle.

Tolerances.  BF16 keeps an 8-bit significand, so one rounding has relative
error at most u = 2^-8 (~0.39%).  Along every path through the network an
output carries one rounding of each weight and of each stored activation per
layer: two per layer, ten over the five hidden layers, each relative to the
magnitude of the term it rounds; FP32 accumulation adds nothing visible.
The sums of 9 x 32 terms cancel, so a term's magnitude is about the size of
the output's scale |ref| + rms(ref) (measured ratio below 2).  Per element:

    |gpu - oracle| <= 20 u (|ref| + rms(ref))  (= 7.8e-2)

for the network output.  A gradient adds the backward pass's roundings to
those of the forward pass that feed the loss: the deepest one (W2, a sum of
x1 dZ2 over the pixels) has dZ2 rounded after each of the four backward
layers with the (flipped) BF16 weights of each, ten more roundings, and its
sums over few pixels (1428 at 2 x 21 x 34) cancel more than the network's
output does, so its bound is 32 u (= 0.125).  Measured: output 4.4e-2
(multi-strip shapes); gradients 9.5e-2 (W2 at 2 x 21 x 34), 2.2e-2 at
4 x 250 x 260.  A mis-indexed tap, strip or channel makes errors of the
order of the values themselves, far above either bound.  The loss is a
mean of squares of the output error: 3e-2 relative.
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

# Per-element bounds, |d| <= TOL (|ref| + rms(ref)): see the module docstring.
U_BF16 = 2.0 ** -8
FWD_TOL = 20 * U_BF16
GRAD_TOL = 32 * U_BF16
LOSS_TOL = 3e-2


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_batch_pixel_limit_is_rejected_before_any_access():
    """N H W >= 2^31 is refused with CM_ERR_INVALID up front (the kernels
    index rows and strips in int); the small buffer is never read."""
    net = ws.Net(ws.init_params(1, zero_last=True))
    f = dev(np.zeros((1, 4, 4)))
    lib = ws._lib()
    rc = lib.cm_net_forward(net._h, f.data_ptr(), 2 ** 27, 4, 4, f.data_ptr(), None)
    assert rc == cm.CM_ERR_INVALID
    assert lib.cm_net_forward(net._h, f.data_ptr(), 1, 4, 4, f.data_ptr(), None) == cm.CM_OK
    torch.cuda.synchronize()


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
    rms = np.sqrt(np.mean(out_o ** 2))
    assert rms > 1e-3
    assert np.all(np.abs(out_g - out_o) <= FWD_TOL * (np.abs(out_o) + rms))


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
    assert Lg == pytest.approx(Lo, rel=LOSS_TOL)
    _check_gradients(gg, go, "2x21x34")


def _check_gradients(gg, go, label):
    """Every gradient element within GRAD_TOL (|ref| + rms of its layer)."""
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in ocnn.SHAPES])
    worst = []
    for (name, _), a, b in zip(ocnn.SHAPES, offs[:-1], offs[1:]):
        ref, got = go[a:b], gg[a:b].astype(np.float64)
        rms = np.sqrt(np.mean(ref ** 2))
        ratio = np.abs(got - ref) / (np.abs(ref) + rms)
        worst.append(f"{name}:{ratio.max():.2e}")
        assert np.all(ratio <= GRAD_TOL), (label, name, ratio.max())
    print(f"\ngradients {label}: " + " ".join(worst))


def _strips(N, H, W):
    """Work units of the tcgen05 convolution: strips of 4 rows x 128 columns."""
    return N * (-(-H // 4)) * (-(-W // 128))


# Shapes with more strips than the persistent grid has CTAs (one per SM, 152
# on a GB300): the first gives most CTAs five strips, so the halo ring wraps
# (strip 4 reuses buffer 0 of the four), the TMEM accumulator set of strip 0
# is reused by strip 4 after its drain, and the halo of strip k + 3 is
# refilled while strip k is in the tensor cores; both have W > 128 (column strips that share a halo column,
# a ragged last column strip) and H not a multiple of 4 (a ragged last row
# strip); the second has W not a multiple of 4, so its activation rows carry
# a pad that the last column strip's halo zeroes.
MULTI_STRIP = [(4, 250, 260), (2, 202, 301)]


def _oracle_forward_out(p, f):
    """conv6(...) of the FP64 oracle, one image at a time (each image is
    independent; this keeps the oracle's im2col matrices small)."""
    outs = []
    for n in range(f.shape[0]):
        u0, _ = ocnn.forward(p, f[n:n + 1].astype(np.float64))
        outs.append(u0[0] - f[n].astype(np.float64))
    return np.stack(outs)


@pytest.mark.parametrize("shape", MULTI_STRIP)
def test_forward_parity_multi_strip(shape):
    """Element by element on the persistent multi-strip path that the
    16 x 1024^2 inference runs (MODE 0 layers and the MODE 2 output layer)."""
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert _strips(*shape) > nsm
    if shape == MULTI_STRIP[0]:
        assert _strips(*shape) > 4 * nsm   # some CTAs run five strips: ring and set wrap
    rng = np.random.default_rng(sum(shape) + 1)
    p = ws.init_params(17, zero_last=False)
    f = rng.random(shape).astype(np.float32)
    net = ws.Net(p)
    out_g = (net.forward(dev(f)) - dev(f)).cpu().numpy().astype(np.float64)
    out_o = _oracle_forward_out(p.astype(np.float64), f)
    err = np.abs(out_g - out_o)
    rms = np.sqrt(np.mean(out_o ** 2))
    ratio = err / (np.abs(out_o) + rms)
    print(f"\nforward {shape}: max|d|/max|out| {err.max() / np.abs(out_o).max():.3e} "
          f"max|d|/(|out|+rms) {ratio.max():.3e} p99.9 {np.quantile(ratio, 0.999):.3e}")
    assert rms > 1e-3
    assert np.all(err <= FWD_TOL * (np.abs(out_o) + rms))


def test_gradient_parity_multi_strip():
    """Every parameter's gradient, element by element, at the multi-strip
    shape (the MODE 1 dX layers and the weight-gradient reductions over many
    tiles)."""
    shape = MULTI_STRIP[0]
    rng = np.random.default_rng(31)
    p = ws.init_params(19, zero_last=False)
    p[-289:] *= 3.0   # a livelier last layer
    f = rng.random(shape).astype(np.float32)
    us = (f + 0.05 * rng.normal(size=shape)).astype(np.float32)
    net = ws.Net(p)
    Lg, gg = net.gradients(dev(f), dev(us))
    # the loss is the mean over all pixels of equal-sized images: the batch
    # gradient is the mean of the per-image gradients
    Lo, go = 0.0, np.zeros(ocnn.N_PARAMS)
    for n in range(shape[0]):
        L1, g1 = ocnn.gradients(p.astype(np.float64), f[n:n + 1].astype(np.float64),
                                us[n:n + 1].astype(np.float64))
        Lo += L1 / shape[0]
        go += g1 / shape[0]
    assert Lg == pytest.approx(Lo, rel=LOSS_TOL)
    _check_gradients(gg, go, "x".join(map(str, shape)))


def test_inference_16x1024_sampled():
    """The warm-start workload's inference, as the bench launches it: the
    shipped network on a batch of 16 test images of 1024^2.  The network's
    receptive field has radius 6 (six 3 x 3 layers), so the oracle's output at
    a pixel is exact from the crop of radius 6 around it, clipped at the image
    border (where every layer's own zero padding then applies as in the whole
    image); 640 sampled pixels, corners and edges included, element by
    element."""
    import os
    path = os.path.join(os.path.dirname(ws.__file__), "data", "warmstart_mean_a20.npz")
    p = np.load(path)["params"].astype(np.float64)
    net = ws.Net.load(path)
    F = np.stack([synth.warmstart_image("test", i, 1024).f for i in range(16)])
    out_g = (net.forward(dev(F)) - dev(F)).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(16)
    R = 6
    picks = []
    for n in range(16):
        rc = [(0, 0), (0, 1023), (1023, 0), (1023, 1023), (0, 500), (511, 1023)]
        rc += [tuple(x) for x in rng.integers(0, 1024, size=(34, 2))]
        picks += [(n, r, c) for r, c in rc]
    ref = np.zeros(len(picks))
    for i, (n, r, c) in enumerate(picks):
        r0, c0 = max(0, r - R), max(0, c - R)
        crop = F[n, r0:r + R + 1, c0:c + R + 1].astype(np.float64)
        u0, _ = ocnn.forward(p, crop[None])
        ref[i] = u0[0, r - r0, c - c0] - crop[r - r0, c - c0]
    got = np.array([out_g[n, r, c] for n, r, c in picks])
    rms = np.sqrt(np.mean(ref ** 2))
    ratio = np.abs(got - ref) / (np.abs(ref) + rms)
    print(f"\ninference 16x1024^2: {len(picks)} pixels, max |d|/(|ref|+rms) {ratio.max():.3e}")
    assert rms > 1e-3
    assert np.all(ratio <= FWD_TOL)


def test_gradient_parity_training_batch():
    """Every gradient element at the training workload's batch shape (16
    images of 256^2, the shape the training loop steps on)."""
    shape = (16, 256, 256)
    rng = np.random.default_rng(41)
    p = ws.init_params(23, zero_last=False)
    p[-289:] *= 3.0
    f = rng.random(shape).astype(np.float32)
    us = (f + 0.05 * rng.normal(size=shape)).astype(np.float32)
    net = ws.Net(p)
    Lg, gg = net.gradients(dev(f), dev(us))
    Lo, go = 0.0, np.zeros(ocnn.N_PARAMS)
    for n in range(shape[0]):
        L1, g1 = ocnn.gradients(p.astype(np.float64), f[n:n + 1].astype(np.float64),
                                us[n:n + 1].astype(np.float64))
        Lo += L1 / shape[0]
        go += g1 / shape[0]
    assert Lg == pytest.approx(Lo, rel=LOSS_TOL)
    _check_gradients(gg, go, "16x256x256")


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
