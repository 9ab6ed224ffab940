"""The library's own 2-D DFT (cm_fft2d, the transform of the MRI-like
operator A = M F of Sec. 5) against numpy's FFT, element by element.

Tolerance.  A radix-2 transform of length M has log2(M) stages; each stage
rounds one complex product with an FP32 twiddle and one sum per element, a
relative error of a few eps (eps = 2^-24), so the error of a 2-D transform
has 2-norm at most about c K eps ||X||_2 with K = sum over the two axes of
log2(M) (power of two) or 3 log2(M) + 2 (Bluestein: a forward transform, a
product with the chirp spectrum, an inverse transform and two chirp
products) and c ~ 2.  Each element is held to that 2-norm bound, with
||X||_2 = sqrt(HW) ||x||_2 (Parseval); a wrong twiddle, permutation or
chirp gives errors of the size of the values, ~||x||_2 per element.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_07921_gb300 as cm  # noqa: E402

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -24


def _stages(n):
    M = 1
    while M < (n if n & (n - 1) == 0 else 2 * n - 1):
        M *= 2
    lg = M.bit_length() - 1
    return lg if n & (n - 1) == 0 else 3 * lg + 2


def _bound(H, W, x):
    K = _stages(H) + _stages(W)
    return 2.0 * K * EPS * np.sqrt(H * W) * np.linalg.norm(x)


SHAPES = [(64, 64), (1024, 1024), (67, 45), (33, 70), (1, 37), (37, 1), (1, 1), (2, 3),
          (256, 8192), (3, 5000), (16384, 2), (1000, 777)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2d_matches_numpy(shape, inverse):
    H, W = shape
    rng = np.random.default_rng(H * 7919 + W + int(inverse))
    x = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    y = cm.cm_fft2d(xd, inverse=inverse).cpu().numpy().astype(np.complex128)
    x64 = x.astype(np.complex128)
    ref = np.fft.ifft2(x64) * (H * W) if inverse else np.fft.fft2(x64)
    err = np.abs(y - ref)
    bound = _bound(H, W, x64)
    print(f"\n{shape} inv={inverse}: max err {err.max():.3e} bound {bound:.3e} "
          f"2-norm rel {np.linalg.norm(y - ref) / np.linalg.norm(ref):.2e}")
    assert np.all(err <= bound)
    assert np.linalg.norm(y - ref) <= bound


def test_fft2d_round_trip_and_in_place():
    """inverse(forward(x)) = H W x; the transform in place equals the
    out-of-place one bit for bit."""
    H, W = 96, 130
    rng = np.random.default_rng(3)
    x = (rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    y = cm.cm_fft2d(xd)
    z = xd.clone()
    cm.cm_fft2d(z, out=z)
    torch.cuda.synchronize()
    assert torch.equal(y, z)
    back = cm.cm_fft2d(y, inverse=True).cpu().numpy() / (H * W)
    assert np.abs(back - x).max() <= 2 * _bound(H, W, x.astype(np.complex128)) / (H * W) * 2


def test_fft2d_rejects_unsupported_sizes():
    lib = cm.load()
    ctx = cm.Context(0)
    x = torch.zeros((4, 4), dtype=torch.complex64, device="cuda")
    for H, W in ((8193, 2), (2, 8193), (16385, 2), (32768, 1), (0, 4)):
        rc = lib.cm_fft2d(ctx.handle, x.data_ptr(), x.data_ptr(), H, W, 0, None)
        assert rc == cm.CM_ERR_INVALID, (H, W)
    rc = lib.cm_fft2d(ctx.handle, x.data_ptr(), x.data_ptr(), 4, 4, 2, None)
    assert rc == cm.CM_ERR_INVALID
    assert lib.cm_fft2d(ctx.handle, None, x.data_ptr(), 4, 4, 0, None) == cm.CM_ERR_INVALID
    assert lib.cm_fft2d(ctx.handle, x.data_ptr(), x.data_ptr(), 4, 4, 1, None) == cm.CM_OK
