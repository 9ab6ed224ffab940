"""Batched solve (many images of uneven sizes in one graph per cycle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2204_07921_gb300 as cm  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


SHAPES = [(67, 45), (130, 97), (64, 64), (200, 150), (1, 37), (300, 260), (37, 1), (5, 3)]


@pytest.mark.parametrize("tol,cycles", [(1e-4, 300), (0.0, 4)])
def test_batched_equals_single_solves(tol, cycles):
    """Every image of the batch: u and statistics bit-identical to cm_solve
    of that image alone (same kernels in the same order), whatever the other
    images do (different sizes, level counts, kinds, alphas and stopping
    cycles)."""
    imgs = [synth.piecewise_image(H, W, 900 + i, 6, 0.08) for i, (H, W) in enumerate(SHAPES)]
    kinds = [i % 4 for i in range(len(imgs))]   # all four curvature kinds
    alphas = [20.0 if i % 3 else 10.0 for i in range(len(imgs))]
    fs = [dev(im.f) for im in imgs]
    ub, sb = cm.cm_solve_batched(fs, alphas, kinds, cycles=cycles, tol=tol)
    torch.cuda.synchronize()
    cyc = []
    for i in range(len(imgs)):
        us, ss = cm.cm_solve(fs[i], alphas[i], kinds[i], cycles=cycles, tol=tol)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ub[i].cpu().numpy(), us.cpu().numpy())
        assert sb[i].cycles_run == ss.cycles_run
        assert sb[i].converged == ss.converged
        assert sb[i].monotone_violations == ss.monotone_violations
        assert sb[i].trace() == ss.trace()
        assert sb[i].energy_final == ss.energy_final
        cyc.append(ss.cycles_run)
    if tol > 0:
        assert len(set(cyc)) > 1    # images stopped at different cycles


def test_batched_repeat_is_deterministic_and_reuses_graph():
    items = synth.uneven_batch(6, sides=(128, 192, 256))
    fs = [dev(it.image.f) for it in items]
    al = [it.alpha for it in items]
    kd = [it.kind for it in items]
    ctx = cm.Context(0)
    u1, s1 = cm.cm_solve_batched(fs, al, kd, tol=1e-4, ctx=ctx)
    u1 = [t.clone() for t in u1]
    u2, s2 = cm.cm_solve_batched(fs, al, kd, tol=1e-4, ctx=ctx)
    for a, b in zip(u1, u2):
        assert torch.equal(a, b)
    assert [s.cycles_run for s in s1] == [s.cycles_run for s in s2]
    assert all(s.converged for s in s1)
    # the denoised images are closer to the clean ones
    for it, u in zip(items, u1):
        assert synth.psnr(u.cpu().numpy(), it.image.clean) > synth.psnr(it.image.f, it.image.clean)


def test_batched_invalid_arguments():
    f = dev(np.zeros((8, 8)))
    with pytest.raises(cm.CMError):
        cm.cm_solve_batched([f, f], [1.0, -1.0], [0, 0])
    with pytest.raises(cm.CMError):
        cm.cm_solve_batched([f], [1.0], [4])    # kinds are 0..3
