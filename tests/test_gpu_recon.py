"""GPU parity of the reconstruction extension (Sec. 5: MRI-like A = M F, and
CT with the Radon pair) against the FP64 oracle in oracle/recon.py.

Tolerances: the GPU runs the same algorithm in FP32 (the library's own FFT,
FP32 CG vectors, FP64 reductions), the oracle in FP64.  One FFT round trip
keeps ~1e-6 relative accuracy; the eight CG iterations of a colour step
amplify rounding by at most a few times the system's condition number
(<= 1 + 1/(2 alpha) on the finest level), so per-pixel differences after a
level stay below 2e-4 on images of range ~1, and the objective traces agree
to 1e-4 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2204_07921_gb300 as cm  # noqa: E402
import synth  # noqa: E402
from oracle import recon  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev_case(case):
    return (torch.from_numpy(case.kspace).to(DEV), torch.from_numpy(case.mask).to(DEV))


@pytest.mark.parametrize("shape", [(64, 64), (67, 45), (33, 70)])
@pytest.mark.parametrize("kind", [cm.MEAN, cm.GAUSS])
def test_finest_level_cycle_matches_oracle(shape, kind):
    """One cycle of the finest level only (every colour, CG on the coupled
    system): the image and J against the oracle's."""
    H, W = shape
    case = synth.mri_case(H, W, 21 + H, accel=3.0, sigma=0.01)
    kd, md = dev_case(case)
    alpha = 0.02
    u, tr = cm.cm_recon(kd, md, alpha, kind, levels=1, cycles=1, cg_iters=8)
    torch.cuda.synchronize()
    uo, tro = recon.solve(case.kspace, case.mask, alpha, kind, levels=1, cycles=1, cg_iters=8)
    ug = u.cpu().numpy()
    assert np.max(np.abs(ug - uo)) < 2e-4
    np.testing.assert_allclose(tr, tro, rtol=1e-4)


@pytest.mark.parametrize("ncolors,sides", [(4, 0), (2, 0), (4, 1), (0, 0)])
def test_full_cycles_match_oracle(ncolors, sides):
    """Three cycles over every level (coupled solves at block sides up to
    32, or the paper's odd sides; 2, 4 or decoupled colours): J after each
    cycle against the oracle's, and the reconstruction beats the
    zero-filled start."""
    case = synth.mri_case(64, 64, 7, accel=3.0, sigma=0.01)
    kd, md = dev_case(case)
    opts = cm.default_options(ncolors=ncolors, block_sides=sides)
    u, tr = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=3, cg_iters=8, options=opts)
    torch.cuda.synchronize()
    uo, tro = recon.solve(case.kspace, case.mask, 0.02, cm.MEAN, cycles=3, cg_iters=8,
                          ncolors=ncolors, sides=sides)
    np.testing.assert_allclose(tr, tro, rtol=1e-4)
    ug = u.cpu().numpy()
    assert np.max(np.abs(ug - uo)) < 1e-3
    u0 = np.real(recon.adjoint(case.kspace.astype(complex), case.mask.astype(float)))
    assert synth.psnr(ug, case.clean) > synth.psnr(u0, case.clean) + 0.5


def test_full_mask_is_the_closed_form_and_repeatable():
    """Every entry sampled: A^H A = I and each colour step is the diagonal
    closed form, which CG reaches in one iteration; a second run on the same
    context reuses the captured cycle and gives the same bits."""
    case = synth.mri_case(40, 36, 3, accel=1.0, sigma=0.02)
    kd, md = dev_case(case)
    ctx = cm.Context(0)
    u1, t1 = cm.cm_recon(kd, md, 0.3, cm.MEAN, cycles=2, cg_iters=3, ctx=ctx)
    u1 = u1.clone()
    u2, t2 = cm.cm_recon(kd, md, 0.3, cm.MEAN, cycles=2, cg_iters=3, ctx=ctx)
    torch.cuda.synchronize()
    assert torch.equal(u1, u2) and np.array_equal(t1, t2)
    uo, tro = recon.solve(case.kspace, case.mask, 0.3, cm.MEAN, cycles=2, cg_iters=3)
    assert np.max(np.abs(u1.cpu().numpy() - uo)) < 1e-4
    np.testing.assert_allclose(t1, tro, rtol=1e-5)


def test_initial_guess_and_zero_cycles():
    case = synth.mri_case(32, 32, 5, accel=3.0, sigma=0.01)
    kd, md = dev_case(case)
    u, tr = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=0)
    torch.cuda.synchronize()
    u0 = np.real(recon.adjoint(case.kspace.astype(complex), case.mask.astype(float)))
    assert np.max(np.abs(u.cpu().numpy() - u0)) < 1e-5
    assert tr.shape == (1,)
    assert tr[0] == pytest.approx(recon.objective(u0, case.kspace, case.mask, 0.02, cm.MEAN),
                                  rel=1e-4)
    start = torch.full((32, 32), 0.5, device=DEV)
    u, tr = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=1, u0=start)
    torch.cuda.synchronize()
    uo, tro = recon.solve(case.kspace, case.mask, 0.02, cm.MEAN, cycles=1,
                          u0=np.full((32, 32), 0.5))
    np.testing.assert_allclose(tr, tro, rtol=1e-4)


def test_recon_invalid_arguments():
    case = synth.mri_case(16, 16, 5)
    kd, md = dev_case(case)
    for kw in (dict(alpha=-1.0), dict(cg_iters=0), dict(kind=4)):
        args = dict(alpha=0.02, kind=cm.MEAN, cg_iters=8)
        args.update(kw)
        with pytest.raises(cm.CMError) as e:
            cm.cm_recon(kd, md, args["alpha"], args["kind"], cg_iters=args["cg_iters"])
        assert e.value.code == cm.CM_ERR_INVALID


def test_more_cycles_on_the_same_context():
    """A call asking for more cycles than the last one grows the trace buffer;
    the captured cycle must follow it: the trace equals a fresh context's."""
    case = synth.mri_case(48, 40, 11, accel=3.0, sigma=0.01)
    kd, md = dev_case(case)
    ctx = cm.Context(0)
    cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=1, ctx=ctx)
    u1, t1 = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=4, ctx=ctx)
    u1 = u1.clone()
    u2, t2 = cm.cm_recon(kd, md, 0.02, cm.MEAN, cycles=4, ctx=cm.Context(0))
    torch.cuda.synchronize()
    assert np.all(np.isfinite(t1)) and np.all(t1 > 0)
    assert np.array_equal(t1, t2) and torch.equal(u1, u2)


# ---------------------------------------------------------------------------
# CT: A = R, the parallel-beam Radon transform.

def ct_case(H, W, n, sigma, seed):
    clean = synth.piecewise_image(H, W, seed, 6, 0.0).clean.astype(np.float64)
    rng = np.random.default_rng(seed)
    sino = recon.radon_forward(clean, n)
    sino = sino + sigma * rng.normal(size=sino.shape)
    return clean, sino.astype(np.float32)


def test_radon_pair_matches_oracle_and_is_adjoint():
    H, W, n = 33, 40, 17
    rng = np.random.default_rng(8)
    u = rng.random((H, W), dtype=np.float32)
    y = rng.normal(size=(n, cm.cm_radon_bins(H, W))).astype(np.float32)
    assert cm.cm_radon_bins(H, W) == recon.radon_geometry(H, W, n)[0]
    Ru = cm.cm_radon(torch.from_numpy(u).cuda(), n).cpu().numpy()
    Rty = cm.cm_radon_adjoint(torch.from_numpy(y).cuda(), H, W).cpu().numpy()
    Ru_o = recon.radon_forward(u.astype(np.float64), n)
    Rty_o = recon.radon_adjoint(y.astype(np.float64), H, W)
    assert np.max(np.abs(Ru - Ru_o)) <= 1e-4 * np.max(np.abs(Ru_o))
    assert np.max(np.abs(Rty - Rty_o)) <= 1e-4 * np.max(np.abs(Rty_o))
    lhs = np.sum(Ru.astype(np.float64) * y)
    rhs = np.sum(u.astype(np.float64) * Rty)
    assert lhs == pytest.approx(rhs, rel=1e-5)


@pytest.mark.parametrize("shape", [(48, 48), (37, 52)])
def test_ct_start_and_finest_cycle_match_oracle(shape):
    H, W = shape
    clean, sino = ct_case(H, W, 45, 0.1, 3 + H)
    sd = torch.from_numpy(sino).cuda()
    u0, t0 = cm.cm_recon_ct(sd, H, W, 1.0, cm.MEAN, cycles=0)
    fbp = recon.fbp(sino.astype(np.float64), H, W)
    assert np.max(np.abs(u0.cpu().numpy() - fbp)) < 1e-3
    u, tr = cm.cm_recon_ct(sd, H, W, 1.0, cm.MEAN, levels=1, cycles=1, cg_iters=8)
    torch.cuda.synchronize()
    uo, tro = recon.solve_ct(sino.astype(np.float64), H, W, 1.0, cm.MEAN, levels=1, cycles=1,
                             cg_iters=8)
    assert np.max(np.abs(u.cpu().numpy() - uo)) < 2e-3
    np.testing.assert_allclose(tr, tro, rtol=1e-3)


def test_ct_full_cycles_match_oracle_and_improve_on_fbp():
    H = W = 48
    clean, sino = ct_case(H, W, 45, 0.1, 21)
    sd = torch.from_numpy(sino).cuda()
    u, tr = cm.cm_recon_ct(sd, H, W, 1.0, cm.MEAN, cycles=3, cg_iters=8)
    torch.cuda.synchronize()
    uo, tro = recon.solve_ct(sino.astype(np.float64), H, W, 1.0, cm.MEAN, cycles=3, cg_iters=8)
    np.testing.assert_allclose(tr, tro, rtol=2e-3)
    ug = u.cpu().numpy()
    assert np.max(np.abs(ug - uo)) < 5e-3
    assert np.all(np.diff(tr) < 0)
    fbp = recon.fbp(sino.astype(np.float64), H, W)
    assert synth.psnr(ug, clean) > synth.psnr(fbp, clean) + 0.3
