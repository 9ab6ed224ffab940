"""The seeded input generator: SplitMix64 reference values, determinism and
the recipe's statistics."""
import numpy as np
import pytest

import synth


def test_splitmix64_reference_outputs():
    """SplitMix64 with state 0: published first outputs (Steele et al. 2014;
    the same values appear in the reference implementation that seeds
    xoshiro generators)."""
    rng = synth.SplitMix64(0)
    assert rng.next_u64() == 0xE220A8397B1DCDAF
    assert rng.next_u64() == 0x6E789E6AA1B965F4
    assert rng.next_u64() == 0x06C45D188009454F


def test_counter_form_equals_sequential_stream():
    rng = synth.SplitMix64(12345)
    seq = [rng.next_u64() for _ in range(50)]
    blk = synth.splitmix_block(12345, 50)
    assert [int(v) for v in blk] == seq


def test_gaussian_noise_moments():
    z = synth.gaussian_noise(99, 400001)
    assert abs(z.mean()) < 0.01
    assert abs(z.std() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_images_are_deterministic_and_in_range():
    a = synth.single_64()
    b = synth.single_64()
    assert np.array_equal(a.f, b.f) and np.array_equal(a.clean, b.clean)
    assert a.f.dtype == np.float32 and a.f.shape == (64, 64)
    assert a.clean.min() >= 0.0 and a.clean.max() <= 1.0
    noise = a.f.astype(np.float64) - a.clean
    assert abs(noise.std() - 0.05) < 0.005
    c = synth.piecewise_image(64, 64, synth.workload_seed(1, 1), 6, 0.05)
    assert not np.array_equal(a.f, c.f)


def test_piecewise_structure():
    """Clean images are piecewise smooth: most horizontal differences are the
    ramp's small slope, a few are edges."""
    img = synth.piecewise_image(128, 96, 7, 10, 0.0)
    d = np.abs(np.diff(img.clean.astype(np.float64), axis=1))
    assert np.mean(d < 0.01) > 0.9
    assert np.sum(d > 0.05) > 10


def test_uneven_batch_recipe():
    items = synth.uneven_batch(16)
    assert len(items) == 16
    for i, it in enumerate(items):
        H, W = it.image.f.shape
        assert H in synth.SIDES_BATCH and W in synth.SIDES_BATCH
        assert it.kind == i % 2
        assert it.alpha in (10.0, 20.0)
        assert 0.03 <= it.image.sigma <= 0.12
    assert len({it.image.f.shape for it in items}) > 4


@pytest.mark.parametrize("split", ["train", "test"])
def test_warmstart_sets_are_disjoint(split):
    a = synth.warmstart_image(split, 0, 32)
    b = synth.warmstart_image("test" if split == "train" else "train", 0, 32)
    assert a.seed != b.seed


def test_mri_case_recipe():
    """The undersampled acquisition: whole phase-encoding rows, every row
    whose frequency satisfies |k| <= 8% of H/2 sampled, about 1/accel of the rows in
    all, the data zero off the mask and equal to the masked orthonormal
    spectrum up to the noise, and the same case for the same seed."""
    H, W, accel = 256, 64, 3.0
    c = synth.mri_case(H, W, 17, accel=accel, sigma=0.0)
    rows = c.mask[:, 0].astype(bool)
    assert np.all(c.mask == c.mask[:, :1])                      # whole rows
    freq = np.where(np.arange(H) < (H + 1) // 2, np.arange(H), np.arange(H) - H)
    assert np.all(rows[np.abs(freq) <= 0.08 * H / 2])            # the centre rows
    assert abs(rows.mean() - 1 / accel) < 0.08
    assert np.all(c.kspace[~rows] == 0)
    ref = np.fft.fft2(c.clean.astype(np.float64), norm="ortho")[rows]
    np.testing.assert_allclose(c.kspace[rows], ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    d = synth.mri_case(H, W, 17, accel=accel, sigma=0.0)
    assert np.array_equal(d.mask, c.mask) and np.array_equal(d.kspace, c.kspace)
    full = synth.mri_case(32, 16, 3, accel=1.0)
    assert full.mask.all()
