"""Seeded synthetic workloads shared by the oracle tests and the CUDA path.

This module only draws input data.  It holds none of the method's
arithmetic (no curvature, no energy, no block search), so both sides of a
parity test may use it without sharing any part of the method.

The paper measures on natural photographs ('Triangle', 'Peppers', 'Parrot',
'Man' and a 30-image set, Sec. 4) that are not available here; these images
stand in for them.  Each clean image is a linear intensity ramp with a number
of constant-intensity disks and axis-aligned rectangles painted over it, so it
is piecewise smooth with sharp edges and corners, the structure curvature
regularisation is meant to keep (Sec. 1).  The noisy observation adds i.i.d.
Gaussian noise (Sec. 4 corrupts its test images with zero-mean white Gaussian
noise) without clipping.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) and Gaussian variates from the
Box-Muller transform.  The i-th SplitMix64 output from state ``s`` is
``mix(s + (i + 1) * GAMMA)``, so the per-pixel noise stream is evaluated
counter-style with numpy and equals the sequential stream bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1
# Base seed of the synthetic workloads: image i of workload k uses
# BASE_SEED + 1000 * k + i.
BASE_SEED = 2204079210


def _mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


class SplitMix64:
    """Sequential SplitMix64 stream."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return _mix64(self.state)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform on [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def choice(self, values):
        return values[int(self.uniform() * len(values)) % len(values)]


def splitmix_block(state: int, n: int) -> np.ndarray:
    """Outputs 0..n-1 of the SplitMix64 stream that starts at ``state``."""
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & MASK64) + idx * np.uint64(GAMMA)
    return _mix64_np(z)


def gaussian_noise(seed: int, n: int) -> np.ndarray:
    """n i.i.d. N(0, 1) variates (float64), Box-Muller on a SplitMix64 stream.

    Pair j uses outputs 2j and 2j+1: u1 = 1 - U(out_2j) in (0, 1],
    u2 = U(out_2j+1); the pair is (R cos 2 pi u2, R sin 2 pi u2) with
    R = sqrt(-2 ln u1).
    """
    npairs = (n + 1) // 2
    raw = splitmix_block(_mix64(seed ^ 0x6E6F697365), 2 * npairs)
    uni = (raw >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    u1 = 1.0 - uni[0::2]
    u2 = uni[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


@dataclass
class Image:
    f: np.ndarray       # noisy observation, float32, (H, W)
    clean: np.ndarray   # clean image, float32, (H, W)
    seed: int
    sigma: float


def piecewise_image(H: int, W: int, seed: int, n_shapes: int, sigma: float) -> Image:
    """One seeded piecewise-smooth image on [0, 1] plus Gaussian noise.

    Ramp: r0 + r1 * x / (W - 1) + r2 * y / (H - 1) with r0 ~ U(0.2, 0.6) and
    r1, r2 ~ U(-0.2, 0.2) (x = column, y = row; a one-pixel axis uses 0).
    Each shape is, with probability 1/2, a disk whose centre is uniform over
    the image and whose radius is U(0.04, 0.2) * min(H, W), or else an
    axis-aligned rectangle with uniform centre and sides U(0.08, 0.4) * W by
    U(0.08, 0.4) * H.  A shape replaces the intensity under it with its own
    constant U(0, 1); shapes are painted in order.
    """
    if H < 1 or W < 1:
        raise ValueError("image sides must be >= 1")
    rng = SplitMix64(seed)
    r0 = rng.uniform(0.2, 0.6)
    r1 = rng.uniform(-0.2, 0.2)
    r2 = rng.uniform(-0.2, 0.2)
    y = np.arange(H, dtype=np.float64)[:, None]
    x = np.arange(W, dtype=np.float64)[None, :]
    xs = x / (W - 1) if W > 1 else np.zeros_like(x)
    ys = y / (H - 1) if H > 1 else np.zeros_like(y)
    clean = r0 + r1 * xs + r2 * ys
    clean = np.broadcast_to(clean, (H, W)).copy()
    m = min(H, W)
    for _ in range(n_shapes):
        is_disk = rng.uniform() < 0.5
        if is_disk:
            cx = rng.uniform(0.0, W)
            cy = rng.uniform(0.0, H)
            rad = rng.uniform(0.04, 0.2) * m
            val = rng.uniform()
            mask = (x - cx) ** 2 + (y - cy) ** 2 <= rad * rad
        else:
            cx = rng.uniform(0.0, W)
            cy = rng.uniform(0.0, H)
            sw = rng.uniform(0.08, 0.4) * W
            sh = rng.uniform(0.08, 0.4) * H
            val = rng.uniform()
            mask = (np.abs(x - cx) <= 0.5 * sw) & (np.abs(y - cy) <= 0.5 * sh)
        clean[np.broadcast_to(mask, (H, W))] = val
    noise = gaussian_noise(seed, H * W).reshape(H, W)
    f = clean + sigma * noise
    return Image(f=f.astype(np.float32), clean=clean.astype(np.float32),
                 seed=seed, sigma=sigma)


def workload_seed(k: int, i: int) -> int:
    return BASE_SEED + 1000 * k + i


# ---------------------------------------------------------------------------
# The five synthetic workloads (single image, single image, large image,
# uneven batch, warm-start training/test sets).  Numbering k = 1..5.


def single_64(i: int = 0) -> Image:
    """64x64, 6 shapes, sigma 0.05 (mean curvature, alpha 20, 20 cycles)."""
    return piecewise_image(64, 64, workload_seed(1, i), 6, 0.05)


def single_512(i: int = 0) -> Image:
    """512x512, 20 shapes, sigma 0.1 (Gaussian curvature, alpha 15)."""
    return piecewise_image(512, 512, workload_seed(2, i), 20, 0.1)


def large(side: int, i: int = 0) -> Image:
    """side x side (1024 or 2048), 20 shapes, sigma 0.08 (mean, alpha 20)."""
    return piecewise_image(side, side, workload_seed(3, i), 20, 0.08)


SIDES_BATCH = tuple(range(128, 1025, 64))   # 128, 192, ..., 1024 (15 values)


@dataclass
class BatchItem:
    image: Image
    alpha: float
    kind: int   # 0 mean, 1 Gaussian


def uneven_batch(n: int = 64, sides=SIDES_BATCH) -> list[BatchItem]:
    """n images with independently drawn H and W from ``sides``, kind i mod 2,
    sigma ~ U(0.03, 0.12), alpha in {10, 20} by a fair coin, 20 shapes."""
    items = []
    for i in range(n):
        seed = workload_seed(4, i)
        rng = SplitMix64(_mix64(seed ^ 0x6261746368))
        H = rng.choice(sides)
        W = rng.choice(sides)
        sigma = rng.uniform(0.03, 0.12)
        alpha = 10.0 if rng.uniform() < 0.5 else 20.0
        items.append(BatchItem(piecewise_image(H, W, seed, 20, sigma), alpha, i % 2))
    return items


def warmstart_image(split: str, i: int, side: int) -> Image:
    """Warm-start data: 'train' images (256x256) and 'test' images
    (1024x1024) from disjoint seed ranges; sigma ~ U(0.03, 0.12), 20 shapes."""
    if split not in ("train", "test"):
        raise ValueError(split)
    seed = workload_seed(5, i + (0 if split == "train" else 500000))
    rng = SplitMix64(_mix64(seed ^ 0x7761726D))
    sigma = rng.uniform(0.03, 0.12)
    return piecewise_image(side, side, seed, 20, sigma)


def psnr(u: np.ndarray, clean: np.ndarray) -> float:
    """10 log10(1 / MSE) for images on [0, 1]."""
    mse = float(np.mean((np.asarray(u, np.float64) - np.asarray(clean, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(1.0 / mse)


# ---------------------------------------------------------------------------
# MRI-like reconstruction inputs (Sec. 5; the paper's MRI data are not
# available here).

@dataclass
class MriCase:
    clean: np.ndarray    # phantom, float32 (H, W)
    mask: np.ndarray     # sampled k-space rows, uint8 (H, W), 0 or 1
    kspace: np.ndarray   # observed data b, complex64 (H, W), zero off the mask
    seed: int
    sigma: float


def mri_case(H: int, W: int, seed: int, accel: float = 3.0, centre: float = 0.08,
             sigma: float = 0.01, n_shapes: int = 12) -> MriCase:
    """A seeded undersampled-acquisition case.

    Phantom: the clean image of piecewise_image(H, W, seed, n_shapes, 0).
    Mask: Cartesian phase-encoding rows of the unshifted 2-D spectrum; every
    row whose signed frequency |k| (k = i for i < H/2, else i - H) is at most
    centre * H / 2 is sampled, every other row with the probability that
    makes the expected sampled fraction 1 / accel (SplitMix64 uniforms).
    Data: b = mask * (F clean + sigma (n1 + i n2)), F the orthonormal 2-D DFT
    (numpy.fft.fft2 with norm="ortho"), n1, n2 i.i.d. N(0, 1).  This only
    simulates the acquisition; the reconstruction applies its own operator.
    """
    clean = piecewise_image(H, W, seed, n_shapes, 0.0).clean.astype(np.float64)
    rng = SplitMix64(_mix64(seed ^ 0x6D7269))
    freq = np.where(np.arange(H) < (H + 1) // 2, np.arange(H), np.arange(H) - H)
    low = np.abs(freq) <= centre * H / 2
    n_low = int(low.sum())
    p = min(1.0, max(0.0, (H / accel - n_low) / max(H - n_low, 1)))
    rows = low.copy()
    for i in range(H):
        u = rng.uniform()
        if not low[i] and u < p:
            rows[i] = True
    mask = np.broadcast_to(rows[:, None], (H, W)).astype(np.uint8)
    g = gaussian_noise(_mix64(seed ^ 0x6B7370), 2 * H * W)
    noise = g[0::2].reshape(H, W) + 1j * g[1::2].reshape(H, W)
    data = mask * (np.fft.fft2(clean, norm="ortho") + sigma * noise)
    return MriCase(clean=clean.astype(np.float32), mask=mask,
                   kspace=data.astype(np.complex64), seed=seed, sigma=sigma)
