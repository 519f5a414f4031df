"""Seeded synthetic inputs for the SE(2,N) inpainting path.

The paper's test images are not available, so every input here is synthesised
from a seed, with the shapes and corruption structure of the paper's workloads
(256x256 grey images corrupted by bars of width 3-10 px over 37-69 % of the
pixels, Table 1 of the paper) scaled to the sizes of the benchmark
configurations.

This module holds no arithmetic of the method itself (no lift, transform,
diffusion, restoration or projection): only image and mask synthesis, random
volumes, and the parameter sets of each workload. Both the CPU oracle tests
and the CUDA path tests draw their inputs from here.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy import ndimage

__all__ = [
    "Workload",
    "lines_circles_image",
    "curves_noise_image",
    "lines_patches_image",
    "bernoulli_mask",
    "bar_mask",
    "workload_small",
    "workload_512",
    "workload_batch",
    "workload_2048",
    "random_volume",
    "random_real_volume",
]


@dataclasses.dataclass
class Workload:
    """One inpainting problem: the clean image, the known-pixel mask and the
    method parameters (canonical pixel units: dpsi_r/dt = -a_r^2 psi_r +
    beta * (psi_{r+1} - 2 psi_r + psi_{r-1}))."""

    name: str
    clean: np.ndarray          # [H][W] float64 in [0.05, 1]
    mask: np.ndarray           # [H][W] uint8, 1 = known (good set G), 0 = corrupted (B)
    N: int
    beta: float
    T: float                   # total diffusion time over all rounds
    steps: int                 # Crank-Nicolson steps per round
    rounds: int                # number of restoration intervals (the paper's n)
    eps: float = 0.5           # restoration strength (every row of Table 1 uses 0.5)
    sigma: float = 1.0         # Gaussian smoothing of the lift, in pixels

    @property
    def f(self) -> np.ndarray:
        """Corrupted input: zero on B, as the paper assumes."""
        return self.clean * (self.mask != 0)

    @property
    def H(self) -> int:
        return self.clean.shape[0]

    @property
    def W(self) -> int:
        return self.clean.shape[1]

    def updates(self) -> int:
        """Mathieu updates of the whole inpaint: frequencies x angles x steps x rounds."""
        return self.H * self.W * self.N * self.steps * self.rounds


# ----------------------------------------------------------------------------
# drawing primitives (anti-aliased by a clipped distance ramp)
# ----------------------------------------------------------------------------

def _draw_segment(img, p0, p1, width, value):
    """Max-composite an anti-aliased segment of the given width into img."""
    H, W = img.shape
    r = width / 2.0 + 1.0
    x0, x1 = sorted((p0[0], p1[0]))
    y0, y1 = sorted((p0[1], p1[1]))
    xa, xb = max(int(np.floor(x0 - r)), 0), min(int(np.ceil(x1 + r)) + 1, W)
    ya, yb = max(int(np.floor(y0 - r)), 0), min(int(np.ceil(y1 + r)) + 1, H)
    if xa >= xb or ya >= yb:
        return
    yy, xx = np.mgrid[ya:yb, xa:xb].astype(np.float64)
    dx, dy = p1[0] - p0[0], p1[1] - p0[1]
    L2 = dx * dx + dy * dy
    if L2 == 0.0:
        t = np.zeros_like(xx)
    else:
        t = np.clip(((xx - p0[0]) * dx + (yy - p0[1]) * dy) / L2, 0.0, 1.0)
    d = np.hypot(xx - (p0[0] + t * dx), yy - (p0[1] + t * dy))
    cov = np.clip(width / 2.0 + 0.5 - d, 0.0, 1.0)
    sub = img[ya:yb, xa:xb]
    np.maximum(sub, value * cov, out=sub)


def _draw_circle(img, c, radius, width, filled, value):
    H, W = img.shape
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    d = np.hypot(xx - c[0], yy - c[1])
    if filled:
        cov = np.clip(radius + 0.5 - d, 0.0, 1.0)
    else:
        cov = np.clip(width / 2.0 + 0.5 - np.abs(d - radius), 0.0, 1.0)
    np.maximum(img, value * cov, out=img)


def _draw_quad_bezier(img, p0, p1, p2, width, value, pieces=24):
    t = np.linspace(0.0, 1.0, pieces + 1)
    pts = ((1 - t) ** 2)[:, None] * p0 + (2 * (1 - t) * t)[:, None] * p1 + (t ** 2)[:, None] * p2
    for a, b in zip(pts[:-1], pts[1:]):
        _draw_segment(img, a, b, width, value)


# ----------------------------------------------------------------------------
# images
# ----------------------------------------------------------------------------

def lines_circles_image(H, W, seed, n_lines=6, n_circles=3, background=0.05):
    """Anti-aliased random lines (width 1-3 px, intensity U[0.2,1]) and circles
    (radius 4-20 px, filled or outlined) on a constant background, clipped to
    [0.05, 1], float64."""
    rng = np.random.default_rng(seed)
    img = np.full((H, W), background, dtype=np.float64)
    for _ in range(n_lines):
        p0 = rng.uniform([0, 0], [W - 1, H - 1])
        p1 = rng.uniform([0, 0], [W - 1, H - 1])
        width = rng.uniform(1.0, 3.0)
        value = rng.uniform(0.2, 1.0)
        _draw_segment(img, p0, p1, width, value)
    for _ in range(n_circles):
        radius = rng.uniform(4.0, min(20.0, 0.45 * min(H, W)))
        c = rng.uniform([radius, radius], [W - 1 - radius, H - 1 - radius])
        filled = bool(rng.integers(0, 2))
        width = rng.uniform(1.0, 3.0)
        value = rng.uniform(0.2, 1.0)
        _draw_circle(img, c, radius, width, filled, value)
    return np.clip(img, 0.05, 1.0)


def curves_noise_image(H, W, seed, n_curves=40, noise_sigma=8.0, noise_amp=0.1):
    """Piecewise-smooth image: random lines and quadratic Bezier curves plus
    Gaussian-smoothed noise (sigma 8 px, amplitude 0.1), mapped into [0.05, 1]."""
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), dtype=np.float64)
    span = np.array([W - 1, H - 1], dtype=np.float64)
    for i in range(n_curves):
        width = rng.uniform(1.0, 4.0)
        value = rng.uniform(0.3, 1.0)
        if i % 2 == 0:
            _draw_segment(img, rng.uniform(0, 1, 2) * span, rng.uniform(0, 1, 2) * span, width, value)
        else:
            p0, p1, p2 = (rng.uniform(0, 1, 2) * span for _ in range(3))
            _draw_quad_bezier(img, p0, p1, p2, width, value)
    noise = ndimage.gaussian_filter(rng.standard_normal((H, W)), noise_sigma, mode="wrap")
    noise *= noise_amp / max(np.abs(noise).max(), 1e-300)
    img = img + noise
    lo, hi = img.min(), img.max()
    return 0.05 + 0.95 * (img - lo) / (hi - lo)


def lines_patches_image(H, W, seed, n_lines=60, n_patches=24, patch_radius=32.0):
    """Lines plus textured patches (band-limited noise inside 64-px discs),
    mapped into [0.05, 1]."""
    rng = np.random.default_rng(seed)
    img = np.zeros((H, W), dtype=np.float64)
    span = np.array([W - 1, H - 1], dtype=np.float64)
    for _ in range(n_lines):
        _draw_segment(img, rng.uniform(0, 1, 2) * span, rng.uniform(0, 1, 2) * span,
                      rng.uniform(1.0, 5.0), rng.uniform(0.3, 1.0))
    white = rng.standard_normal((H, W))
    band = ndimage.gaussian_filter(white, 1.5, mode="wrap") - ndimage.gaussian_filter(white, 4.0, mode="wrap")
    band /= max(np.abs(band).max(), 1e-300)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(n_patches):
        c = rng.uniform(0, 1, 2) * span
        inside = np.hypot(xx - c[0], yy - c[1]) <= patch_radius
        img[inside] = np.maximum(img[inside], 0.5 + 0.4 * band[inside])
    lo, hi = img.min(), img.max()
    return 0.05 + 0.95 * (img - lo) / (hi - lo)


# ----------------------------------------------------------------------------
# masks (1 = known pixel, 0 = corrupted)
# ----------------------------------------------------------------------------

def bernoulli_mask(H, W, seed, corrupted_fraction):
    rng = np.random.default_rng(seed)
    return (rng.random((H, W)) >= corrupted_fraction).astype(np.uint8)


def bar_mask(H, W, width, period):
    """Horizontal and vertical occluding bars: 0 on the bars, 1 elsewhere."""
    y = np.arange(H)[:, None]
    x = np.arange(W)[None, :]
    bars = ((y % period) < width) | ((x % period) < width)
    return (~bars).astype(np.uint8)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def workload_small(H=64, W=64, seed=1, mask_seed=101):
    """64x64 lines-and-circles image, 50 % of the pixels masked at random,
    N=16, beta=0.5, T=1 in 100 Crank-Nicolson steps, one round."""
    clean = lines_circles_image(H, W, seed)
    mask = bernoulli_mask(H, W, mask_seed, 0.5)
    return Workload("lines_circles_64_N16", clean, mask, N=16, beta=0.5, T=1.0, steps=100, rounds=1)


def workload_512(H=512, W=512, seed=2, steps=500, rounds=10, N=32):
    """512x512 piecewise-smooth image, 80 % random mask OR 4-px bars every
    32 px, N=32, beta=0.25, 500 steps per round, 10 rounds, T=2 per round."""
    clean = curves_noise_image(H, W, seed)
    rnd = bernoulli_mask(H, W, seed + 1000, 0.8)
    mask = (rnd & bar_mask(H, W, 4, 32)).astype(np.uint8)
    return Workload(f"curves_noise_{H}_N{N}", clean, mask, N=N, beta=0.25,
                    T=2.0 * rounds, steps=steps, rounds=rounds)


def workload_batch(count=256, seed=3, sides=(128, 256, 384, 512, 768, 1024), Ns=(16, 32, 64)):
    """Uneven batch: side lengths and N drawn uniformly, mask density U[0.6,0.9]
    (corrupted fraction), the 512x512 generator, beta=0.25, T=2, 100 steps, one round."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.choice(sides))
        N = int(rng.choice(Ns))
        dens = float(rng.uniform(0.6, 0.9))
        clean = curves_noise_image(side, side, seed * 100000 + i, n_curves=max(8, side // 16))
        mask = bernoulli_mask(side, side, seed * 100000 + 50000 + i, dens)
        out.append(Workload(f"batch{i}_{side}_N{N}", clean, mask, N=N, beta=0.25, T=2.0, steps=100, rounds=1))
    return out


def workload_2048(stress=False, seed=4, side=2048):
    """2048x2048 lines-plus-texture image, N=64, 85 % of the pixels masked,
    1000 fused steps. Main run: beta=0.25, T=50 (dt=0.05); stress run:
    beta=10, dt=1, so beta*dt=10. `side` draws the same recipe on a smaller
    square image (for profiling a smaller case)."""
    H = W = side
    clean = lines_patches_image(H, W, seed)
    mask = bernoulli_mask(H, W, seed + 1000, 0.85)
    if stress:
        return Workload(f"lines_patches_{side}_N64_stress", clean, mask, N=64, beta=10.0, T=1000.0, steps=1000,
                        rounds=1)
    return Workload(f"lines_patches_{side}_N64", clean, mask, N=64, beta=0.25, T=50.0, steps=1000, rounds=1)


# the surrogate's data: the 64x64 generator at 256x256, half of the pixels
# corrupted; training seeds 10000..29999, validation seeds 30000..30511
SURROGATE_SIDE = 256
SURROGATE_TRAIN_SEEDS = (10000, 20000)   # first seed, count
SURROGATE_VAL_SEEDS = (30000, 512)


def surrogate_example(seed, H=SURROGATE_SIDE, W=SURROGATE_SIDE):
    """(clean, mask) of one surrogate example: the lines-and-circles image at
    this seed and a 50 % random mask drawn from seed + 1_000_000."""
    return lines_circles_image(H, W, seed), bernoulli_mask(H, W, seed + 1_000_000, 0.5)


def surrogate_examples(first, count, H=SURROGATE_SIDE, W=SURROGATE_SIDE):
    """Stacked (clean float32 [count][H][W], mask uint8 [count][H][W]) for
    seeds first .. first + count - 1."""
    clean = np.empty((count, H, W), np.float32)
    mask = np.empty((count, H, W), np.uint8)
    for i in range(count):
        c, m = surrogate_example(first + i, H, W)
        clean[i] = c
        mask[i] = m
    return clean, mask


def surrogate_method_params():
    """Method parameters the surrogate's targets are made with: N=32 and the
    64x64 workload's beta=0.5, T=1 in 100 steps, one round."""
    return dict(N=32, beta=0.5, T=1.0, steps=100, rounds=1)


def random_volume(N, H, W, seed, dtype=np.complex128):
    """Random complex volume [N][H][W] with unit-variance Gaussian parts
    (drawn directly in float32 when dtype is complex64, to keep large
    volumes cheap)."""
    rng = np.random.default_rng(seed)
    if np.dtype(dtype) == np.complex64:
        v = np.empty((N, H, W), np.complex64)
        v.real = rng.standard_normal((N, H, W), dtype=np.float32)
        v.imag = rng.standard_normal((N, H, W), dtype=np.float32)
        return v
    v = rng.standard_normal((N, H, W)) + 1j * rng.standard_normal((N, H, W))
    return v.astype(dtype)


def random_real_volume(N, H, W, seed):
    """Random real volume [N][H][W] with entries U[0,1) (float64)."""
    rng = np.random.default_rng(seed)
    return rng.random((N, H, W))
