"""FP32 rounding injected into the FP64 oracle's method: how far any FP32
implementation of the method must be expected to move the FP64 result.

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only the tests and the
scripts that write stored values under tests/golden/ use it.

The method runs stage by stage exactly as oracle.inpaint does (lift, 2-D DFT,
Crank-Nicolson diffusion of every frequency, inverse DFT, static
restoration, projection; Sections 1.2.4, 4 and 5), with one kind of
rounding injected:

* "none"     -- nothing (with half=True this is the same method on the
                Hermitian half of the spectrum, equal to oracle.inpaint up
                to FP64 rounding: the lifted volume is real, so the system of
                frequency (-k, -l) is the conjugate of that of (k, l));
* "storage"  -- the volume rounded to FP32 wherever an implementation keeps
                it in memory between two stages;
* "perturb"  -- every stored value multiplied by 1 + 2^-24 or 1 - 2^-24 at
                random (one unit of FP32 rounding, without its correlation);
* "fp32"     -- storage rounding, and the 2-D transforms computed in single
                precision (scipy.fft on float32 / complex64 data, the
                library's own FP32 arithmetic).

The diffusion itself always runs in FP64 (the C core), so "fp32" measures
what FP32 transforms and storage alone do to the result: a floor for an
implementation that also rounds the diffusion and the restoration in FP32.
"""
from __future__ import annotations

import numpy as np

from . import Params, diffuse, forward, inverse, lift, mix, orient, project

MODES = ("none", "storage", "perturb", "fp32")


def inpaint_rounded(f, mask, p: Params, bins=None, mode="storage", half=True, seed=0, nthreads=0):
    """The whole method (static restoration, max or mean projection) with
    the rounding `mode` injected; half=True integrates the H (W/2 + 1)
    frequencies l <= W/2 with real-to-complex transforms, half=False all
    H W with complex ones. Returns the projected image (float64)."""
    if mode not in MODES:
        raise ValueError(f"mode must be one of {MODES}")
    if p.dynamic or p.final_mix or p.reinject:
        raise ValueError("static restoration between intervals only")
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    if bins is None:
        bins = orient(f, mask, p.N, p.sigma, p.angle_conv, p.flat_tol)["bins"]
    rng = np.random.default_rng(seed)
    Wc = W // 2 + 1

    def st(v):
        if mode == "none":
            return v
        if mode == "perturb":
            u = 2.0 ** -24
            if np.iscomplexobj(v):
                return (v.real * (1 + u * rng.choice((-1.0, 1.0), v.shape))
                        + 1j * v.imag * (1 + u * rng.choice((-1.0, 1.0), v.shape)))
            return v * (1 + u * rng.choice((-1.0, 1.0), v.shape))
        if np.iscomplexobj(v):
            return v.astype(np.complex64).astype(np.complex128)
        return v.astype(np.float32).astype(np.float64)

    def fwd(x):
        if mode == "fp32":
            import scipy.fft as sf
            if half:
                return sf.rfft2(x.real.astype(np.float32), axes=(1, 2)).astype(np.complex128)
            return sf.fft2(x.astype(np.complex64), axes=(1, 2)).astype(np.complex128)
        return np.fft.rfft2(x.real, axes=(1, 2)) if half else forward(x)

    def inv(s):
        if mode == "fp32":
            import scipy.fft as sf
            if half:
                return sf.irfft2(s.astype(np.complex64), s=(H, W), axes=(1, 2)).astype(np.complex128)
            return sf.ifft2(s.astype(np.complex64), axes=(1, 2)).astype(np.complex128)
        return np.fft.irfft2(s, s=(H, W), axes=(1, 2)).astype(np.complex128) if half else inverse(s)

    if half:
        kk, ll = np.meshgrid(np.arange(H), np.arange(Wc), indexing="ij")
        freqs = (kk * W + ll).ravel()

    def dif(s):
        Tr = p.T / p.rounds
        if not half:
            return diffuse(s, p.beta, Tr, p.steps, p.angle_conv, nthreads=nthreads)
        full = np.zeros((p.N, H, W), np.complex128)
        full[:, :, :Wc] = s
        full = diffuse(full, p.beta, Tr, p.steps, p.angle_conv, freqs=freqs, nthreads=nthreads)
        return full[:, :, :Wc]

    v = st(dif(st(fwd(st(lift(f, mask, bins, p.N))))))
    for _ in range(1, p.rounds):
        x = st(inv(v))
        x = st(mix(x, f, mask, bins, p.eps, p.guard))
        v = st(dif(st(fwd(x))))
    return project(st(inv(v)), p.proj)
