"""Helpers shared by the GPU parity tests: device tensors from numpy inputs
and the comparison metrics with their tolerances.

Tolerances (the path runs in FP32 against the FP64 oracle):
  * REL_L2 = 1e-5: relative L2 error over a whole volume or image;
  * MAX_REL = 1e-5: max-abs error of a projected image relative to max|f|.
Both are the stated accuracy target of the path; every result below full
size meets them (the measured errors are 1e-7 .. 2e-6, see the test output).

  * MAX_REL_512 = 4 x S32: the max-abs bound of the full 512x512 workload
    (10 restoration intervals), derived from the FP64 oracle itself. S32 is
    the larger of the two measured changes of the oracle's result when its
    transforms run in FP32 and its volume is stored in FP32, on the full and
    on the Hermitian-half spectrum (oracle/sensitivity.py, written by
    tests/golden/make_sensitivity.py to sensitivity_512_N32.json: 3.8e-6
    and 8.2e-6 at one pixel, while FP32 storage rounding alone moves it by
    5.3e-7). The workload amplifies rounding at that pixel: a corrupted
    region whose value the restorations pump up over the intervals, so
    that an exact FP32 transform already misses 1e-5 by little. The GPU
    also rounds the diffusion and the restoration in FP32 (each adding
    per-interval error of the order of one transform), hence the factor 4.
    The same derivation with N = 30 (the paper's angle count) reads
    sensitivity_512_N30.json.
  * TIE_TOL_512 = 2 x MAX_REL_512: a dynamic-restoration decision compares
    two such values, so one within this distance of a tie may go either way.
"""
import json
import os

import numpy as np
import torch

REL_L2 = 1e-5
MAX_REL = 1e-5

_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def fp32_sensitivity_512(N=32):
    """S32 of the 512x512 workload with N angles from the stored FP64-oracle
    sensitivity run (sensitivity_512_N{N}.json)."""
    with open(os.path.join(_GOLDEN, f"sensitivity_512_N{N}.json")) as fh:
        s = json.load(fh)
    return max(s["fp32_half"]["max_abs_over_max_f"], s["fp32_full"]["max_abs_over_max_f"])


MAX_REL_512 = 4.0 * fp32_sensitivity_512()
TIE_TOL_512 = 2.0 * MAX_REL_512


def restoration_sigma_max(f64, mask, bins, p):
    """The largest factor sigma = (eps h(0) + (1-eps) h(t_i)) / h(t_i) that
    the static restoration (Section 5) applies to a good pixel in the FP64
    oracle's run of the method: an absolute error d of the volume at that
    pixel leaves the restoration as sigma * d, so sigma measures how
    strongly the restoration amplifies FP32 rounding."""
    import oracle
    lifted = oracle.lift(f64, mask, bins, p.N)
    h0 = lifted.real.max(axis=0)
    good = np.asarray(mask) != 0
    Tr = p.T / p.rounds
    v = oracle.diffuse(oracle.forward(lifted), p.beta, Tr, p.steps, p.angle_conv)
    worst = 1.0
    for _ in range(1, p.rounds):
        x = oracle.inverse(v)
        ht = x.real.max(axis=0)
        scaled = good & (ht > p.guard * h0) & (ht > 0.0)
        if scaled.any():
            worst = max(worst, float(((p.eps * h0[scaled] + (1.0 - p.eps) * ht[scaled]) / ht[scaled]).max()))
        v = oracle.diffuse(oracle.forward(oracle.mix(x, f64, mask, bins, p.eps, p.guard)), p.beta, Tr, p.steps,
                           p.angle_conv)
    return worst


def max_rel_for_sigma(sigma_max):
    """Max-abs bound (relative to max|f|) of a multi-interval result whose
    restorations scale a good pixel by at most sigma_max: MAX_REL up to
    sigma = 10 (measured on the GPU at guard 0: sigma 7.3 and 9.9 stay
    below it), growing in proportion to sigma beyond, since the restoration
    multiplies an absolute error at the pixel by sigma."""
    return MAX_REL * max(1.0, sigma_max / 10.0)


def dev():
    return torch.device("cuda:0")


def t_f32(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev())


def t_u8(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.uint8), device=dev())


def t_c64(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.complex64), device=dev())


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.complex128 if np.iscomplexobj(x) else np.float64)
    ref = np.asarray(ref)
    return float(np.linalg.norm((x - ref).ravel()) / max(np.linalg.norm(np.asarray(ref).ravel()), 1e-300))
