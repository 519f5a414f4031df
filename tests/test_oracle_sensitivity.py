"""Pins of oracle/sensitivity.py (the FP64 method with FP32 rounding
injected) and of the bounds the GPU tests derive from its stored run.

The module must be the oracle's method exactly when nothing is rounded, on
both spectrum layouts (the Hermitian half integrates H (W/2 + 1) of the
frequencies and lets the inverse real transform rebuild the rest); each
rounding must move the result by an amount of the size FP32 arithmetic
explains; and the stored full-size run must hold the fields the tolerances
are computed from.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import sensitivity

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def case():
    w = synth.workload_512(H=48, W=64, steps=30, rounds=3)
    f = w.f.astype(np.float32).astype(np.float64)
    p = oracle.Params(N=16, beta=0.25, T=6.0, steps=30, rounds=3)
    bins = oracle.orient(f, w.mask, p.N)["bins"]
    ref = oracle.inpaint(f, w.mask, p, bins=bins)["out"]
    return w, f, p, bins, ref


@pytest.mark.parametrize("half", [True, False])
def test_no_rounding_is_the_oracle(case, half):
    w, f, p, bins, ref = case
    out = sensitivity.inpaint_rounded(f, w.mask, p, bins=bins, mode="none", half=half)
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("mode,lo,hi", [("storage", 1e-9, 2e-6), ("perturb", 1e-9, 2e-6), ("fp32", 1e-9, 2e-5)])
def test_roundings_move_the_result_by_fp32_amounts(case, mode, lo, hi):
    """One FP32 rounding of every stored value (relative 2^-24) moves a
    3-interval result by far less than 1e-5 but not by nothing; FP32
    transforms add the error of their own arithmetic."""
    w, f, p, bins, ref = case
    out = sensitivity.inpaint_rounded(f, w.mask, p, bins=bins, mode=mode, half=True)
    d = np.abs(out - ref).max() / np.abs(f).max()
    assert lo < d < hi, d


def test_storage_rounding_is_exactly_a_complex64_round_trip():
    """Planted check: with one interval and no transforms rounded, the
    storage mode equals rounding the lift, the spectrum after each stage and
    the volume before the projection; done by hand here on a tiny case."""
    w = synth.workload_small(16, 16)
    f = w.f.astype(np.float64)
    p = oracle.Params(N=8, beta=0.5, T=1.0, steps=10, rounds=1)
    bins = oracle.orient(f, w.mask, p.N)["bins"]
    r = lambda v: v.astype(np.complex64).astype(np.complex128)  # noqa: E731
    x = r(oracle.lift(f, w.mask, bins, p.N))
    s = r(np.fft.rfft2(x.real, axes=(1, 2)))
    full = np.zeros((p.N, 16, 16), np.complex128)
    full[:, :, :9] = s
    kk, ll = np.meshgrid(np.arange(16), np.arange(9), indexing="ij")
    s = r(oracle.diffuse(full, p.beta, p.T, p.steps, freqs=(kk * 16 + ll).ravel())[:, :, :9])
    expect = oracle.project(r(np.fft.irfft2(s, s=(16, 16), axes=(1, 2)).astype(np.complex128)))
    got = sensitivity.inpaint_rounded(f, w.mask, p, bins=bins, mode="storage", half=True)
    np.testing.assert_array_equal(got, expect)


def test_stored_full_size_sensitivity_and_derived_bounds():
    """The stored run on the 512x512 workload (make_sensitivity.py) and the
    bounds that tests/_gpu.py derives from it: MAX_REL_512 = 4 x S32 with S32
    the larger FP32-transform change, below 1e-4; the tie tolerance of
    dynamic restoration twice that; FP32 storage alone moves the result by
    far less than the transforms do."""
    with open(os.path.join(GOLDEN, "sensitivity_512_N32.json")) as fh:
        s = json.load(fh)
    for k in ("storage_full", "perturb_full", "fp32_full", "fp32_half"):
        assert 0.0 < s[k]["max_abs_over_max_f"] < 1e-4
        assert 0.0 < s[k]["rel_l2"] < 1e-5
    s32 = max(s["fp32_half"]["max_abs_over_max_f"], s["fp32_full"]["max_abs_over_max_f"])
    assert s["storage_full"]["max_abs_over_max_f"] < s32
    import _gpu
    assert _gpu.MAX_REL_512 == pytest.approx(4.0 * s32, rel=1e-12)
    assert _gpu.MAX_REL_512 < 1e-4
    assert _gpu.TIE_TOL_512 == pytest.approx(2.0 * _gpu.MAX_REL_512, rel=1e-12)
