"""GPU parity of the pixel-wise stages and transforms against the oracle,
through the C ABI: orientation (bins), lift, forward/inverse DFT, static
restoration, projection.

The orientation is a floating-point decision. The GPU takes it in FP32
from FP32 spectral gradients, the oracle in FP64; a pixel whose angle sits
within FP32 rounding of a bin boundary (or whose gradient sits within FP32
rounding of the flat threshold) may legitimately land on either side. Such
pixels are identified from the oracle's own margins with an FP32 error
model, the GPU must pick one of the valid candidates there, and must agree
exactly everywhere else.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import REL_L2, host, rel_l2, t_c64, t_f32, t_u8

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")

import torch  # noqa: E402

FP32_GRAD_ERR = 2e-5  # bound on |grad error| / max|grad| of the FP32 spectral gradient


def _gpu_bins(f32, mask, N, conv=0, sigma=1.0, flat_tol=1e-4):
    H, W = f32.shape
    plan = se2n.se2n_plan_create(H, W, N, conv)
    b = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    se2n.se2n_orient(plan, t_f32(f32), t_u8(mask), sigma, flat_tol, b)
    out = host(b)
    plan.close()
    return out


def _check_bins(got, o, N, flat_tol):
    """Exact agreement where the oracle's decision is far from a boundary
    (in units of the FP32 gradient error), a valid neighbouring choice
    elsewhere. Returns the fraction of pixels where the two differ."""
    rel = o["rel"]
    # angle uncertainty in bins: (N/pi) * (grad error / |grad|)
    ang = (N / np.pi) * FP32_GRAD_ERR / np.maximum(rel, 1e-30)
    ambiguous_flat = np.abs(rel - flat_tol) <= FP32_GRAD_ERR
    ambiguous_bin = (o["bins"] != oracle.BIN_FLAT) & (o["margin"] <= ang)
    sure = ~(ambiguous_flat | ambiguous_bin)
    np.testing.assert_array_equal(got[sure], o["bins"][sure])
    # elsewhere the GPU's bin must be one of the two nearest bins, or flat near the threshold
    u = o["phi"] * N / np.pi + 0.5
    lo = np.mod(np.floor(u - 0.5), N).astype(int)
    hi = np.mod(lo + 1, N)
    amb = ~sure
    ok = (got[amb] == lo[amb]) | (got[amb] == hi[amb]) | (got[amb] == o["bins"][amb])
    ok |= ambiguous_flat[amb] & (got[amb] == oracle.BIN_FLAT)
    assert ok.all()
    return (got != o["bins"]).mean(), amb.mean()


@pytest.mark.parametrize("maker,N", [(lambda: synth.workload_small(64, 64), 16),
                                     (lambda: synth.workload_512(), 32),
                                     (lambda: synth.workload_small(96, 128, seed=7), 8)])
def test_orientation_bins(maker, N):
    w = maker()
    f32 = w.f.astype(np.float32)
    o = oracle.orient(f32.astype(np.float64), w.mask, N)
    got = _gpu_bins(f32, w.mask, N)
    diff, amb = _check_bins(got, o, N, 1e-4)
    print(f"{w.H}x{w.W} N={N}: differing bins {diff:.2e}, near-tie pixels {amb:.2e}")
    assert diff < 1e-3


def test_orientation_flat_regions_and_2pi_convention():
    """A constant background with a few features: most pixels are flat."""
    H, W, N = 64, 64, 16
    f = synth.lines_circles_image(H, W, 3)
    mask = np.ones((H, W), np.uint8)
    f32 = f.astype(np.float32)
    o = oracle.orient(f32.astype(np.float64), mask, N, angle_conv=1)
    got = _gpu_bins(f32, mask, N, conv=1)
    assert (o["bins"] == oracle.BIN_FLAT).mean() > 0.1
    sure_flat = (o["bins"] == oracle.BIN_FLAT) & (o["rel"] < 1e-4 - FP32_GRAD_ERR)
    assert (got[sure_flat] == oracle.BIN_FLAT).all()
    # 2 pi / N grid: directions mod pi land on bins 0 .. N/2
    sure = (o["bins"] != oracle.BIN_FLAT) & (o["margin"] > 1e-2) & (o["rel"] > 1e-2)
    np.testing.assert_array_equal(got[sure], o["bins"][sure])
    assert got[got != oracle.BIN_FLAT].max() <= N // 2


def test_lift_is_exact():
    w = synth.workload_512()
    N = 32
    f32 = w.f.astype(np.float32)
    o = oracle.orient(f32.astype(np.float64), w.mask, N)
    rng = np.random.default_rng(0)
    bins = o["bins"].copy()
    bins[rng.random(bins.shape) < 0.01] = oracle.BIN_FLAT  # exercise the all-angle lift too
    plan = se2n.se2n_plan_create(w.H, w.W, N)
    vol = torch.full((N, w.H, w.W), 7.0, dtype=torch.complex64, device="cuda")
    se2n.se2n_lift(plan, t_f32(f32), t_u8(w.mask), t_u8(bins), vol)
    got = host(vol)
    plan.close()
    ref = oracle.lift(f32.astype(np.float64), w.mask, bins, N)
    np.testing.assert_array_equal(got, ref.astype(np.complex64))


@pytest.mark.parametrize("N,H,W", [(32, 512, 512), (16, 96, 130), (8, 2, 2)])
def test_forward_and_inverse_transforms(N, H, W):
    vol = synth.random_volume(N, H, W, seed=3, dtype=np.complex64)
    plan = se2n.se2n_plan_create(H, W, N)
    v = t_c64(vol)
    se2n.se2n_forward(plan, v)
    fwd = host(v)
    se2n.se2n_inverse(plan, v)
    back = host(v)
    plan.close()
    ref = np.fft.fft2(vol.astype(np.complex128), axes=(1, 2))
    assert rel_l2(fwd, ref) <= 2e-6
    assert rel_l2(back, vol) <= 2e-6


@pytest.mark.parametrize("eps", [0.0, 0.5, 1.0])
def test_static_restoration(eps):
    w = synth.workload_small(64, 96, seed=5, mask_seed=8)
    N = 16
    f32 = w.f.astype(np.float32)
    o = oracle.orient(f32.astype(np.float64), w.mask, N)
    rng = np.random.default_rng(2)
    vol = (rng.uniform(0.05, 1.0, (N, w.H, w.W)) + 1j * rng.standard_normal((N, w.H, w.W)) * 1e-3).astype(np.complex64)
    vol[:, 3, 5] = -0.25  # h(t) <= 0: the linear branch (if the pixel is known)
    vol[:, 7, 9] = 0.01   # h(t) = 0.01 <= 0.1 h(0) when f > 0.1: the linear branch
    plan = se2n.se2n_plan_create(w.H, w.W, N)
    v = t_c64(vol)
    se2n.se2n_mix(plan, v, t_f32(f32), t_u8(w.mask), t_u8(o["bins"]), eps, 0.1)
    got = host(v)
    plan.close()
    ref = oracle.mix(vol.astype(np.complex128), f32.astype(np.float64), w.mask, o["bins"], eps)
    assert np.abs(got.imag).max() == 0
    np.testing.assert_allclose(got.real, ref.real, rtol=2e-6, atol=1e-7)


@pytest.mark.parametrize("proj", [0, 1])
def test_projection(proj):
    N, H, W = 32, 66, 40
    vol = synth.random_volume(N, H, W, seed=9, dtype=np.complex64)
    plan = se2n.se2n_plan_create(H, W, N)
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    se2n.se2n_project(plan, t_c64(vol), proj, out)
    got = host(out)
    plan.close()
    ref = oracle.project(vol.astype(np.complex128), proj)
    if proj == 0:
        np.testing.assert_array_equal(got, ref.astype(np.float32))
    else:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6)


def test_stage_composition_matches_oracle_volume():
    """lift -> forward -> diffuse -> inverse -> mix -> forward -> diffuse ->
    inverse through the individual entry points: the whole volume against
    the oracle's, stage by stage."""
    w = synth.workload_small(64, 64)
    N, beta, T, S, eps = 16, 0.5, 1.0, 50, 0.5
    f32 = w.f.astype(np.float32)
    o = oracle.orient(f32.astype(np.float64), w.mask, N)
    plan = se2n.se2n_plan_create(w.H, w.W, N)
    f_d, m_d, b_d = t_f32(f32), t_u8(w.mask), t_u8(o["bins"])
    v = torch.empty((N, w.H, w.W), dtype=torch.complex64, device="cuda")
    se2n.se2n_lift(plan, f_d, m_d, b_d, v)
    se2n.se2n_forward(plan, v)
    se2n.se2n_diffuse(plan, v, beta, T / 2, S)
    se2n.se2n_inverse(plan, v)
    se2n.se2n_mix(plan, v, f_d, m_d, b_d, eps)
    mixed = host(v)
    se2n.se2n_forward(plan, v)
    se2n.se2n_diffuse(plan, v, beta, T / 2, S)
    se2n.se2n_inverse(plan, v)
    got = host(v)
    plan.close()
    f64 = f32.astype(np.float64)
    r = oracle.forward(oracle.lift(f64, w.mask, o["bins"], N))
    r = oracle.mix(oracle.inverse(oracle.diffuse(r, beta, T / 2, S)), f64, w.mask, o["bins"], eps)
    assert rel_l2(mixed, r) <= REL_L2
    r = oracle.inverse(oracle.diffuse(oracle.forward(r), beta, T / 2, S))
    err = rel_l2(got, r)
    print(f"stage composition volume rel-L2 {err:.2e}")
    assert err <= REL_L2
