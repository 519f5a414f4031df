"""End-to-end parity of se2n_inpaint (lift, DFT, fused CN diffusion, static
restoration between intervals, inverse DFT, projection) against the FP64
oracle through the C ABI.

The orientation bins are a floating-point decision (tested on their own in
test_gpu_stages.py); here both sides get the oracle's bins so the rest of
the path is compared at the FP32 tolerance. The GPU's own-bins path is
checked to be the same computation (bitwise) as orient + inpaint.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from _gpu import (MAX_REL, MAX_REL_512, REL_L2, host, max_rel_for_sigma, rel_l2, restoration_sigma_max, t_f32,
                  t_u8)

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")

import torch  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "curves_noise_512_N32.npz")


def _gpu_inpaint(f32, mask, bins, prm, conv=0, tune=None):
    H, W = f32.shape
    plan = se2n.se2n_plan_create(H, W, prm.N, conv)
    if tune:
        se2n.se2n_plan_tune_diffuse(plan, *tune)
    vol = torch.empty((prm.N, H, W), dtype=torch.complex64, device="cuda")
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    se2n.se2n_inpaint(plan, t_f32(f32), t_u8(mask), None if bins is None else t_u8(bins), prm, vol, out)
    got = host(out)
    plan.close()
    return got


def _params(p: oracle.Params, flags=0, full=0):
    return se2n.se2n_params_default(N=p.N, beta=p.beta, T=p.T, steps=p.steps, rounds=p.rounds, eps=p.eps,
                                    sigma_smooth=p.sigma, flat_tol=p.flat_tol, proj=p.proj,
                                    final_mix=p.final_mix, guard=p.guard, diffuse_flags=flags,
                                    reinject=p.reinject, full_spectrum=full)


def _compare(w, p, conv=0, flags=0, tune=None, full=0):
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, conv, p.flat_tol)["bins"]
    p.angle_conv = conv
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    got = _gpu_inpaint(f32, w.mask, bins, _params(p, flags, full), conv, tune)
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    r2 = rel_l2(got, ref)
    print(f"{w.H}x{w.W} N={p.N} S={p.steps} R={p.rounds}: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e}")
    assert mx <= MAX_REL
    assert r2 <= REL_L2
    return got


def test_small_workload_single_round():
    """64x64 lines and circles, 50 % random mask, N=16, beta=0.5, T=1 in
    100 steps, one round (the plain method)."""
    w = synth.workload_small()
    _compare(w, oracle.Params(N=16, beta=0.5, T=1.0, steps=100, rounds=1))


def test_reduced_512_geometry_three_rounds():
    w = synth.workload_512(H=128, W=128, steps=100, rounds=3)
    _compare(w, oracle.Params(N=32, beta=0.25, T=6.0, steps=100, rounds=3))


@pytest.mark.parametrize("variant", ["mean", "final_mix", "conv1", "fp64", "N64", "P4", "nonsquare", "reinject",
                                     "full_spectrum", "full_spectrum_nonsquare"])
def test_variants(variant):
    w = synth.workload_512(H=96, W=96, steps=60, rounds=3)
    p = oracle.Params(N=32, beta=0.25, T=6.0, steps=60, rounds=3)
    conv, flags, tune = 0, 0, None
    if variant == "mean":
        p.proj = 1
    elif variant == "final_mix":
        p.final_mix = 1
    elif variant == "conv1":
        conv = 1
    elif variant == "fp64":
        flags = se2n.SE2N_DIFFUSE_SM_FP64
    elif variant == "N64":
        p.N = 64
    elif variant == "P4":
        tune = (4, 128, 0)
    elif variant == "nonsquare":
        w = synth.workload_512(H=64, W=160, steps=60, rounds=3)
    elif variant == "reinject":
        p.reinject = 1
    full = 1 if variant.startswith("full_spectrum") else 0
    if variant == "full_spectrum_nonsquare":
        w = synth.workload_512(H=64, W=160, steps=60, rounds=3)
    got = _compare(w, p, conv, flags, tune, full)
    if variant == "reinject":
        k = w.mask != 0
        np.testing.assert_array_equal(got[k], w.f.astype(np.float32)[k])


@pytest.mark.parametrize("case", ["96", "128", "64x128", "full_spectrum", "fp64", "table1"])
def test_paper_sigma_rule_guard_zero(case):
    """The static restoration exactly as Section 5 states it: sigma =
    (eps h(0) + (1-eps) h(t_i)) / h(t_i) at every good pixel with h(t_i) > 0
    (guard = 0 on both sides, no relative guard), several intervals. Without
    the guard a good pixel whose value has decayed to a small h(t_i) is
    scaled by a large sigma, which multiplies the FP32 error there: the
    bound is MAX_REL while the largest sigma of the oracle's run stays below
    10 (96x96: 7.3, 128x128: 9.9, Table 1: below 10) and grows with it
    beyond (64x128: sigma 233 at the second restoration)."""
    if case == "table1":
        beta, T = oracle.params_from_paper(0.30, 4.0, 256, 30)
        clean = synth.curves_noise_image(64, 64, 8, n_curves=12)
        mask = synth.bar_mask(64, 64, 3, 10)
        w = synth.Workload("table1", clean, mask, N=30, beta=beta, T=T / 160 * 4, steps=20, rounds=4)
        p = oracle.Params(N=30, beta=beta, T=T / 160 * 4, steps=20, rounds=4, guard=0.0)
    else:
        H, W = {"128": (128, 128), "64x128": (64, 128)}.get(case, (96, 96))
        steps = 100 if case == "128" else 60
        w = synth.workload_512(H=H, W=W, steps=steps, rounds=3)
        p = oracle.Params(N=32, beta=0.25, T=6.0, steps=steps, rounds=3, guard=0.0)
    flags = se2n.SE2N_DIFFUSE_SM_FP64 if case == "fp64" else 0
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, 0, p.flat_tol)["bins"]
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    got = _gpu_inpaint(f32, w.mask, bins, _params(p, flags, 1 if case == "full_spectrum" else 0))
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    r2 = rel_l2(got, ref)
    sig = restoration_sigma_max(f64, w.mask, bins, p)
    print(f"guard 0, {case}: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e}, largest sigma {sig:.3g}, "
          f"bound {max_rel_for_sigma(sig):.2e}")
    if case != "64x128":
        assert sig <= 10.0
    assert mx <= max_rel_for_sigma(sig)
    assert r2 <= REL_L2


@pytest.mark.parametrize("H,W,conv", [(96, 96, 0), (64, 160, 0), (128, 66, 1)])
def test_hermitian_half_equals_full_spectrum(H, W, conv):
    """The Hermitian-half path (R2C transforms, frequencies l <= W/2) and the
    full complex path are the same method: they agree to FP32 rounding of the
    transforms, far inside the oracle tolerance."""
    w = synth.workload_512(H=H, W=W, steps=60, rounds=3)
    p = oracle.Params(N=32, beta=0.25, T=6.0, steps=60, rounds=3)
    bins = oracle.orient(w.f.astype(np.float32).astype(np.float64), w.mask, p.N, p.sigma, conv, p.flat_tol)["bins"]
    f32 = w.f.astype(np.float32)
    half = _gpu_inpaint(f32, w.mask, bins, _params(p, 0, 0), conv)
    full = _gpu_inpaint(f32, w.mask, bins, _params(p, 0, 1), conv)
    r = rel_l2(half, full)
    print(f"{H}x{W} conv {conv}: half vs full rel-L2 {r:.2e}")
    assert r <= 1e-6


def test_table1_parameters_in_pixel_units():
    """A Table 1 row (alpha=0.3, T=4, n=160 in the paper's units, M=256,
    N=30) mapped to pixel units, on a bar-corrupted 64x64 image with a few
    of its restoration intervals."""
    beta, T = se2n.se2n_params_from_paper(0.30, 4.0, 256, 30)
    ob, oT = oracle.params_from_paper(0.30, 4.0, 256, 30)
    assert abs(beta - ob) < 1e-15 and abs(T - oT) < 1e-12
    clean = synth.curves_noise_image(64, 64, 8, n_curves=12)
    mask = synth.bar_mask(64, 64, 3, 10)
    w = synth.Workload("table1", clean, mask, N=30, beta=beta, T=T / 160 * 4, steps=20, rounds=4)
    _compare(w, oracle.Params(N=30, beta=beta, T=T / 160 * 4, steps=20, rounds=4))


def test_full_512_N32_ten_rounds_against_stored_oracle():
    """The full workload (512x512, N=32, beta=0.25, 10 intervals of 500
    steps) against the FP64 oracle's result written by
    tests/golden/make_references.py."""
    if not os.path.exists(GOLDEN):
        pytest.fail("missing tests/golden/curves_noise_512_N32.npz: run tests/golden/make_references.py")
    g = np.load(GOLDEN)
    w = synth.workload_512()
    p = oracle.Params(N=32, beta=0.25, T=20.0, steps=500, rounds=10)
    got = _gpu_inpaint(w.f.astype(np.float32), w.mask, g["bins"], _params(p))
    ref = g["out"].astype(np.float64)
    mx = np.abs(got - ref).max() / np.abs(w.f).max()
    r2 = rel_l2(got, ref)
    print(f"512^2 N=32 10x500: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e} (bound {MAX_REL_512:.2e})")
    assert mx <= MAX_REL_512
    assert r2 <= REL_L2


GOLDEN_2048 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lines_patches_2048_N64.npz")


@pytest.mark.parametrize("run,flags", [("main", 0), ("main", se2n.SE2N_DIFFUSE_PROPAGATOR), ("stress", 0),
                                       ("stress", se2n.SE2N_DIFFUSE_SM_FP64)])
def test_2048_N64_against_stored_oracle(run, flags):
    """The 2048x2048, N=64 workload (2 GiB volume, one interval of 1000
    steps, 85 % corrupted) against the FP64 oracle's result written by
    tests/golden/make_reference_2048.py, compared at every 4th row and
    column: the main run (beta = 0.25) step by step and with propagators,
    and the stiff run (beta dt = 10: split diagonal; the propagator flag
    falls back to the steps there) with the FP32 and the FP64 corner
    correction. One interval, so the single-result bound applies."""
    if not os.path.exists(GOLDEN_2048):
        pytest.fail("missing tests/golden/lines_patches_2048_N64.npz: run tests/golden/make_reference_2048.py")
    g = np.load(GOLDEN_2048)
    st = int(g["stride"][0])
    w = synth.workload_2048(stress=run == "stress")
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, w.N)["bins"]
    p = oracle.Params(N=w.N, beta=w.beta, T=w.T, steps=w.steps, rounds=w.rounds, eps=w.eps)
    got = _gpu_inpaint(f32, w.mask, bins, _params(p, flags))[::st, ::st].astype(np.float64)
    ref = g[f"{run}_out"].astype(np.float64)
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    r2 = rel_l2(got, ref)
    print(f"2048^2 N=64 {run} flags={flags}: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e} (every {st}th row and column)")
    assert mx <= MAX_REL
    assert r2 <= REL_L2


def test_own_bins_path_is_orient_then_inpaint():
    w = synth.workload_512(H=128, W=128, steps=20, rounds=2)
    p = oracle.Params(N=32, beta=0.25, T=4.0, steps=20, rounds=2)
    f32 = w.f.astype(np.float32)
    plan = se2n.se2n_plan_create(w.H, w.W, 32)
    b = torch.empty((w.H, w.W), dtype=torch.uint8, device="cuda")
    se2n.se2n_orient(plan, t_f32(f32), t_u8(w.mask), 1.0, 1e-4, b)
    bins = host(b)
    plan.close()
    a = _gpu_inpaint(f32, w.mask, None, _params(p))
    c = _gpu_inpaint(f32, w.mask, bins, _params(p))
    np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("flags", [0, se2n.SE2N_DIFFUSE_PROPAGATOR])
def test_host_entry_point_matches_device_entry_point(flags):
    """se2n_inpaint_host gives se2n_inpaint's bits, step by step and on the
    row and column passes (where it starts the propagator build before its
    host copies; the second call reuses the propagators)."""
    w = synth.workload_512(H=128, W=64, steps=20, rounds=2)
    p = oracle.Params(N=32, beta=0.25, T=4.0, steps=20, rounds=2)
    f32 = np.ascontiguousarray(w.f.astype(np.float32))
    mask = np.ascontiguousarray(w.mask.astype(np.uint8))
    prm = _params(p)
    prm.diffuse_flags = flags
    dev = _gpu_inpaint(f32, mask, None, prm)
    plan = se2n.se2n_plan_create(w.H, w.W, 32)
    out = np.zeros((w.H, w.W), np.float32)
    for _ in range(2):  # the second call reuses the plan's buffers
        se2n.se2n_inpaint_host(plan, f32, mask, prm, out)
        np.testing.assert_array_equal(out, dev)
    plan.close()


def test_rotation_equivariance_full_size():
    """Property at the full 512x512 size: rotating the input by 90 degrees
    rotates the output (bins rotated with their channel shift N/2)."""
    w = synth.workload_512(steps=100, rounds=2)
    N = 32
    p = oracle.Params(N=N, beta=0.25, T=4.0, steps=100, rounds=2)
    f32 = w.f.astype(np.float32)
    bins = oracle.orient(f32.astype(np.float64), w.mask, N)["bins"]
    rb = np.rot90(bins).copy()
    single = rb != oracle.BIN_FLAT
    rb[single] = (rb[single].astype(int) + N // 2) % N
    a = _gpu_inpaint(f32, w.mask, bins, _params(p))
    b = _gpu_inpaint(np.rot90(f32).copy(), np.rot90(w.mask).copy(), rb, _params(p))
    assert rel_l2(b, np.rot90(a)) <= REL_L2


def test_inpaint_rejects_bad_parameters():
    plan = se2n.se2n_plan_create(16, 16, 16)
    f = t_f32(np.ones((16, 16)))
    m = t_u8(np.ones((16, 16)))
    vol = torch.empty((16, 16, 16), dtype=torch.complex64, device="cuda")
    out = torch.empty((16, 16), dtype=torch.float32, device="cuda")
    bad = [dict(N=32), dict(eps=1.5), dict(rounds=0), dict(steps=0), dict(beta=0.0), dict(proj=3),
           dict(sigma_smooth=0.0), dict(final_mix=2), dict(diffuse_flags=16), dict(reinject=2), dict(dynamic=2)]
    for b in bad:
        prm = se2n.se2n_params_default(N=16)
        for k, v in b.items():
            setattr(prm, k, v)
        with pytest.raises(se2n.Se2nError) as e:
            se2n.se2n_inpaint(plan, f, m, None, prm, vol, out)
        assert e.value.status == se2n.SE2N_EINVAL, b
    prm = se2n.se2n_params_default(N=16)
    with pytest.raises(se2n.Se2nError):
        se2n.se2n_inpaint(plan, np.ones((16, 16), np.float32), m, None, prm, vol, out)   # host image
    plan.close()
