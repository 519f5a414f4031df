"""The S-step propagator path (SE2N_DIFFUSE_PROPAGATOR) against the FP64
oracle's step-by-step Crank-Nicolson integration, through the C ABI.

Rows H/2 + s and H - s take the propagator of rows s and H/2 - s with the
angles reversed, so a class covers up to eight frequencies; plane heights
2, 4, 6, 10 and 4m + 2 cover the slots where rows coincide (s = 0, H/4).

The propagator is the same linear map as S steps, built in FP32 by binary
powering in increment form, so it is held to the step kernel's tolerance:
single calls over every supported N, S from 1 to 500 (powers of two and
not), beta dt from 1e-3 to 10, odd-sized and non-square planes; whole
inpaints on both spectrum layouts; the full 512x512, N=32 workload against
the stored oracle result; and the plan's reuse of the matrices."""
import os

import numpy as np
import pytest

import oracle
import synth
from _gpu import (MAX_REL, MAX_REL_512, REL_L2, fp32_sensitivity_512, host, max_rel_for_sigma, rel_l2,
                  restoration_sigma_max, t_c64, t_f32, t_u8)

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")

import torch  # noqa: E402

PROP = se2n.SE2N_DIFFUSE_PROPAGATOR
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "curves_noise_512_N32.npz")


def _run(vol, N, beta, T, S, flags):
    _, H, W = vol.shape
    plan = se2n.se2n_plan_create(H, W, N)
    v = t_c64(vol)
    se2n.se2n_diffuse(plan, v, beta, T, S, flags)
    out = host(v)
    plan.close()
    return out


@pytest.mark.parametrize("N,H,W,beta,T,S", [
    (16, 34, 22, 0.5, 1.0, 20), (32, 30, 26, 0.3, 2.0, 15), (64, 18, 14, 0.25, 2.0, 37),
    (32, 40, 40, 0.25, 2.0, 500), (32, 20, 24, 0.25, 2.0, 1), (32, 20, 24, 0.25, 2.0, 2),
    (16, 12, 64, 0.25, 2.0, 256), (64, 22, 30, 0.7, 3.0, 100),
    (32, 18, 14, 10.0, 20.0, 20), (64, 18, 14, 10.0, 20.0, 20), (16, 2, 6, 0.5, 1.0, 9),
    (16, 4, 8, 0.5, 2.0, 30), (32, 6, 10, 0.5, 2.0, 30), (16, 10, 4, 0.4, 2.0, 25),
    (64, 16, 20, 0.25, 2.0, 500), (64, 18, 14, 0.5, 2.0, 30), (32, 18, 14, 10.0, 30.0, 30),
    (30, 34, 22, 0.25, 2.0, 500), (30, 6, 10, 0.5, 2.0, 30), (30, 18, 14, 0.3, 2.0, 15), (30, 2, 6, 0.5, 1.0, 9)])
def test_propagator_matches_oracle(N, H, W, beta, T, S):
    """The powering programs of S = 15, 30 and 500 square R into P (op 1);
    the others only square P and combine. N = 30 (the angle count of the
    paper's experiments) runs as a 30-angle system in the top-left block of
    32-angle matrices, the padding zero."""
    vol = synth.random_volume(N, H, W, seed=N + H + S).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), beta, T, S)
    got = _run(vol, N, beta, T, S, PROP)
    steps = _run(vol, N, beta, T, S, 0)
    e_ref, e_steps = rel_l2(got, ref), rel_l2(got, steps)
    print(f"N={N} {H}x{W} beta*dt={beta * T / S:.3g} S={S}: rel-L2 vs oracle {e_ref:.2e}, "
          f"vs the step kernel {e_steps:.2e}")
    assert e_ref <= REL_L2
    assert e_steps <= 2 * REL_L2


@pytest.mark.parametrize("N,H,W,beta,T,S,builds", [
    (64, 18, 14, 10.0, 30.0, 30, 0),     # beta dt = 10: propagators measured at 1.3e-5, the step kernel runs
    (32, 18, 14, 10.0, 30.0, 30, 0),
    (32, 18, 14, 0.5, 0.5, 1, 1),        # one step of dt = 0.5: dt (2 + 4 beta) = 2, admitted
    (32, 18, 14, 0.25, 2.0, 3, 1),       # dt = 2/3: dt (2 + 4 beta) = 2, the edge, still admitted
    (32, 18, 14, 0.25, 2.0, 2, 0)])      # dt = 1: dt (2 + 4 beta) = 3 > 2
def test_stiff_steps_fall_back_to_the_step_kernel(N, H, W, beta, T, S, builds):
    """The propagator form is used only where every Crank-Nicolson factor of
    the system is >= 0 (dt (2 + 4 beta) <= 2); elsewhere the step kernel
    runs, and the result is within the bound either way."""
    vol = synth.random_volume(N, H, W, seed=7 + N + S).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), beta, T, S)
    plan = se2n.se2n_plan_create(H, W, N)
    se2n.se2n_plan_profile(plan, True)
    v = t_c64(vol)
    se2n.se2n_diffuse(plan, v, beta, T, S, PROP)
    got = host(v)
    prof = se2n.se2n_plan_profile_read(plan)
    plan.close()
    dt = T / S
    expect = 1 if dt * (2 + 4 * beta) <= 2 else 0
    assert expect == builds
    assert prof["propagator"][1] == builds
    err = rel_l2(got, ref)
    print(f"N={N} beta*dt={beta * dt:.3g} S={S}: {'propagator' if builds else 'step kernel'}, rel-L2 {err:.2e}")
    assert err <= REL_L2


@pytest.mark.parametrize("N,H,conv", [(16, 24, 0), (32, 40, 0), (64, 20, 0), (32, 40, 1), (64, 28, 1), (16, 12, 1),
                                      (30, 36, 0), (30, 20, 1)])
def test_transposed_classes_share_one_build(N, H, conv):
    """On square planes a class and its transpose (row and column slots
    swapped) are one operator up to the angle reflection r -> N/2 - r
    (N/4 - r on the 2 pi r / N grid), so the build computes the upper
    triangle of slot pairs and stores each matrix permuted for its
    transpose: every frequency must still match the oracle. N = 30 on the
    2 pi r / N grid has no such reflection (4 does not divide 30): every
    class is built."""
    vol = synth.random_volume(N, H, H, seed=N + 3 * H + conv).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 0.25, 2.0, 60, angle_conv=conv)
    plan = se2n.se2n_plan_create(H, H, N, conv)
    v = t_c64(vol)
    se2n.se2n_diffuse(plan, v, 0.25, 2.0, 60, PROP)
    got = host(v)
    plan.close()
    err = rel_l2(got, ref)
    print(f"N={N} {H}x{H} conv={conv}: rel-L2 {err:.2e}")
    assert err <= REL_L2


@pytest.mark.parametrize("N,conv", [(32, 1), (16, 1), (32, 0), (30, 0), (30, 1)])
def test_square_inpaint_on_the_passes_with_either_angle_grid(N, conv):
    """The row and column passes on a square plane (transposed classes share
    one build, the matrices stored as rows) with both angle grids."""
    w = synth.workload_512(H=128, W=128, steps=60, rounds=3)
    p = oracle.Params(N=N, beta=0.25, T=6.0, steps=60, rounds=3, angle_conv=conv)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, conv, p.flat_tol)["bins"]
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    plan = se2n.se2n_plan_create(128, 128, N, conv)
    se2n.se2n_plan_profile(plan, True)
    vol = torch.empty((N, 128, 128), dtype=torch.complex64, device="cuda")
    out = torch.empty((128, 128), dtype=torch.float32, device="cuda")
    se2n.se2n_inpaint(plan, t_f32(f32), t_u8(w.mask), t_u8(bins), _params(p), vol, out)
    got = host(out)
    prof = se2n.se2n_plan_profile_read(plan)
    plan.close()
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    print(f"128x128 N={N} conv={conv}: max-abs/max|f| {mx:.2e}, rel-L2 {rel_l2(got, ref):.2e}")
    assert prof["propagator"][1] == 1 and prof["diffuse"][1] == 3
    assert mx <= MAX_REL
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("H,W,conv", [(136, 136, 0), (136, 136, 1), (72, 136, 0), (136, 72, 0), (20, 20, 1),
                                      (64, 64, 0), (22, 22, 1), (26, 18, 0)])
def test_tiled_apply_N64_on_the_hermitian_half(H, W, conv):
    """N = 64 on the Hermitian half: the propagators stored as rows (a
    square plane builds only the classes with row slot <= column slot) and
    applied a tile of 16 column slots at a time, a transposed class through
    the permuted vectors. 136 x 136 has 35 row and column slots: two
    super-tiles a side, the second ragged, and a ragged last tile in every
    row slot; sides of 4m + 2 pair columns l, W/2 - l with W/2 odd (no
    self-paired column) and have no self-paired row."""
    w = synth.workload_512(H=H, W=W, steps=60, rounds=3)
    p = oracle.Params(N=64, beta=0.25, T=6.0, steps=60, rounds=3, angle_conv=conv)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, conv, p.flat_tol)["bins"]
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    plan = se2n.se2n_plan_create(H, W, 64, conv)
    se2n.se2n_plan_profile(plan, True)
    vol = torch.empty((64, H, W), dtype=torch.complex64, device="cuda")
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    se2n.se2n_inpaint(plan, t_f32(f32), t_u8(w.mask), t_u8(bins), _params(p), vol, out)
    got = host(out)
    prof = se2n.se2n_plan_profile_read(plan)
    plan.close()
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    print(f"{H}x{W} N=64 conv={conv}: max-abs/max|f| {mx:.2e}, rel-L2 {rel_l2(got, ref):.2e}")
    assert prof["propagator"][1] == 1 and prof["diffuse"][1] == 3
    assert mx <= MAX_REL
    assert rel_l2(got, ref) <= REL_L2


def test_lifted_image_spectrum():
    """The workload's shape: the DFT of a lifted image, dominated by the low
    frequencies, 500 steps."""
    w = synth.workload_512(H=64, W=96, steps=500, rounds=1)
    bins = oracle.orient(w.f, w.mask, 32)["bins"]
    vol = oracle.forward(oracle.lift(w.f, w.mask, bins, 32))
    ref = oracle.diffuse(vol, 0.25, 2.0, 500)
    got = _run(vol.astype(np.complex64), 32, 0.25, 2.0, 500, PROP)
    err = rel_l2(got, ref)
    print(f"lifted 64x96 N=32 500 steps: rel-L2 {err:.2e}")
    assert err <= REL_L2


def test_unsupported_angle_count():
    plan = se2n.se2n_plan_create(8, 8, 24)
    v = torch.zeros((24, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse(plan, v, 0.25, 1.0, 10, PROP)
    assert e.value.status == se2n.SE2N_EUNSUPPORTED
    plan.close()


def test_matrices_are_rebuilt_only_when_the_step_changes():
    vol = synth.random_volume(32, 16, 20, seed=4).astype(np.complex64)
    plan = se2n.se2n_plan_create(16, 20, 32)
    se2n.se2n_plan_profile(plan, True)
    outs = []
    for beta, T, S in [(0.25, 2.0, 50), (0.25, 2.0, 50), (0.5, 2.0, 50), (0.5, 2.0, 60), (0.5, 2.0, 60)]:
        v = t_c64(vol)
        se2n.se2n_diffuse(plan, v, beta, T, S, PROP)
        outs.append((host(v), oracle.diffuse(vol.astype(np.complex128), beta, T, S)))
    for free in (False, True):   # dropped matrices are built again, with or without their memory
        se2n.se2n_plan_drop_propagators(plan, free)
        v = t_c64(vol)
        se2n.se2n_diffuse(plan, v, 0.5, 2.0, 60, PROP)
        outs.append((host(v), outs[-1][1]))
    prof = se2n.se2n_plan_profile_read(plan)
    plan.close()
    assert prof["propagator"][1] == 5 and prof["diffuse"][1] == 7
    for got, ref in outs:
        assert rel_l2(got, ref) <= REL_L2
    np.testing.assert_array_equal(outs[-1][0], outs[-3][0])


def _params(p, full=0):
    return se2n.se2n_params_default(N=p.N, beta=p.beta, T=p.T, steps=p.steps, rounds=p.rounds, eps=p.eps,
                                    sigma_smooth=p.sigma, flat_tol=p.flat_tol, proj=p.proj,
                                    final_mix=p.final_mix, guard=p.guard, reinject=p.reinject,
                                    full_spectrum=full, diffuse_flags=PROP)


def _gpu_inpaint(f32, mask, bins, prm, profile=False):
    H, W = f32.shape
    plan = se2n.se2n_plan_create(H, W, prm.N)
    vol = torch.empty((prm.N, H, W), dtype=torch.complex64, device="cuda")
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    if profile:
        se2n.se2n_plan_profile(plan, True)
    se2n.se2n_inpaint(plan, t_f32(f32), t_u8(mask), t_u8(bins), prm, vol, out)
    got = host(out)
    prof = se2n.se2n_plan_profile_read(plan) if profile else None
    plan.close()
    return got, prof


@pytest.mark.parametrize("H,W,N,full", [(96, 96, 32, 0), (64, 160, 32, 1), (64, 64, 16, 0), (48, 80, 64, 0),
                                         (66, 70, 16, 0), (70, 66, 32, 1), (96, 96, 30, 0), (64, 80, 30, 1)])
def test_inpaint_with_propagators_matches_oracle(H, W, N, full):
    w = synth.workload_512(H=H, W=W, steps=60, rounds=3)
    p = oracle.Params(N=N, beta=0.25, T=6.0, steps=60, rounds=3)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, 0, p.flat_tol)["bins"]
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    got, prof = _gpu_inpaint(f32, w.mask, bins, _params(p, full), profile=True)
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    r2 = rel_l2(got, ref)
    print(f"{H}x{W} N={N} full={full}: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e}")
    assert prof["propagator"][1] == 1 and prof["diffuse"][1] == 3   # built once, applied every interval
    assert mx <= MAX_REL
    assert r2 <= REL_L2


def test_full_512_N32_ten_rounds_against_stored_oracle():
    if not os.path.exists(GOLDEN):
        pytest.fail("missing tests/golden/curves_noise_512_N32.npz: run tests/golden/make_references.py")
    g = np.load(GOLDEN)
    w = synth.workload_512()
    p = oracle.Params(N=32, beta=0.25, T=20.0, steps=500, rounds=10)
    got, _ = _gpu_inpaint(w.f.astype(np.float32), w.mask, g["bins"], _params(p))
    ref = g["out"].astype(np.float64)
    mx = np.abs(got - ref).max() / np.abs(w.f).max()
    r2 = rel_l2(got, ref)
    print(f"512x512 propagators: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e} (bound {MAX_REL_512:.2e})")
    assert mx <= MAX_REL_512
    assert r2 <= REL_L2


def test_full_512_paper_angle_count_N30_against_stored_oracle():
    """The 512x512 workload with the paper's N = 30 on the row and column
    passes (the 30-angle system in 32 slots), against the FP64 oracle's
    stored result; the bound is derived as for N = 32, from the oracle's own
    sensitivity to FP32 rounding at N = 30."""
    path = os.path.join(os.path.dirname(GOLDEN), "curves_noise_512_N30.npz")
    if not os.path.exists(path):
        pytest.fail("missing tests/golden/curves_noise_512_N30.npz: run tests/golden/make_references.py n30")
    g = np.load(path)
    w = synth.workload_512(N=30)
    p = oracle.Params(N=30, beta=0.25, T=20.0, steps=500, rounds=10)
    got, prof = _gpu_inpaint(w.f.astype(np.float32), w.mask, g["bins"], _params(p), profile=True)
    ref = g["out"].astype(np.float64)
    bound = 4.0 * fp32_sensitivity_512(30)
    mx = np.abs(got - ref).max() / np.abs(w.f).max()
    r2 = rel_l2(got, ref)
    print(f"512x512 N=30 propagators: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e} (bound {bound:.2e})")
    assert prof["propagator"][1] == 1 and prof["diffuse"][1] == 10 and prof["fft"][1] == 11
    assert mx <= bound
    assert r2 <= REL_L2


@pytest.mark.parametrize("H,W,N,dynamic,final_mix,proj,reinject", [
    (64, 128, 32, 0, 0, 0, 0), (128, 64, 16, 0, 1, 0, 0), (256, 64, 32, 0, 0, 1, 1), (64, 64, 16, 1, 0, 0, 0),
    (128, 128, 32, 1, 1, 0, 1), (512, 256, 16, 0, 1, 1, 0), (1024, 128, 32, 0, 0, 0, 0),
    (128, 1024, 16, 0, 0, 0, 1), (1024, 64, 32, 1, 0, 0, 0), (384, 256, 32, 0, 0, 0, 0), (256, 768, 16, 0, 1, 1, 0),
    (768, 64, 32, 1, 0, 0, 1), (384, 384, 32, 0, 0, 0, 0),
    (64, 128, 30, 0, 0, 0, 0), (128, 128, 30, 1, 1, 0, 1), (256, 64, 30, 0, 0, 1, 1), (384, 128, 30, 0, 1, 0, 0)])
def test_row_and_column_passes_match_oracle(H, W, N, dynamic, final_mix, proj, reinject):
    """Plane sizes with H and W in {64, 128, 256, 384, 512, 768, 1024} and N =
    16, 30 or 32 run the fused passes (N = 30, the paper's angle count, as a
    30-angle system in 32 slots: angle r at slot r below 15, 15 at slot 16,
    the others two slots up, so that angle reversal modulo 30 is slot reversal
    modulo 32 and slots 15 and 17 stay empty): a row pass (lift, or inverse DFT along x,
    restoration and forward DFT along x, or projection) and a column pass
    (DFT along y, propagators, inverse DFT along y) an interval. Cases cover
    every radix mix of both lengths (8 x 4 .. 16 x 16, 8 x 8 x 8 and the
    radix-3 lengths 3 x 8 x 8 (x 2)), the final restoration, mean projection,
    reinjection and dynamic restoration (a row pass gives the image value and
    its argmax angle to each growth step; the restoration pulls the grown set
    to its references while reinjection keeps the given known pixels)."""
    w = synth.workload_512(H=H, W=W, steps=60, rounds=3)
    p = oracle.Params(N=N, beta=0.25, T=6.0, steps=60, rounds=3, dynamic=dynamic, final_mix=final_mix, proj=proj,
                      reinject=reinject)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, 0, p.flat_tol)["bins"]
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    prm = _params(p)
    prm.dynamic = dynamic
    got, prof = _gpu_inpaint(f32, w.mask, bins, prm, profile=True)
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    r2 = rel_l2(got, ref)
    print(f"{H}x{W} N={N} dynamic={dynamic} final_mix={final_mix} proj={proj} reinject={reinject}: "
          f"max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e}")
    # one build; one column pass an interval; row passes: lift, one between
    # intervals, last, and with dynamic restoration one more (image value and
    # argmax) before each growth step
    assert prof["propagator"][1] == 1 and prof["diffuse"][1] == 3
    assert prof["fft"][1] == 4 + (2 + final_mix if dynamic else 0)
    assert prof["dr"][1] == (2 + final_mix if dynamic else 0) and prof["mix"][1] == 0
    assert mx <= MAX_REL
    assert r2 <= REL_L2


@pytest.mark.parametrize("H,W,N", [(64, 128, 32), (128, 64, 16), (128, 128, 32), (96, 96, 32)])
def test_paper_sigma_rule_guard_zero_on_the_propagator_paths(H, W, N):
    """Section 5's restoration with no relative guard (guard = 0 on both
    sides) on the row and column passes (power-of-two planes) and on the
    separate propagator apply (96 x 96), several intervals; the max-abs bound
    is MAX_REL up to a largest restoration factor sigma of 10 and grows with
    sigma beyond (64x128 reaches 233 at guard 0)."""
    w = synth.workload_512(H=H, W=W, steps=60, rounds=3)
    p = oracle.Params(N=N, beta=0.25, T=6.0, steps=60, rounds=3, guard=0.0)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, p.N, p.sigma, 0, p.flat_tol)["bins"]
    ref = oracle.inpaint(f64, w.mask, p, bins=bins)["out"]
    got, prof = _gpu_inpaint(f32, w.mask, bins, _params(p), profile=True)
    mx = np.abs(got - ref).max() / np.abs(f64).max()
    r2 = rel_l2(got, ref)
    sig = restoration_sigma_max(f64, w.mask, bins, p)
    print(f"guard 0, {H}x{W} N={N}: max-abs/max|f| {mx:.2e}, rel-L2 {r2:.2e}, largest sigma {sig:.3g}, "
          f"bound {max_rel_for_sigma(sig):.2e}")
    assert prof["propagator"][1] == 1
    assert mx <= max_rel_for_sigma(sig)
    assert r2 <= REL_L2


def test_side_stream_build_is_ordered_with_the_plan_stream():
    """se2n_inpaint builds its propagators on a side stream while the
    orientation and the lift run. Inpaints queued back to back with a new
    beta dt each (every one forks a build while the previous one's passes
    may still run), a drop with its memory freed in between, and a plan
    destroyed with work still queued must all give the oracle's results."""
    H, W, N = 64, 128, 32
    w = synth.workload_512(H=H, W=W, steps=40, rounds=2)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, N, 1.0, 0, 1e-4)["bins"]
    plan = se2n.se2n_plan_create(H, W, N)
    f_d, m_d, b_d = t_f32(f32), t_u8(w.mask), t_u8(bins)
    vol = torch.empty((N, H, W), dtype=torch.complex64, device="cuda")
    outs, refs = [], []
    for i, T in enumerate([2.0, 4.0, 4.0, 6.0]):
        p = oracle.Params(N=N, beta=0.25, T=T, steps=40, rounds=2)
        out = torch.empty((H, W), dtype=torch.float32, device="cuda")
        se2n.se2n_inpaint(plan, f_d, m_d, b_d, _params(p), vol, out)   # no synchronisation in between
        if i == 1:
            se2n.se2n_plan_drop_propagators(plan, True)
        outs.append(out)
        refs.append(oracle.inpaint(f64, w.mask, p, bins=bins)["out"])
    plan.close()   # destroys the plan (and its side stream) with nothing synchronised yet
    for out, ref in zip(outs, refs):
        got = host(out)
        assert rel_l2(got, ref) <= REL_L2
        assert np.abs(got - ref).max() <= MAX_REL * np.abs(f64).max()
