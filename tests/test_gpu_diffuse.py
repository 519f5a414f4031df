"""GPU parity of the fused Crank-Nicolson diffusion (se2n_diffuse) against
the FP64 oracle, element by element, through the C ABI.

Sizes are chosen so the frequency count spans many blocks with a ragged
tail; every (N, threads per frequency) instantiation is exercised; the full
512x512 N=32 and 2048x2048 N=64 sizes run in the default launch
configuration (the one bench.py times) and are compared on sampled
frequencies the oracle integrates one by one.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu import REL_L2, host, rel_l2, t_c64

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")


def _run(vol, N, beta, T, S, conv=0, flags=0, tune=None):
    _, H, W = vol.shape
    plan = se2n.se2n_plan_create(H, W, N, conv)
    if tune:
        se2n.se2n_plan_tune_diffuse(plan, *tune)
    v = t_c64(vol)
    se2n.se2n_diffuse(plan, v, beta, T, S, flags)
    out = host(v)
    plan.close()
    return out


VARIANTS = [(4, 1), (8, 1), (8, 2), (12, 1), (12, 2), (16, 1), (16, 2), (16, 4), (24, 2), (24, 4), (30, 2),
            (32, 2), (32, 4), (48, 4), (64, 4)]


@pytest.mark.parametrize("N,P", VARIANTS)
def test_diffuse_matches_oracle_every_instantiation(N, P):
    vol = synth.random_volume(N, 34, 22, seed=N * 10 + P).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 0.5, 1.0, 20)
    got = _run(vol, N, 0.5, 1.0, 20, tune=(P, 128, 0))
    err = rel_l2(got, ref)
    print(f"N={N} P={P} rel-L2 {err:.2e}")
    assert err <= REL_L2


@pytest.mark.parametrize("block,blocks", [(32, 1), (64, 3), (256, 0), (96, 7), (384, 0), (0, 0)])
def test_grid_stride_and_block_shapes(block, blocks):
    """Few blocks force many passes of the grid-stride loop; odd block
    counts leave partially filled warps at the tail."""
    vol = synth.random_volume(32, 30, 26, seed=5).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 0.3, 2.0, 15)
    got = _run(vol, 32, 0.3, 2.0, 15, tune=(2, block, blocks))
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("N,P", [(16, 1), (32, 2), (64, 4)])
def test_every_launch_shape_gives_the_same_bits(N, P):
    """Each frequency's arithmetic does not depend on which thread or block
    takes it: the default shape (128-thread blocks over all frequencies
    below N = 48, resident 384-thread blocks from N = 48 on), resident and
    one-pass grids, 384-thread blocks (lowered to 256 below N = 48) and a
    few-block grid-stride launch give bitwise the same volume."""
    vol = synth.random_volume(N, 36, 50, seed=N + 7).astype(np.complex64)
    outs = [_run(vol, N, 0.25, 1.0, 50, tune=(P, block, blocks))
            for block, blocks in [(0, 0), (128, 0), (128, 1 << 20), (256, 0), (384, 0), (384, 1 << 20), (64, 5)]]
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint64), outs[0].view(np.uint64))


@pytest.mark.parametrize("conv", [0, 1])
def test_angle_conventions(conv):
    vol = synth.random_volume(16, 20, 20, seed=3).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 0.7, 1.5, 25, angle_conv=conv)
    got = _run(vol, 16, 0.7, 1.5, 25, conv=conv)
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("N,flags", [(16, 0), (32, 0), (64, 0), (32, 1), (64, 1)])
def test_stiff_beta_dt_10(N, flags):
    """beta*dt = 10: the corner correction is far from negligible; with
    and without the FP64 Sherman-Morrison scalars."""
    vol = synth.random_volume(N, 18, 14, seed=11).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 10.0, 20.0, 20)
    got = _run(vol, N, 10.0, 20.0, 20, flags=flags)
    err = rel_l2(got, ref)
    print(f"N={N} flags={flags} beta*dt=10 rel-L2 {err:.2e}")
    assert err <= REL_L2


def test_long_integration_500_steps():
    vol = synth.random_volume(32, 40, 40, seed=2).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 0.25, 2.0, 500)
    got = _run(vol, 32, 0.25, 2.0, 500)
    err = rel_l2(got, ref)
    print(f"500 steps rel-L2 {err:.2e}")
    assert err <= REL_L2


def test_lifted_image_spectrum():
    """The real workload shape: the DFT of a lifted image (dominated by the
    low frequencies), not a white random volume."""
    w = synth.workload_small(64, 64)
    p = oracle.Params(N=16, beta=0.5, T=1.0, steps=100)
    vol, _ = oracle.lift_from_image(w.f.astype(np.float32), w.mask, p)
    vh = oracle.forward(vol).astype(np.complex64)
    ref = oracle.diffuse(vh.astype(np.complex128), 0.5, 1.0, 100)
    got = _run(vh, 16, 0.5, 1.0, 100)
    assert rel_l2(got, ref) <= REL_L2


def test_zero_frequency_constant_mode_is_exact():
    """The constant angular vector at omega = 0 is a fixed point of the
    increment form in FP32 arithmetic: it must come back bit-identical."""
    vol = np.zeros((32, 8, 8), np.complex64)
    vol[:, 0, 0] = np.complex64(3.25 - 1.5j)
    got = _run(vol, 32, 0.25, 5.0, 200)
    assert (got[:, 0, 0] == vol[:, 0, 0]).all()


def test_mass_preservation_on_gpu():
    vol = synth.random_volume(32, 16, 16, seed=4).astype(np.complex64)
    got = _run(vol, 32, 0.25, 20.0, 300)
    s0 = vol[:, 0, 0].astype(np.complex128).sum()
    s1 = got[:, 0, 0].astype(np.complex128).sum()
    assert abs(s1 - s0) <= 1e-5 * abs(s0)


def test_t_zero_is_a_no_op():
    vol = synth.random_volume(16, 6, 8, seed=1).astype(np.complex64)
    got = _run(vol, 16, 0.5, 0.0, 10)
    np.testing.assert_array_equal(got, vol)


def test_smallest_grid():
    vol = synth.random_volume(8, 2, 2, seed=6).astype(np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), 0.5, 1.0, 10)
    assert rel_l2(_run(vol, 8, 0.5, 1.0, 10), ref) <= REL_L2


def _sampled(H, W, count, seed):
    rng = np.random.default_rng(seed)
    # always include the zero frequency, the Nyquist corners and the last index
    fixed = [0, W // 2, (H // 2) * W, (H // 2) * W + W // 2, H * W - 1]
    return np.unique(np.concatenate([fixed, rng.choice(H * W, count, replace=False)]))


def test_full_size_512_N32_500_steps_sampled():
    """512x512, N=32, one interval of 500 steps (dt = 0.004, beta = 0.25):
    the GPU integrates the whole volume in the default launch
    configuration; the oracle integrates 600 sampled frequencies."""
    N, H, W = 32, 512, 512
    vol = synth.random_volume(N, H, W, seed=21).astype(np.complex64)
    freqs = _sampled(H, W, 600, 1)
    got = _run(vol, N, 0.25, 2.0, 500).reshape(N, -1)[:, freqs]
    ref = oracle.diffuse(vol.astype(np.complex128), 0.25, 2.0, 500, freqs=freqs).reshape(N, -1)[:, freqs]
    err = rel_l2(got, ref)
    print(f"512^2 N=32 S=500 sampled rel-L2 {err:.2e}")
    assert err <= REL_L2


@pytest.mark.parametrize("beta,T,flags", [(0.25, 50.0, 0), (10.0, 1000.0, 0), (10.0, 1000.0, 1)])
def test_full_size_2048_N64_1000_steps_sampled(beta, T, flags):
    """2048x2048, N=64 (a 2 GiB complex64 volume), 1000 fused steps; the
    main run (dt = 0.05) and the beta*dt = 10 stress run, sampled."""
    N, H, W = 64, 2048, 2048
    vol_h = synth.random_volume(N, H, W, seed=44, dtype=np.complex64)
    freqs = _sampled(H, W, 200, 2)
    before = vol_h.reshape(N, -1)[:, freqs].astype(np.complex128)
    vol = t_c64(vol_h)
    del vol_h
    plan = se2n.se2n_plan_create(H, W, N)
    se2n.se2n_diffuse(plan, vol, beta, T, 1000, flags)
    after = vol.reshape(N, -1)[:, torch.tensor(freqs, device=vol.device)].cpu().numpy()
    plan.close()
    del vol
    torch.cuda.empty_cache()
    # the oracle integrates exactly the sampled frequencies of the same input
    full = np.zeros((N, H * W), np.complex128)
    full[:, freqs] = before
    ref = oracle.diffuse(full.reshape(N, H, W), beta, T, 1000, freqs=freqs).reshape(N, -1)[:, freqs]
    err = rel_l2(after, ref)
    print(f"2048^2 N=64 beta={beta} flags={flags} sampled rel-L2 {err:.2e}")
    assert err <= REL_L2


def test_rejects_bad_arguments():
    plan = se2n.se2n_plan_create(8, 8, 16)
    v = t_c64(np.zeros((16, 8, 8)))
    for args, status in [((0.0, 1.0, 10), se2n.SE2N_EINVAL), ((-1.0, 1.0, 10), se2n.SE2N_EINVAL),
                         ((0.5, -1.0, 10), se2n.SE2N_EINVAL), ((0.5, 1.0, 0), se2n.SE2N_EINVAL),
                         ((1e6, 1e6, 1), se2n.SE2N_ENUMERIC), ((1e-40, 1.0, 1), se2n.SE2N_ENUMERIC)]:
        with pytest.raises(se2n.Se2nError) as e:
            se2n.se2n_diffuse(plan, v, *args)
        assert e.value.status == status, args
    host_buf = np.zeros((16, 8, 8), np.complex64)
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse(plan, host_buf, 0.5, 1.0, 10)
    assert e.value.status == se2n.SE2N_EINVAL
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse(plan, v.data_ptr() + 8, 0.5, 1.0, 10)   # misaligned
    assert e.value.status == se2n.SE2N_EINVAL
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse(plan, v, 0.5, 1.0, 10, 16)   # unknown flag
    assert e.value.status == se2n.SE2N_EINVAL
    # nothing was enqueued: the volume is untouched and the context healthy
    assert (host(v) == 0).all()
    plan.close()


def test_unsupported_and_invalid_plans():
    for H, W, N, status in [(7, 8, 16, se2n.SE2N_EINVAL), (8, 8, 2, se2n.SE2N_EINVAL),
                            (8, 8, 65, se2n.SE2N_EINVAL), (8, 8, 10, se2n.SE2N_EUNSUPPORTED)]:
        with pytest.raises(se2n.Se2nError) as e:
            se2n.se2n_plan_create(H, W, N)
        assert e.value.status == status
    plan = se2n.se2n_plan_create(8, 8, 30)
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_plan_tune_diffuse(plan, 4, 128, 0)
    assert e.value.status == se2n.SE2N_EUNSUPPORTED
    for block in (100, 416, -32):
        with pytest.raises(se2n.Se2nError) as e:
            se2n.se2n_plan_tune_diffuse(plan, 2, block, 0)
        assert e.value.status == se2n.SE2N_EINVAL
    plan.close()


@pytest.mark.parametrize("N,P", [(16, 1), (16, 2), (32, 2), (32, 4), (64, 4), (30, 2)])
@pytest.mark.parametrize("beta,T,S", [(0.25, 2.0, 500), (0.5, 2.0, 14), (1.0, 1.3, 20)])
def test_fast_path_equals_general_path_and_oracle(N, P, beta, T, S):
    """The packed fast path (truncated corner correction) against the
    general kernel (full correction) and the oracle. beta*dt = 1e-3, 0.0714
    (just past the truncation threshold, 0.0675: general kernel on both
    sides) and 0.065 (just inside it)."""
    vol = synth.random_volume(N, 26, 34, seed=N + P, dtype=np.complex64)
    ref = oracle.diffuse(vol.astype(np.complex128), beta, T, S)
    fast = _run(vol, N, beta, T, S, tune=(P, 128, 0))
    full = _run(vol, N, beta, T, S, flags=se2n.SE2N_DIFFUSE_FULL_CORRECTION, tune=(P, 128, 0))
    ef, eg = rel_l2(fast, ref), rel_l2(full, ref)
    print(f"N={N} P={P} beta*dt={beta * T / S:.4f}: fast {ef:.2e} general {eg:.2e}")
    assert ef <= REL_L2 and eg <= REL_L2
    assert rel_l2(fast, full) <= 2e-6
