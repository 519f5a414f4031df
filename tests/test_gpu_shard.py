"""The entry points that let one image spread over several GPUs, on one GPU:
se2n_diffuse_rows (the diffusion of a row shard of the spectrum) and
se2n_mix_given (the restoration of an angle shard given h(t) over all
angles), and the sharded method (paper_1304_2062_gb300/shard.py) with its
ranks emulated in one process, one after the other (no rank waits on
another's kernels), against the whole-volume path and the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu import MAX_REL, REL_L2, host, rel_l2, t_c64, t_f32, t_u8

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")
from paper_1304_2062_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("N,H,W,k0,rows", [(32, 64, 48, 16, 16), (16, 40, 40, 0, 40), (64, 24, 30, 23, 1)])
def test_row_shard_diffusion_is_bitwise_the_whole_volume(N, H, W, k0, rows):
    """Each frequency's system depends only on its own (k, l), so the rows
    k0 .. k0 + rows - 1 integrated alone give the bits of the whole-volume
    integration."""
    vol = synth.random_volume(N, H, W, seed=N + H + k0).astype(np.complex64)
    plan = se2n.se2n_plan_create(H, W, N)
    whole = t_c64(vol)
    se2n.se2n_diffuse(plan, whole, 0.25, 2.0, 40)
    part = t_c64(np.ascontiguousarray(vol[:, k0:k0 + rows]))
    se2n.se2n_diffuse_rows(plan, part, k0, 0.25, 2.0, 40)
    got, ref = host(part), host(whole)[:, k0:k0 + rows]
    plan.close()
    np.testing.assert_array_equal(got, ref)


def test_row_shard_rejects_rows_outside_the_plane():
    plan = se2n.se2n_plan_create(16, 16, 16)
    v = torch.zeros((16, 8, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(se2n.Se2nError):
        se2n.se2n_diffuse_rows(plan, v, 9, 0.25, 1.0, 10)
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse_rows(plan, v, 0, 0.25, 1.0, 10, se2n.SE2N_DIFFUSE_PROPAGATOR)
    assert e.value.status == se2n.SE2N_EUNSUPPORTED
    plan.close()


def test_restoration_with_given_maximum_is_bitwise_se2n_mix():
    """With h(t) taken over all the planes beforehand, the restoration of the
    whole volume and of each half of its planes (bins renumbered) give the
    bits of se2n_mix."""
    N, H, W = 32, 48, 64
    w = synth.workload_512(H=H, W=W, steps=10, rounds=2)
    f32 = w.f.astype(np.float32)
    bins = oracle.orient(f32.astype(np.float64), w.mask, N)["bins"]
    vol = synth.random_real_volume(N, H, W, seed=5).astype(np.complex64) * 0.3
    plan = se2n.se2n_plan_create(H, W, N)
    ref = t_c64(vol)
    se2n.se2n_mix(plan, ref, t_f32(f32), t_u8(w.mask), t_u8(bins), 0.5, 0.1)
    h_t = torch.empty((H, W), dtype=torch.float32, device="cuda")
    se2n.se2n_project(plan, t_c64(vol), se2n.SE2N_PROJ_MAX, h_t)
    half_plan = se2n.se2n_plan_create(H, W, N // 2)
    parts = []
    for p in range(2):
        v = t_c64(np.ascontiguousarray(vol[p * N // 2:(p + 1) * N // 2]))
        se2n.se2n_mix_given(half_plan, v, t_f32(f32), t_u8(w.mask), t_u8(shard.local_bins(bins, N, 2, p)), h_t, 0.5,
                            0.1)
        parts.append(host(v))
    got = np.concatenate(parts, axis=0)
    expect = host(ref)
    plan.close()
    half_plan.close()
    np.testing.assert_array_equal(got, expect)


@pytest.mark.parametrize("P", [2, 4])
def test_sharded_inpaint_on_one_gpu_matches_the_whole_path_and_the_oracle(P):
    N, H, W = 32, 96, 64
    w = synth.workload_512(H=H, W=W, steps=40, rounds=3)
    f32 = w.f.astype(np.float32)
    f64 = f32.astype(np.float64)
    bins = oracle.orient(f64, w.mask, N)["bins"]
    prm = shard.ShardParams(N=N, beta=0.25, T=6.0, steps=40, rounds=3)
    backend = shard.GpuBackend(H, W, N, P, list(range(P)))
    outs = shard.inpaint_sharded(backend, shard.LocalExchange(P), f32, w.mask, bins, prm)
    got = [host(outs[p]) for p in range(P)]
    backend.close()
    # the whole volume on the complex (full-spectrum) path, step by step
    plan = se2n.se2n_plan_create(H, W, N)
    vol = torch.empty((N, H, W), dtype=torch.complex64, device="cuda")
    out = torch.empty((H, W), dtype=torch.float32, device="cuda")
    p_all = se2n.se2n_params_default(N=N, beta=0.25, T=6.0, steps=40, rounds=3, eps=0.5, full_spectrum=1)
    se2n.se2n_inpaint(plan, t_f32(f32), t_u8(w.mask), t_u8(bins), p_all, vol, out)
    whole = host(out)
    plan.close()
    ref = oracle.inpaint(f64, w.mask, oracle.Params(N=N, beta=0.25, T=6.0, steps=40, rounds=3), bins=bins)["out"]
    for g in got:
        np.testing.assert_array_equal(g, got[0])   # every rank holds the same image
    print(f"P={P}: vs whole path rel-L2 {rel_l2(got[0], whole):.2e}, vs oracle rel-L2 {rel_l2(got[0], ref):.2e}, "
          f"max-abs {np.abs(got[0] - ref).max() / np.abs(f64).max():.2e}")
    assert rel_l2(got[0], whole) <= 1e-6
    assert rel_l2(got[0], ref) <= REL_L2
    assert np.abs(got[0] - ref).max() <= MAX_REL * np.abs(f64).max()
