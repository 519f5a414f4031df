"""se2n_diffuse_many_noalloc: the diffusion entry point for callers that
cannot let a library allocate device memory (an application that owns all
device memory through its own pool or arena, or a latency-critical loop that
cannot afford the synchronisation cudaMalloc may cause). It uses only the
caller's volumes and a fixed scratch array inside the library.

Checked through the C ABI against the per-volume entry point se2n_diffuse,
on two calls in a row (the scratch array keeps the previous call's contents,
so the second call shows that each call resets what it needs), and against
the FP64 oracle's Crank-Nicolson integration, so that a fault shared by both
GPU kernels cannot pass; a full call of SE2N_NOALLOC_MAX_VOLUMES volumes of
mixed N runs on a side stream with the 2 pi r / N angle grid. This file is
collected last so that a failure here does not stop the rest of a -x run.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from _gpu import REL_L2, host, rel_l2, t_c64

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")

SHAPES = [(64, 48, 16), (32, 32, 32), (40, 24, 64), (16, 16, 32), (48, 66, 16)]


def _reference(vol, beta, T, steps, angle_conv=0):
    N, H, W = vol.shape
    plan = se2n.se2n_plan_create(H, W, N, angle_conv)
    t = t_c64(vol)
    se2n.se2n_diffuse(plan, t, beta, T, steps)
    out = host(t)
    plan.close()
    return out


@pytest.mark.parametrize("beta,T,steps", [(0.25, 2.0, 100), (1.0, 10.0, 20)])
def test_noalloc_entry_point_matches_se2n_diffuse_on_two_calls_in_a_row(beta, T, steps):
    """beta*dt = 0.005 (packed fast path) and 0.5 (general kernel)."""
    for call in range(2):
        vols = [synth.random_volume(N, H, W, seed=100 * call + i, dtype=np.complex64)
                for i, (H, W, N) in enumerate(SHAPES[call:] + SHAPES[:call])]
        ref = [_reference(v, beta, T, steps) for v in vols]
        dev = [t_c64(v) for v in vols]
        se2n.se2n_diffuse_many_noalloc(dev, beta, T, steps)
        got = [host(t) for t in dev]
        for g, r in zip(got, ref):
            err = rel_l2(g, r)
            assert err <= REL_L2, (call, err)
        # and the FP64 oracle on the same FP32 inputs
        for g, v in zip(got, vols):
            exact = oracle.diffuse(v.astype(np.complex128), beta, T, steps)
            assert rel_l2(g, exact) <= REL_L2, (call, rel_l2(g, exact))


def test_noalloc_full_call_of_mixed_volumes_on_a_side_stream():
    """Exactly SE2N_NOALLOC_MAX_VOLUMES volumes of N = 16, 32 and 64 with
    uneven sizes, angles 2 pi r / N, on a non-default stream, twice in a row
    (the second call with the volumes in reverse order); each volume against
    se2n_diffuse and the FP64 oracle."""
    n = se2n.SE2N_NOALLOC_MAX_VOLUMES
    Ns = (16, 32, 64)
    shapes = [(2 * (2 + (7 * i) % 11), 2 * (3 + (5 * i) % 9), Ns[i % 3]) for i in range(n)]
    beta, T, steps = 0.25, 1.0, 40
    side = torch.cuda.Stream()
    for call in range(2):
        order = list(range(n)) if call == 0 else list(range(n))[::-1]
        vols = [synth.random_volume(N, H, W, seed=1000 * call + i, dtype=np.complex64)
                for i, (H, W, N) in enumerate(shapes)]
        dev = [t_c64(vols[i]) for i in order]
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            se2n.se2n_diffuse_many_noalloc(dev, beta, T, steps, angle_conv=1, stream=side)
        side.synchronize()
        for j, i in enumerate(order):
            got = host(dev[j])
            ref = _reference(vols[i], beta, T, steps, angle_conv=1)
            assert rel_l2(got, ref) <= REL_L2, (call, i, shapes[i], rel_l2(got, ref))
            exact = oracle.diffuse(vols[i].astype(np.complex128), beta, T, steps, angle_conv=1)
            assert rel_l2(got, exact) <= REL_L2, (call, i, shapes[i], rel_l2(got, exact))


def test_noalloc_rejects_requests_beyond_its_limits():
    small = t_c64(np.zeros((16, 4, 4), np.complex64))
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse_many_noalloc([small] * (se2n.SE2N_NOALLOC_MAX_VOLUMES + 1), 0.25, 1.0, 10)
    assert e.value.status == se2n.SE2N_EINVAL
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse_many_noalloc([], 0.25, 1.0, 10)
    assert e.value.status == se2n.SE2N_EINVAL
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse_many_noalloc([t_c64(np.zeros((30, 4, 4), np.complex64))], 0.25, 1.0, 10)
    assert e.value.status == se2n.SE2N_EUNSUPPORTED
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_diffuse_many_noalloc([small], 0.25, 1.0, 10, flags=se2n.SE2N_DIFFUSE_SM_FP64)
    assert e.value.status == se2n.SE2N_EINVAL
    # the wrapper checks the tensors before the C side sees them: a float32
    # volume of the same shape would be half the bytes the kernel touches
    with pytest.raises(ValueError):
        se2n.se2n_diffuse_many_noalloc([torch.zeros((16, 4, 4), dtype=torch.float32, device="cuda")], 0.25, 1.0, 10)
    with pytest.raises(ValueError):
        se2n.se2n_diffuse_many_noalloc([torch.zeros((16, 4, 4), dtype=torch.complex64)], 0.25, 1.0, 10)
    # the array keeps working after rejected calls
    v = synth.random_volume(16, 4, 4, seed=3, dtype=np.complex64)
    t = t_c64(v)
    se2n.se2n_diffuse_many_noalloc([t], 0.25, 1.0, 10)
    assert rel_l2(host(t), _reference(v, 0.25, 1.0, 10)) <= REL_L2
