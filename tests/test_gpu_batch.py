"""The batched path (se2n_batch_*): many images of uneven size and N
through one persistent diffusion launch per interval, captured in a CUDA
graph. Checked bitwise against the per-image path, against the oracle, and
for every autotuner candidate shape."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import MAX_REL, REL_L2, host, rel_l2, t_f32, t_u8

pytestmark = pytest.mark.gpu

se2n = pytest.importorskip("paper_1304_2062_gb300.se2n")

import torch  # noqa: E402

SHAPES = [(16, 24, 32), (32, 32, 16), (24, 16, 64), (48, 40, 32), (16, 16, 16), (40, 64, 64), (32, 48, 16)]


def _inputs(shapes, seed=0):
    out = []
    for i, (H, W, N) in enumerate(shapes):
        clean = synth.curves_noise_image(H, W, seed + i, n_curves=6)
        mask = synth.bernoulli_mask(H, W, seed + 100 + i, 0.7)
        out.append((clean * mask, mask, N))
    return out


def _params(steps=30, rounds=2, T=4.0):
    return se2n.se2n_params_default(beta=0.25, T=T, steps=steps, rounds=rounds, eps=0.5)


def _batch(inputs, prm, flags=0, bins=None):
    imgs = []
    for i, (f, m, N) in enumerate(inputs):
        H, W = f.shape
        out = torch.zeros((H, W), dtype=torch.float32, device="cuda")
        img = (t_f32(f.astype(np.float32)), t_u8(m), out, N)
        if bins is not None:
            img = img + (t_u8(bins[i]),)
        imgs.append(img)
    b = se2n.se2n_batch_create(imgs, prm, 0, flags)
    return b, [img[2] for img in imgs]


def test_batched_equals_per_image_bitwise_and_replays():
    inputs = _inputs(SHAPES)
    b, outs = _batch(inputs, _params())
    se2n.se2n_batch_run(b)
    first = [host(o).copy() for o in outs]
    se2n.se2n_batch_run(b)  # the graph replays to the same result
    second = [host(o).copy() for o in outs]
    for o in outs:
        o.zero_()
    se2n.se2n_batch_run_per_image(b)
    per = [host(o).copy() for o in outs]
    info = se2n.se2n_batch_get_info(b)
    b.close()
    for a, c, d in zip(first, second, per):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(a, d)
    assert info["images"] == len(SHAPES) and info["items"] > 0 and info["fast"] == 1


def test_batched_matches_oracle():
    inputs = _inputs(SHAPES, seed=50)
    T, S, R = 4.0, 30, 2
    bins = [oracle.orient(f.astype(np.float32).astype(np.float64), m, N)["bins"] for f, m, N in inputs]
    b, outs = _batch(inputs, _params(S, R, T), bins=bins)
    se2n.se2n_batch_run(b)
    got = [host(o).copy() for o in outs]
    b.close()
    for (f, m, N), bb, g in zip(inputs, bins, got):
        f64 = f.astype(np.float32).astype(np.float64)
        ref = oracle.inpaint(f64, m, oracle.Params(N=N, beta=0.25, T=T, steps=S, rounds=R), bins=bb)["out"]
        assert rel_l2(g, ref) <= REL_L2
        assert np.abs(g - ref).max() <= MAX_REL * np.abs(f64).max()


def test_autotuned_shape_gives_the_same_result():
    inputs = _inputs(SHAPES, seed=7)
    b0, o0 = _batch(inputs, _params())
    se2n.se2n_batch_run(b0)
    ref = [host(o).copy() for o in o0]
    b0.close()
    b1, o1 = _batch(inputs, _params(), flags=se2n.SE2N_BATCH_AUTOTUNE)
    se2n.se2n_batch_run(b1)
    info = se2n.se2n_batch_get_info(b1)
    got = [host(o).copy() for o in o1]
    b1.close()
    assert info["candidates"] == 12 and info["best_ms"] <= info["worst_ms"]
    assert info["tile_passes"] in (2, 8, 32) and info["block"] in (128, 256)
    # tile and block do not change any frequency's arithmetic; another table
    # of threads per frequency splits the angles differently (another torn
    # elimination), which is the same method to FP32 rounding
    same_split = (info["p16"], info["p32"], info["p64"]) == (1, 2, 4)
    for a, c in zip(ref, got):
        if same_split:
            np.testing.assert_array_equal(a, c)
        else:
            assert rel_l2(c, a) <= REL_L2


def test_general_kernel_batch_large_beta_dt():
    """beta*dt = 0.5 is past the truncation bound: the general kernel runs
    inside the persistent launch."""
    inputs = _inputs(SHAPES[:4], seed=9)
    prm = se2n.se2n_params_default(beta=1.0, T=10.0, steps=20, rounds=1)
    b, outs = _batch(inputs, prm)
    info = se2n.se2n_batch_get_info(b)
    se2n.se2n_batch_run(b)
    a = [host(o).copy() for o in outs]
    se2n.se2n_batch_run_per_image(b)
    c = [host(o).copy() for o in outs]
    b.close()
    assert info["fast"] == 0
    for x, y in zip(a, c):
        np.testing.assert_array_equal(x, y)


def test_batch_rejects_bad_input():
    f = t_f32(np.ones((8, 8)))
    m = t_u8(np.ones((8, 8)))
    o = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_batch_create([(f, m, o, 30)], _params())
    assert e.value.status == se2n.SE2N_EUNSUPPORTED
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_batch_create([], _params())
    assert e.value.status == se2n.SE2N_EINVAL
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_batch_create([(np.ones((8, 8), np.float32), m, o, 16)], _params())
    assert e.value.status == se2n.SE2N_EINVAL
    with pytest.raises(se2n.Se2nError) as e:
        se2n.se2n_batch_create([(f, m, o, 16)], _params(), flags=2)
    assert e.value.status == se2n.SE2N_EINVAL


@pytest.mark.parametrize("full", [0, 1])
def test_batch_with_propagators(full):
    """SE2N_DIFFUSE_PROPAGATOR in a batch: each distinct shape's propagators
    are built once in the graph and shared by its images (repeated shapes
    here); the graph replays bitwise, equals the per-image path bitwise and
    matches the oracle."""
    shapes = SHAPES + [(16, 24, 32), (32, 32, 16), (40, 64, 64), (64, 64, 16), (64, 64, 16), (64, 128, 32),
                       (64, 128, 32)]
    inputs = _inputs(shapes, seed=70)
    T, S, R = 4.0, 100, 4
    bins = [oracle.orient(f.astype(np.float32).astype(np.float64), m, N)["bins"] for f, m, N in inputs]
    prm = se2n.se2n_params_default(beta=0.25, T=T, steps=S, rounds=R, eps=0.5,
                                   diffuse_flags=se2n.SE2N_DIFFUSE_PROPAGATOR, full_spectrum=full)
    b, outs = _batch(inputs, prm, bins=bins)
    info = se2n.se2n_batch_get_info(b)
    se2n.se2n_batch_run(b)
    first = [host(o).copy() for o in outs]
    se2n.se2n_batch_run(b)
    second = [host(o).copy() for o in outs]
    for o in outs:
        o.zero_()
    se2n.se2n_batch_run_per_image(b)
    per = [host(o).copy() for o in outs]
    b.close()
    # 4 intervals of 100 steps: the cost estimate sends the small shapes to
    # propagators and the rest to the persistent step-by-step kernel; both
    # paths must be taken for the checks below to cover the mixed graph
    print(f"{info['prop_images']} of {info['images']} images by propagators, {info['fused_images']} of them on "
          "the row and column passes")
    assert 0 < info["prop_images"] < info["images"]
    # the 64 x 64 and 64 x 128 shapes take the row and column passes in the
    # graph (the Hermitian half only)
    assert info["fused_images"] == (0 if full else 4)
    for (f, m, N), bb, a, c, d in zip(inputs, bins, first, second, per):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(a, d)
        f64 = f.astype(np.float32).astype(np.float64)
        ref = oracle.inpaint(f64, m, oracle.Params(N=N, beta=0.25, T=T, steps=S, rounds=R), bins=bb)["out"]
        assert rel_l2(a, ref) <= REL_L2
        assert np.abs(a - ref).max() <= MAX_REL * np.abs(f64).max()
