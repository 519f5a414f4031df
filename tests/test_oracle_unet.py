"""Pins of the FP64 surrogate-network reference (oracle/unet.py): the
convolution against scipy's correlation, the pooling and upsampling against
their definitions, and the whole backward pass against central finite
differences of the loss."""
import numpy as np
import pytest
from scipy import signal

from oracle import unet


def test_conv3x3_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    W = rng.standard_normal((4, 9, 3))
    b = rng.standard_normal(4)
    y = unet.conv3x3(x, W, b)
    for bb in range(2):
        for co in range(4):
            ref = b[co]
            for ci in range(3):
                k = W[co, :, ci].reshape(3, 3)   # tap = (dy+1)*3 + (dx+1): rows dy, columns dx
                ref = ref + signal.correlate2d(x[bb, :, :, ci], k, mode="same", boundary="fill")
            np.testing.assert_allclose(y[bb, :, :, co], ref, atol=1e-12)


def test_pool_and_upsample_definitions():
    x = np.arange(2 * 4 * 6 * 3, dtype=float).reshape(2, 4, 6, 3)
    p = unet.pool(x)
    assert p.shape == (2, 2, 3, 3)
    np.testing.assert_allclose(p[1, 1, 2, 0], x[1, 2:4, 4:6, 0].mean())
    u = unet.up(p)
    np.testing.assert_array_equal(u[:, 0::2, 0::2], p)
    np.testing.assert_array_equal(u[:, 1::2, 1::2], p)
    # adjoints: <pool(x), g> = <x, pool_backward(g)>, <up(y), g> = <y, up_backward(g)>
    rng = np.random.default_rng(1)
    g = rng.standard_normal(p.shape)
    assert abs((p * g).sum() - (x * unet.pool_backward(g)).sum()) < 1e-9
    g2 = rng.standard_normal(u.shape)
    assert abs((u * g2).sum() - (p * unet.up_backward(g2)).sum()) < 1e-9


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 65504.0, 1e-30])
    r = unet.bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0  # a tie rounds to even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] - (-3.140625)) < 1e-12
    assert (np.abs(r - v) <= np.abs(v) * 2 ** -8 + 1e-300).all()


def test_parameter_layout():
    offs, hw, hb, n = unet.layout()
    assert n == hb + 1 and hw == hb - 32
    assert offs[0] == (0, 32 * 9 * 8)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    B, H, W = 1, 8, 8
    p = unet.he_params(seed)
    f = rng.uniform(0.05, 1.0, (B, H, W))
    mask = (rng.random((B, H, W)) > 0.4).astype(np.uint8)
    target = rng.uniform(0.0, 1.0, (B, H, W))
    loss, g = unet.loss_and_grads(p, f, mask, target)
    offs, hw, hb, n = unet.layout()
    idx = []
    for (w, b), (cin, cout, _) in zip(offs, unet.LAYERS):
        idx += [w + int(rng.integers(cout * 9 * min(cin, 2 if cin == 8 else cin))), b + int(rng.integers(cout))]
    idx += [hw + 3, hb]
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        lp = unet.loss_and_grads(p + e, f, mask, target)[0]
        lm = unet.loss_and_grads(p - e, f, mask, target)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
