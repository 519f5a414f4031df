"""FP64 reference of the surrogate U-Net. TEST INFRASTRUCTURE ONLY (the
tests may import it; the CUDA library never does).

The network the library trains (not part of the paper): 3x3 convolutions
with padding 1 and ReLU, 2x2 average pooling, nearest upsampling,
channel concatenation of the upsampled lower level and the skip
connection, a 1x1 head to one channel added to the masked input
(out = f (mask != 0) + head), and the loss mean((out - target)^2).
Layers and the flat parameter layout are those of the C ABI (se2n_unet_*):
for each of the 14 conv layers W[cout][9][cin] then b[cout], then the head
w[32], b[1]; tap = (dy+1)*3 + (dx+1).

Everything here is written from the definitions: a convolution is the sum
over its 9 taps of shifted inputs times the tap's weight matrix; its
backward passes are the adjoint sums. Pinned by finite differences
(tests/test_oracle_unet.py).
"""
from __future__ import annotations

import numpy as np

# (cin, cout, upsampled channels of the concatenated input)
LAYERS = [
    (8, 32, 0), (32, 32, 0), (32, 64, 0), (64, 64, 0), (64, 128, 0), (128, 128, 0), (128, 256, 0), (256, 256, 0),
    (384, 128, 256), (128, 128, 0), (192, 64, 128), (64, 64, 0), (96, 32, 64), (32, 32, 0),
]


def layout():
    """Offsets (w_off, b_off) per layer, head offsets and the total count."""
    offs, o = [], 0
    for cin, cout, _ in LAYERS:
        w = o
        o += cout * 9 * cin
        b = o
        o += cout
        offs.append((w, b))
    hw = o
    o += 32
    hb = o
    o += 1
    return offs, hw, hb, o


def unpack(params):
    offs, hw, hb, n = layout()
    assert params.size == n
    Ws, bs = [], []
    for (cin, cout, _), (w, b) in zip(LAYERS, offs):
        Ws.append(params[w:w + cout * 9 * cin].reshape(cout, 9, cin))
        bs.append(params[b:b + cout])
    return Ws, bs, params[hw:hw + 32], params[hb]


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, W, b):
    """x [B,H,W,Cin], W [Cout,9,Cin], b [Cout] -> [B,H,W,Cout] (padding 1)."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[0]))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        y += xp[:, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd, :] @ W[:, tap, :].T
    return y + b


def conv3x3_backward(x, W, gz):
    """Gradients of sum(gz * conv3x3(x, W, b)) w.r.t. x, W and b."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        sl = (slice(None), slice(1 + dy, 1 + dy + H), slice(1 + dx, 1 + dx + Wd), slice(None))
        gW[:, tap, :] = np.einsum("bhwo,bhwi->oi", gz, xp[sl])
        gxp[sl] += gz @ W[:, tap, :]
    return gxp[:, 1:-1, 1:-1, :], gW, gz.sum(axis=(0, 1, 2))


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def pack_input(f, mask):
    """[B,H,W] image and mask -> [B,H,W,8]: f*(mask!=0), mask, six zeros."""
    m = (np.asarray(mask) != 0).astype(np.float64)
    x = np.zeros(m.shape + (8,))
    x[..., 0] = np.asarray(f, dtype=np.float64) * m
    x[..., 1] = m
    return x


def forward(params, f, mask, bf16=False):
    """Forward pass. With bf16=True every stored activation is rounded to
    bfloat16 where a bfloat16 implementation stores it (conv outputs after
    bias and ReLU, pooled outputs, the packed input); arithmetic stays FP64.
    The ReLU masks are then taken on the rounded outputs."""
    Ws, bs, hw, hb = unpack(np.asarray(params, dtype=np.float64))
    q = bf16_round if bf16 else (lambda v: v)
    x0 = q(pack_input(f, mask))
    cache = {"x0": x0, "z": [None] * 14, "in": [None] * 14, "act": [None] * 14, "bf16": bf16}
    relu = lambda z: np.maximum(z, 0.0)
    e, h = [], x0
    for l in range(4):
        if l > 0:
            h = q(pool(e[l - 1]))
        cache["in"][2 * l] = h
        cache["z"][2 * l] = conv3x3(h, Ws[2 * l], bs[2 * l])
        a = q(relu(cache["z"][2 * l]))
        cache["act"][2 * l] = a
        cache["in"][2 * l + 1] = a
        cache["z"][2 * l + 1] = conv3x3(a, Ws[2 * l + 1], bs[2 * l + 1])
        e.append(q(relu(cache["z"][2 * l + 1])))
        cache["act"][2 * l + 1] = e[-1]
    below = e[3]
    for k in range(3):
        level = 2 - k
        la, lb = 8 + 2 * k, 9 + 2 * k
        xin = np.concatenate([up(below), e[level]], axis=-1)
        cache["in"][la] = xin
        cache["z"][la] = conv3x3(xin, Ws[la], bs[la])
        c = q(relu(cache["z"][la]))
        cache["act"][la] = c
        cache["in"][lb] = c
        cache["z"][lb] = conv3x3(c, Ws[lb], bs[lb])
        below = q(relu(cache["z"][lb]))
        cache["act"][lb] = below
    d0 = below
    out = d0 @ hw + hb + np.asarray(f, dtype=np.float64) * (np.asarray(mask) != 0)
    cache["d0"] = d0
    cache["e"] = e
    return out, cache


def loss_and_grads(params, f, mask, target, bf16=False):
    """mean((out - target)^2) and its gradient w.r.t. the flat parameters.
    With bf16=True the activation gradients are also rounded to bfloat16
    where a bfloat16 implementation stores them (after each masking, each
    data-gradient, each pooling/upsampling adjoint), and the ReLU masks use
    the rounded activations."""
    params = np.asarray(params, dtype=np.float64)
    Ws, bs, hw, hb = unpack(params)
    out, cache = forward(params, f, mask, bf16)
    q = bf16_round if bf16 else (lambda v: v)
    r = out - np.asarray(target, dtype=np.float64)
    loss = np.mean(r ** 2)
    gout = 2.0 * r / r.size
    offs, o_hw, o_hb, n = layout()
    g = np.zeros(n)
    g[o_hw:o_hw + 32] = np.einsum("bhw,bhwc->c", gout, cache["d0"])
    g[o_hb] = gout.sum()
    act = cache["act"]
    relu_mask = lambda layer: (act[layer] > 0).astype(np.float64) if bf16 else (cache["z"][layer] > 0).astype(np.float64)

    def conv_back(layer, gz):
        gx, gW, gb = conv3x3_backward(cache["in"][layer], Ws[layer], gz)
        w, b = offs[layer]
        g[w:w + gW.size] = gW.ravel()
        g[b:b + gb.size] = gb
        return gx

    gz = q(gout[..., None] * hw[None, None, None, :] * relu_mask(13))
    gskip = [None] * 3
    for k in (2, 1, 0):
        la, lb = 8 + 2 * k, 9 + 2 * k
        gc = conv_back(lb, gz)
        gz = q(gc * relu_mask(la))
        gin = conv_back(la, gz)
        lo = LAYERS[la][2]
        gup, gskip[k] = q(gin[..., :lo]), q(gin[..., lo:])
        below_layer = 9 + 2 * (k - 1) if k > 0 else 7
        gz = q(up_backward(gup) * relu_mask(below_layer))
    for l in (3, 2, 1, 0):
        if l < 3:
            gz = q((pool_backward(gp) + gskip[2 - l]) * relu_mask(2 * l + 1))
        ga = conv_back(2 * l + 1, gz)
        gz = q(ga * relu_mask(2 * l))
        gp = q(conv_back(2 * l, gz))
    return loss, g


def he_params(seed):
    """He-normal parameters (numpy generator; the library has its own)."""
    rng = np.random.default_rng(seed)
    offs, hw, hb, n = layout()
    p = np.zeros(n)
    for (cin, cout, _), (w, b) in zip(LAYERS, offs):
        fan = 9 * (2 if cin == 8 else cin)
        p[w:w + cout * 9 * cin] = rng.standard_normal(cout * 9 * cin) * np.sqrt(2.0 / fan)
        p[b:b + cout] = rng.standard_normal(cout) * 0.05
    p[hw:hw + 32] = rng.standard_normal(32) * np.sqrt(1.0 / 32)
    p[hb] = 0.1
    return p
