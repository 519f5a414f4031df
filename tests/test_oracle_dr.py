"""Pins of the oracle's dynamic restoration (Section 5.3): the growth step of
the good set checked on hand-worked examples, by brute force, by symmetry,
and in the whole method against the cases where it must reduce to static
restoration."""
import numpy as np
import pytest

import oracle
import synth


def _vol_from_image(h, N=3, seed=0):
    """A real volume whose maximum over angles is h, reached first at a
    random angle; the other angles hold smaller values."""
    rng = np.random.default_rng(seed)
    H, W = h.shape
    at = rng.integers(0, N, size=(H, W))
    vol = h[None] - 1.0 - rng.random((N, H, W))
    vol[at, np.arange(H)[:, None], np.arange(W)[None, :]] = h
    return vol, at


def test_hand_worked_step_on_a_vertical_edge():
    """Good columns 0-1, bad columns 2-4. Only column 2 touches G. Its four
    pixels have 3x3 means over the bad pixels of columns 2-3 (worked out by
    hand below); (1, 4) is large but not on the boundary."""
    mask = np.array([[1, 1, 0, 0, 0]] * 4, dtype=np.uint8)
    h = np.array([[7.0, 7.0, 0.9, 0.1, 0.1],
                  [7.0, 7.0, 0.1, 0.1, 0.95],
                  [7.0, 7.0, 0.1, 0.1, 0.1],
                  [7.0, 7.0, 0.3, 0.3, 0.3]])
    # (0,2): {0.9, 0.1, 0.1, 0.1} mean 0.3        -> 0.9 > 0.3   joins
    # (1,2): {0.9, 0.1, 0.1, 0.1, 0.1, 0.1} 0.233 -> 0.1         stays bad
    # (2,2): {0.1, 0.1, 0.1, 0.1, 0.3, 0.3} 0.167 -> 0.1         stays bad
    # (3,2): {0.1, 0.1, 0.3, 0.3} mean 0.2        -> 0.3 > 0.2   joins
    vol, at = _vol_from_image(h)
    fref = np.where(mask != 0, 2.0, 0.0)
    bins = np.full(h.shape, 9, dtype=np.uint8)
    m1, f1, b1 = oracle.dr_grow(vol, mask, fref, bins)
    want = mask.copy()
    want[0, 2] = want[3, 2] = 1
    assert np.array_equal(m1, want)
    assert f1[0, 2] == 0.9 and f1[3, 2] == 0.3
    assert b1[0, 2] == at[0, 2] and b1[3, 2] == at[3, 2]
    unchanged = want == mask
    assert np.array_equal(f1[unchanged], fref[unchanged])
    assert np.array_equal(b1[unchanged], bins[unchanged])
    # the closest decision: (2,2) at |0.1 - 1/6|
    *_, margin = oracle.dr_grow(vol, mask, fref, bins, return_margin=True)
    assert margin.min() == pytest.approx(1.0 / 6.0 - 0.1, rel=1e-12)
    assert np.isfinite(margin).sum() == 4 and np.all(np.isfinite(margin[:, 2]))


def test_diagonal_neighbour_counts_and_good_values_are_excluded():
    """Only (0, 0) is good (with a huge value that must not enter any mean).
    (1, 1) touches it diagonally: mean over its 8 bad neighbours and itself
    (7 x 0.1 + 0.8) / 8 = 0.1875 < 0.8, it joins. (0, 1): (4 x 0.1 + 0.8) / 5
    = 0.24 > 0.1, it does not; (0, 2) and the rest do not touch G."""
    mask = np.zeros((3, 3), dtype=np.uint8)
    mask[0, 0] = 1
    h = np.full((3, 3), 0.1)
    h[0, 0] = 50.0
    h[1, 1] = 0.8
    vol, _ = _vol_from_image(h, seed=1)
    m1, _, _ = oracle.dr_grow(vol, mask, np.zeros((3, 3)), np.zeros((3, 3), np.uint8))
    want = np.zeros((3, 3), dtype=np.uint8)
    want[0, 0] = want[1, 1] = 1
    assert np.array_equal(m1, want)


def test_comparison_is_strict():
    """A flat bad region equals its own mean: nothing joins."""
    mask = np.zeros((6, 7), dtype=np.uint8)
    mask[:, :2] = 1
    h = np.where(mask != 0, 3.0, 0.25)
    vol, _ = _vol_from_image(h, seed=2)
    m1, _, _ = oracle.dr_grow(vol, mask, np.zeros(h.shape), np.zeros(h.shape, np.uint8))
    assert np.array_equal(m1, mask)
    h[2, 2] = np.nextafter(0.25, 1.0) + 1e-12     # just above: exactly this pixel joins
    vol, _ = _vol_from_image(h, seed=2)
    m1, _, _ = oracle.dr_grow(vol, mask, np.zeros(h.shape), np.zeros(h.shape, np.uint8))
    assert m1.sum() == mask.sum() + 1 and m1[2, 2] == 1


def test_a_lone_bad_pixel_never_joins_and_has_no_margin():
    """Every neighbour good: the mean is h itself and h > h is false."""
    mask = np.ones((3, 3), dtype=np.uint8)
    mask[1, 1] = 0
    h = np.full((3, 3), 0.1)
    h[1, 1] = 9.0
    vol, _ = _vol_from_image(h, seed=3)
    m1, _, _, margin = oracle.dr_grow(vol, mask, np.zeros((3, 3)), np.zeros((3, 3), np.uint8), return_margin=True)
    assert np.array_equal(m1, mask) and np.all(np.isinf(margin))


def test_first_maximum_gives_the_bin():
    """(0, 1) joins (0.7 > (0.7 + 0.1) / 2); its largest value is tied
    between angles 1 and 2 and the first one is taken."""
    vol = np.zeros((4, 1, 3))
    vol[:, 0, 0] = -5.0
    vol[:, 0, 1] = [0.2, 0.7, 0.7, 0.1]
    vol[:, 0, 2] = [0.1, 0.0, 0.0, 0.0]
    mask = np.array([[1, 0, 0]], dtype=np.uint8)
    m1, f1, b1 = oracle.dr_grow(vol, mask, np.zeros((1, 3)), np.zeros((1, 3), np.uint8))
    assert list(m1[0]) == [1, 1, 0] and f1[0, 1] == 0.7 and b1[0, 1] == 1


def _brute_force(h, mask):
    H, W = h.shape
    out = (mask != 0).astype(np.uint8)
    for y in range(H):
        for x in range(W):
            if mask[y, x]:
                continue
            vals, touches = [], False
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W:
                        if mask[yy, xx]:
                            touches = True
                        else:
                            vals.append(h[yy, xx])
            if touches and h[y, x] > sum(vals) / len(vals):
                out[y, x] = 1
    return out


@pytest.mark.parametrize("seed", range(6))
def test_matches_brute_force_and_only_grows(seed):
    rng = np.random.default_rng(100 + seed)
    H, W = rng.integers(3, 14, size=2)
    mask = (rng.random((H, W)) < 0.4).astype(np.uint8)
    vol = rng.normal(size=(5, H, W))
    fref = rng.random((H, W))
    bins = rng.integers(0, 5, size=(H, W)).astype(np.uint8)
    m1, f1, b1 = oracle.dr_grow(vol, mask, fref, bins)
    assert np.array_equal(m1, _brute_force(vol.max(axis=0), mask))
    assert np.all(m1[mask != 0] == 1)                       # G only grows
    kept = mask != 0
    assert np.array_equal(f1[kept], fref[kept]) and np.array_equal(b1[kept], bins[kept])
    joined = (m1 != 0) & (mask == 0)
    assert np.array_equal(f1[joined], vol.max(axis=0)[joined])
    assert np.array_equal(b1[joined], np.argmax(vol, axis=0)[joined])


@pytest.mark.parametrize("op", ["flipud", "fliplr", "transpose"])
def test_equivariant_under_flips_and_transpose(op):
    """Neighbourhoods are symmetric: flipping or transposing the inputs flips
    or transposes the result (catches a wrong offset or swapped axis)."""
    rng = np.random.default_rng(7)
    mask = (rng.random((11, 9)) < 0.35).astype(np.uint8)
    vol = rng.normal(size=(4, 11, 9))
    z = np.zeros((11, 9))
    zb = np.zeros((11, 9), np.uint8)
    g = {"flipud": lambda a: a[..., ::-1, :], "fliplr": lambda a: a[..., :, ::-1],
         "transpose": lambda a: np.swapaxes(a, -1, -2)}[op]
    m1, _, _ = oracle.dr_grow(vol, mask, z, zb)
    m2, _, _ = oracle.dr_grow(g(vol), g(mask), g(z), g(zb))
    assert np.array_equal(g(m1), m2)


def test_float32_mode_agrees_away_from_ties():
    rng = np.random.default_rng(8)
    mask = (rng.random((40, 40)) < 0.5).astype(np.uint8)
    vol = rng.normal(size=(6, 40, 40))
    z, zb = np.zeros((40, 40)), np.zeros((40, 40), np.uint8)
    m64, _, _ = oracle.dr_grow(vol, mask, z, zb)
    m32, _, _ = oracle.dr_grow(vol, mask, z, zb, dtype=np.float32)
    assert np.array_equal(m64, m32)


def _small(**kw):
    w = synth.workload_small()
    base = dict(N=w.N, beta=w.beta, T=w.T, steps=20, rounds=4, eps=w.eps)
    base.update(kw)
    return w, oracle.Params(**base)


def test_dynamic_reduces_to_static_when_eps_is_zero():
    """eps = 0 makes every restoration the identity, whatever the good set."""
    w, p = _small(eps=0.0)
    a = oracle.inpaint(w.f, w.mask, p)
    b = oracle.inpaint(w.f, w.mask, oracle.Params(**{**p.__dict__, "dynamic": 1}))
    assert np.array_equal(a["out"], b["out"])
    assert b["mask_final"].sum() > (w.mask != 0).sum()       # the set did grow


def test_dynamic_reduces_to_static_without_corrupted_pixels():
    w, p = _small()
    ones = np.ones_like(w.mask)
    a = oracle.inpaint(w.f, ones, p)
    b = oracle.inpaint(w.f, ones, oracle.Params(**{**p.__dict__, "dynamic": 1}))
    assert np.array_equal(a["out"], b["out"])


def test_dynamic_reduces_to_static_with_one_interval():
    w, p = _small(rounds=1)
    a = oracle.inpaint(w.f, w.mask, p)
    b = oracle.inpaint(w.f, w.mask, oracle.Params(**{**p.__dict__, "dynamic": 1}))
    assert np.array_equal(a["out"], b["out"])
    assert np.array_equal(b["mask_final"], (w.mask != 0).astype(np.uint8))


def test_dynamic_changes_the_result_and_grows_monotonically():
    w, p = _small()
    a = oracle.inpaint(w.f, w.mask, p)
    pd = oracle.Params(**{**p.__dict__, "dynamic": 1})
    b = oracle.inpaint(w.f, w.mask, pd)
    grown = b["mask_final"]
    assert np.all(grown[w.mask != 0] == 1)
    assert grown.sum() > (w.mask != 0).sum()
    assert not np.allclose(a["out"], b["out"])
