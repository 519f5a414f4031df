"""The index logic of the tiled propagator apply at N = 64
(propagator.cu, k_prop_apply_tiled), checked on the host from the constants
in the source:

- the blocks' tiles (one row slot times CT column slots, square planes in
  super-tiles of SUPER x SUPER classes, each followed by its transpose)
  cover every class of the Hermitian half exactly once;
- a class's shared-memory slots ([N slots][8 frequencies] complex, swizzled
  by the class and the slot) are a bijection onto its region, every 16-byte
  unit holds the two frequencies of one m-pair, the 16 lanes of a staging
  run fall on 16 different pairs of banks and the eight rows 4 rb + c that a
  quarter-warp updates at the end on eight different groups of four;
- a transposed class (row slot > column slot) applies the propagator of its
  transpose through the angle slots: x + P D P x read back from the slots
  equals the direct product, for both reflections (perm_shift N/2, N/4) and
  with the reversal of rows H/2 + s and H - s."""
import math
import os
import re

import numpy as np

N = 64
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1304_2062_gb300", "csrc", "propagator.cu")


def _constants():
    text = open(SRC).read()
    body = text[text.index("struct TileCfg {"):]
    ct = int(re.search(r"static constexpr int CT = (\d+);", body).group(1))
    sup = int(re.search(r"static constexpr int SUPER = (\d+);", body).group(1))
    return ct, sup


def _tile_of_block(b, H, W, share, CT, SUPER):
    n, nr = W // 4 + 1, H // 4 + 1
    if not share:
        tr = (n + CT - 1) // CT
        srow = b // tr
        return srow < nr, srow, (b - srow * tr) * CT
    per = SUPER * (SUPER // CT)
    sg, w = divmod(b, per)
    J = math.isqrt(sg)
    p = sg - J * J
    R = C = J
    if p < 2 * J:
        if p & 1:
            C = p >> 1
        else:
            R = p >> 1
    srow = R * SUPER + w // (SUPER // CT)
    c0 = C * SUPER + (w % (SUPER // CT)) * CT
    return srow < nr and c0 < n, srow, c0


def _blocks(H, W, share, CT, SUPER):
    n, nr = W // 4 + 1, H // 4 + 1
    if not share:
        return nr * ((n + CT - 1) // CT)
    sb = (n + SUPER - 1) // SUPER
    return sb * sb * SUPER * (SUPER // CT)


def _xrow(a, h):
    return a ^ h ^ ((a >> 2) & 1)


def _xunit(a, u):
    return u ^ ((a >> 3) & 3)


def _xpos(a, m, h, mm):
    return _xrow(a, h) * 16 + 4 * _xunit(a, (m ^ mm) >> 1) + 2 * ((m ^ mm) & 1)


def _slot_rows(s, H):
    quarter = 4 * s == H
    return [s, H // 2 - s, H // 2 + s, (H - s) % H], [True, not quarter, s != 0, s != 0 and not quarter]


def test_tiles_cover_every_class_once():
    CT, SUPER = _constants()
    for H, W, share in [(136, 136, True), (72, 72, True), (22, 22, True), (20, 20, True), (72, 136, False),
                        (136, 72, False), (26, 18, False), (1024, 1024, True)]:
        n, nr = W // 4 + 1, H // 4 + 1
        seen = np.zeros((nr, n), int)
        for b in range(_blocks(H, W, share, CT, SUPER)):
            ok, srow, c0 = _tile_of_block(b, H, W, share, CT, SUPER)
            if ok:
                for q in range(CT):
                    if c0 + q < n:
                        seen[srow, c0 + q] += 1
        assert (seen == 1).all(), (H, W)


def test_transpose_follows_its_super_tile():
    """Each super-tile above the diagonal is followed at once by its transpose."""
    CT, SUPER = _constants()
    H = W = 1024
    per = SUPER * (SUPER // CT)
    order = {}
    for b in range(_blocks(H, W, True, CT, SUPER)):
        ok, srow, c0 = _tile_of_block(b, H, W, True, CT, SUPER)
        order.setdefault((srow // SUPER, c0 // SUPER), b // per)
    for (I, J), sg in order.items():
        if I < J:
            assert order[(J, I)] == sg + 1


def test_class_slots_are_a_bijection_with_paired_units():
    for q in range(16):
        qh, qm = (q >> 3) & 1, q & 7
        pos = [_xpos(a, m, qh, qm) for a in range(N) for m in range(8)]
        assert sorted(pos) == list(range(0, 16 * N, 2))
        for a in range(N):
            for mp in range(4):
                # frequencies 2 mp and 2 mp + 1 of a slot share one 16-byte unit
                u0, u1 = _xpos(a, 2 * mp, qh, qm) // 4, _xpos(a, 2 * mp + 1, qh, qm) // 4
                assert u0 == u1 == _xrow(a, qh) * 4 + _xunit(a, mp ^ (qm >> 1))


def test_staging_and_row_updates_are_free_of_bank_conflicts():
    QF = 16 * N
    for a in range(N):
        for m in range(8):
            banks = [(q * QF + _xpos(a, m, (q >> 3) & 1, q & 7)) % 32 for q in range(16)]
            assert len(set(banks)) == 16
    for ch in (0, 1):
        for cm in range(8):
            for mp in range(4):
                uu = mp ^ (cm >> 1)
                for h in range(2):
                    for p in range(2):
                        for o in range(2):
                            groups = {((_xrow(row, ch) * 16 + 4 * _xunit(row, uu)) % 32) // 4
                                      for row in (4 * (rb + 8 * h) + 2 * p + o for rb in range(8))}
                            assert len(groups) == 8


def test_transposed_classes_through_permuted_slots():
    """x + P D P x (rows 0, 1) and x + R P D P R x (rows 2, 3) of a
    transposed class, computed as the kernel does it (slot of angle r, the
    product in slot space with the transpose's D, read back by slot), equal
    the products formed directly."""
    rng = np.random.default_rng(5)
    D = rng.standard_normal((N, N))
    D = D + D.T
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Rv = np.zeros((N, N))
    Rv[np.arange(N), (-np.arange(N)) % N] = 1
    for sh in (N // 2, N // 4):
        P = np.zeros((N, N))
        P[np.arange(N), (sh - np.arange(N)) % N] = 1
        for mk in range(4):
            for tq in (False, True):
                neg = (mk >= 2) != tq
                slot = [((sh if tq else 0) + (-r if neg else r)) % N for r in range(N)]
                z = np.zeros(N, complex)
                z[slot] = x
                w = z + D @ z
                got = w[slot]
                A = D if not tq else P @ D @ P
                if mk >= 2:
                    A = Rv @ A @ Rv
                np.testing.assert_allclose(got, x + A @ x, rtol=1e-12, atol=1e-12)
