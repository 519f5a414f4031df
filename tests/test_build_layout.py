"""The shared-memory layout of the symmetric propagator build at N = 32
(propagator.cu, SymCfg<32>), checked on the host from the constants in the
source: element (i, j) of a class's matrix sits at
i LD + ((j + SKEW(i / 8)) mod 32), lane t of a class computes the 8 x 8 tile
TILE[t] of the upper triangle, and three classes share a warp with bases
CLASS_FLOATS apart. The layout must be a bijection within each row that
keeps 16-byte vectors contiguous, the tiles must cover the upper triangle
once, and every quarter-warp (the 8 lanes a 16-byte shared access serves
together) must touch 8 different groups of 4 banks in each access of a
product: the k steps (row k of A and of B), the tile's own rows (the loads
of X and Y and the stores) and the mirrored rows (the stores of the
transposed tile)."""
import os
import re

N, LD, TILES, CPW = 32, 36, 10, 3
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1304_2062_gb300", "csrc", "propagator.cu")


def _constants():
    text = open(SRC).read()
    skew = int(re.search(r"N == 32 \? \((0x[0-9A-Fa-f]+)u >> \(8 \* b\)\)", text).group(1), 16)
    tile = int(re.search(r"\((0x[0-9A-Fa-f]+)ULL >> \(4 \* \(t < 10", text).group(1), 16)
    return [(skew >> (8 * b)) & 0xFF for b in range(4)], [(tile >> (4 * t)) & 0xF for t in range(TILES)]


def _at(skew, i, j):
    return i * LD + ((j + skew[i >> 3]) & (N - 1))


def test_layout_is_a_row_bijection_with_contiguous_vectors():
    skew, _ = _constants()
    assert all(s % 4 == 0 for s in skew)
    for i in range(N):
        pos = sorted(_at(skew, i, j) for j in range(N))
        assert pos == list(range(i * LD, i * LD + N))
        for j in range(0, N, 4):
            assert [_at(skew, i, j + q) for q in range(4)] == [_at(skew, i, j) + q for q in range(4)]
            assert _at(skew, i, j) % 4 == 0


def test_tiles_cover_the_upper_triangle_once():
    _, tile = _constants()
    assert sorted((v >> 2, v & 3) for v in tile) == [(bi, bj) for bi in range(4) for bj in range(bi, 4)]


def test_every_quarter_warp_access_is_free_of_bank_conflicts():
    skew, tile = _constants()
    class_floats = 2 * N * LD + 2 * N + 4
    assert class_floats % 32 == 4
    lanes = [(g, tile[t] >> 2, tile[t] & 3) for g in range(CPW) for t in range(TILES)]

    def wavefronts(addresses):
        # distinct 16-byte addresses per group of 4 banks; 1 = conflict-free
        groups = {}
        for a in addresses:
            groups.setdefault((a // 4) % 8, set()).add(a)
        return max(len(v) for v in groups.values())

    for phase in range(4):
        quarter = lanes[8 * phase:8 * phase + 8]
        for half in (0, 4):
            for k in range(N):
                a_rows = [g * class_floats + _at(skew, k, 8 * bi + half) for g, bi, _ in quarter]
                b_rows = [g * class_floats + _at(skew, k, 8 * bj + half) for g, _, bj in quarter]
                assert wavefronts(a_rows) == 1 and wavefronts(b_rows) == 1
            for r in range(8):
                own = [g * class_floats + _at(skew, 8 * bi + r, 8 * bj + half) for g, bi, bj in quarter]
                assert wavefronts(own) == 1, (phase, r)
                mirrored = [g * class_floats + _at(skew, 8 * bj + r, 8 * bi + half)
                            for g, bi, bj in quarter if bi != bj]
                assert wavefronts(mirrored) == 1, (phase, r)


def test_the_unskewed_layout_had_conflicts():
    """The same model on the plain row-major layout and the row order of the
    tiles finds the collisions the skew removes."""
    plain = [0, 0, 0, 0]
    order = [(bi, bj) for bi in range(4) for bj in range(bi, 4)]
    class_floats = 2 * N * LD + 2 * N + 4
    lanes = [(g, bi, bj) for g in range(CPW) for bi, bj in order]
    worst = 1
    for phase in range(4):
        quarter = lanes[8 * phase:8 * phase + 8]
        own = [g * class_floats + _at(plain, 8 * bi, 8 * bj) for g, bi, bj in quarter]
        groups = {}
        for a in own:
            groups.setdefault((a // 4) % 8, set()).add(a)
        worst = max(worst, max(len(v) for v in groups.values()))
    assert worst > 1
