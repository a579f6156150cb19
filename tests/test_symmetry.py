"""Board symmetries and D4-reduced section lists of the library, on the host
(paper, "Abstracting over rotations": D4 and G = L x| D4; "Data layout and
distribution": only sections whose counts are least under D4 are computed).

The library's eight symmetries are checked against the oracle's cell
permutations, its quadrant map and turn reversal against the oracle's values
(f_{s b}(phi_s(g)) = f_b(g)), and its D4 section lists against the oracle's
enumeration, whose totals are pinned to the paper's block counts in
test_enumeration.  No kernel is launched here.
"""
import numpy as np
import pytest

import oracle
from oracle import enumeration as E
from paper_1404_0743_gb300 import inputs


@pytest.fixture(scope="module")
def pp():
    from paper_1404_0743_gb300 import build
    build.build()
    import paper_1404_0743_gb300 as pp
    return pp


def _cell_perm(pp, sym):
    """Image cell of every cell under the library's symmetry sym."""
    perm = []
    for i in range(36):
        cells = [0] * 36
        cells[i] = 1
        img = inputs.unpack_cells(pp.symmetry_board(inputs.pack_cells(cells), sym))
        perm.append(img.index(1))
    return perm


def test_symmetries_are_the_boards_d4(pp):
    lib = [_cell_perm(pp, s) for s in range(8)]
    assert sorted(map(tuple, lib)) == sorted(map(tuple, E.board_symmetries()))
    # numbering: s = k + 4m is a mirror (m = 1) then k anticlockwise quarter turns
    for s in range(8):
        for R in range(6):
            for C in range(6):
                r, c = R, (5 - C if s >= 4 else C)
                for _ in range(s & 3):
                    r, c = 5 - c, r
                assert lib[s][6 * R + C] == 6 * r + c


def test_symmetry_info_matches_cell_maps(pp):
    for s in range(8):
        perm = _cell_perm(pp, s)
        qmap, reflects = pp.symmetry_info(s)
        for q in range(4):
            R, C = 3 * (q >> 1) + 1, 3 * (q & 1) + 1  # quadrant centre
            R2, C2 = divmod(perm[6 * R + C], 6)
            assert qmap[q] == 2 * (R2 >= 3) + (C2 >= 3)
        assert reflects == (s >= 4)


def test_symmetry_board_keeps_patterns_whole(pp):
    rng = inputs.SplitMix64(0xD4D4)
    for _ in range(50):
        cells = [rng.below(3) for _ in range(36)]
        b = inputs.pack_cells(cells)
        for s in range(8):
            img = inputs.unpack_cells(pp.symmetry_board(b, s))
            perm = _cell_perm(pp, s)
            assert all(img[perm[i]] == cells[i] for i in range(36))


@pytest.mark.parametrize("k", [3, 5])
def test_phi_agrees_with_oracle_values(pp, k):
    """f_{s b}(phi_s(g)) = f_b(g), phi_s(g)[qmap[q]] = eps g[q], on the
    oracle's values: the library's quadrant map and turn reversal are the
    ones under which the game's values are invariant."""
    boards = inputs.midgame_boards(3, k, 0xD400 + k)
    for b in boards:
        fb = oracle.midgame(int(b))
        for s in range(8):
            qmap, reflects = pp.symmetry_info(s)
            fsb = oracle.midgame(pp.symmetry_board(int(b), s))
            for beta in range(256):
                g = [(beta >> (2 * q)) & 3 for q in range(4)]
                g2 = [0] * 4
                for q in range(4):
                    g2[qmap[q]] = (-g[q]) % 4 if reflects else g[q]
                for t in (0, 1):
                    assert oracle.bit(fsb, t, oracle.beta_of(g2)) == oracle.bit(fb, t, beta)


@pytest.mark.parametrize("n", [0, 1, 9, 17, 18, 26, 33, 34, 35, 36])
def test_d4_sections_match_oracle(pp, n):
    secs, total = pp.slice_sections(n, d4=True)
    want = [t for t in E.sections(n) if E.is_d4_minimal(t)]
    assert len(secs) == len(want)
    d = E.dims()
    offset = 0
    for s, t in zip(secs, want):
        assert tuple(tuple(int(v) for v in row) for row in s["bw"]) == t
        assert [int(x) for x in s["dim"]] == [d[x] for x in t]
        assert int(s["offset"]) == offset
        offset += int(np.prod([d[x] for x in t]))
    assert total == offset


def test_d4_slice_sizes():
    """Stored boards of the D4-reduced slices 36, 35 and 34: one eighth of the
    full layout plus the symmetric sections' overcount (largest for slice
    36, where many count tuples are their own images)."""
    d = E.dims()
    sizes = {}
    for n in (36, 35, 34):
        full = sum(int(np.prod([d[x] for x in t])) for t in E.sections(n))
        red = sum(int(np.prod([d[x] for x in t])) for t in E.sections(n) if E.is_d4_minimal(t))
        assert full / 8 <= red < full / 4
        sizes[n] = red
    assert sizes == {36: 9397647, 35: 119704992, 34: 985287494}


def test_symmetry_errors(pp):
    with pytest.raises(pp.PentagoError):
        pp.symmetry_info(8)
    with pytest.raises(pp.PentagoError):
        pp.symmetry_board(0, -1)
    with pytest.raises(pp.PentagoError):
        pp.slice_sections(37, d4=True)
