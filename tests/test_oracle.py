"""Pins of the value oracle (O1 brute force, O2 retrograde, O3 sections).

What fixes the oracle from outside itself:
* hand positions whose bits follow from the rules by hand (tests/golden);
* brute force (O1, memoised negamax with the paper's literal h_c rule) against
  the retrograde (O2) on every rotation of small seeded positions;
* group invariants of the rotation-abstracted value: win implies not-lose,
  L-equivariance and invariance under the 8 global symmetries (paper,
  "Abstracting over rotations").
"""
import numpy as np
import pytest

import oracle
from oracle import enumeration as E
from paper_1404_0743_gb300 import inputs
from tests.golden.fixtures import hand_positions


def _bits(sv, table):
    return [oracle.bit(sv, table, beta) for beta in range(256)]


@pytest.mark.parametrize("case", hand_positions(), ids=lambda c: c["name"])
@pytest.mark.parametrize("solver", ["brute_force", "midgame"])
def test_hand_positions(case, solver):
    board = inputs.pack_cells(case["cells"])
    sv = getattr(oracle, solver)(board)
    for beta, win, notlose in case["expect"]:
        assert oracle.bit(sv, 0, beta) == win, (case["name"], beta)
        assert oracle.bit(sv, 1, beta) == notlose, (case["name"], beta)


def _small_boards():
    out = []
    for k in range(0, 7):
        out += [int(b) for b in inputs.midgame_boards(6, k, 0xBEEF + 100 * k)]
    return out


SMALL = _small_boards()


@pytest.mark.parametrize("board", SMALL[::2], ids=lambda b: f"{b:#x}")
def test_brute_force_equals_retrograde(board):
    assert (oracle.brute_force(board) == oracle.midgame(board, check=True)).all()


def test_brute_force_equals_retrograde_eight_empties():
    for board in inputs.midgame_boards(2, 8, 0xC0FFEE):
        assert (oracle.brute_force(int(board), max_empty=8) == oracle.midgame(int(board))).all()


def test_threads_share_levels_without_changing_values():
    """Fills of one level shared among host threads: the same table, bit for
    bit, as one thread (every fill, not only the root), with the explicit
    child check on."""
    for k, seed in ((8, 0x7A), (9, 0x7B)):
        for board in inputs.midgame_boards(2, k, seed):
            one, V1 = oracle.midgame(int(board), check=True, all_values=True)
            many, V4 = oracle.midgame(int(board), check=True, all_values=True, threads=5)
            assert (one == many).all() and (V1 == V4).all()


def test_size_limit():
    """Up to 16 empty cells are accepted; 17 are refused before any work."""
    board = int(inputs.midgame_boards(1, 17, 0x17)[0])
    with pytest.raises(oracle.OracleError):
        oracle.midgame(board, max_empty=17)


@pytest.mark.parametrize("board", SMALL[1::3], ids=lambda b: f"{b:#x}")
def test_win_implies_notlose(board):
    sv = oracle.midgame(board)
    assert (sv[:4] & ~sv[4:] == 0).all()


def _add(g, h):
    return [(a + b) % 4 for a, b in zip(g, h)]


def _g(beta):
    return [(beta >> (2 * q)) & 3 for q in range(4)]


@pytest.mark.parametrize("board", SMALL[2::5], ids=lambda b: f"{b:#x}")
def test_l_equivariance(board):
    # super(h s)[g] = super(s)[g + h]: turning quadrants first only relabels
    # the 256 rotated boards (L is abelian)
    sv = oracle.midgame(board)
    for h in ([1, 0, 0, 0], [0, 3, 0, 0], [0, 0, 2, 1], [3, 1, 2, 3]):
        hs = oracle.rotate(board, oracle.beta_of(h))
        sh = oracle.midgame(hs)
        for table in (0, 1):
            for beta in range(0, 256, 7):
                assert oracle.bit(sh, table, beta) == oracle.bit(
                    sv, table, oracle.beta_of(_add(_g(beta), h)))


def _apply_symmetry(board, perm):
    cells = inputs.unpack_cells(board)
    out = [0] * 36
    for i, v in enumerate(cells):
        out[perm[i]] = v
    return inputs.pack_cells(out)


def _quadrant_map(perm):
    """Quadrant position images and whether the symmetry is a reflection."""
    qmap = []
    for q in range(4):
        R, C = 3 * (q >> 1) + 1, 3 * (q & 1) + 1  # quadrant centre
        i = perm[6 * R + C]
        R2, C2 = divmod(i, 6)
        qmap.append(2 * (R2 >= 3) + (C2 >= 3))
    # orientation: image of the step (0,0)->(0,1) against (0,0)->(1,0)
    def img(R, C):
        return divmod(perm[6 * R + C], 6)
    a, b, c = img(0, 0), img(0, 1), img(1, 0)
    cross = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return qmap, cross > 0


@pytest.mark.parametrize("board", SMALL[3::6], ids=lambda b: f"{b:#x}")
def test_d4_invariance(board):
    # super(d s)[d g d^-1] = super(s)[g]: a global rotation carries quadrant q
    # to position qmap[q] keeping the turn direction; a reflection also
    # reverses it (paper, "Abstracting over rotations": G = Z4^4 x| D4)
    sv = oracle.midgame(board)
    for perm in E.board_symmetries():
        qmap, reflect = _quadrant_map(perm)
        sd = oracle.midgame(_apply_symmetry(board, perm))
        for beta in range(256):
            g = _g(beta)
            g2 = [0] * 4
            for q in range(4):
                g2[qmap[q]] = (-g[q]) % 4 if reflect else g[q]
            for table in (0, 1):
                assert oracle.bit(sd, table, oracle.beta_of(g2)) == oracle.bit(sv, table, beta)


def test_d4_map_has_reflections():
    kinds = [_quadrant_map(p)[1] for p in E.board_symmetries()]
    assert kinds.count(True) == 4 and kinds.count(False) == 4


def test_section_oracle_full_and_near_full():
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS)
    d = E.dims()
    for n in (36, 35, 34, 33, 32):  # down to the slice the dependency-cone tests check
        secs = E.sections(n)
        for _ in range(3):
            t = secs[rng.below(len(secs))]
            idx = inputs.sample_indices(rng, [d[x] for x in t])
            board = E.section_board(t, idx)
            assert (oracle.section_value(n, t, idx, check=True) == oracle.brute_force(board)).all()


def test_retrograde_all_values_root_row():
    board = SMALL[-1]
    sv, V = oracle.midgame(board, all_values=True)
    root = V[0]
    for beta in range(256):
        assert oracle.bit(sv, 0, beta) == int(root[beta] == 1)
        assert oracle.bit(sv, 1, beta) == int(root[beta] >= 0)
