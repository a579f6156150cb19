"""Pins of the oracle's layout enumeration to numbers printed in the paper.

Every figure below is quoted in the paper; the oracle reproduces it from its
own quadrant lists and section enumeration, so a wrong rotation, a wrong
minimality rule or a wrong section definition fails at least one of them.
"""
import math

import pytest

from oracle import enumeration as E


def _orbits_with_counts(b, w):
    """Closed form (Burnside over the quarter turns of a 3x3 quadrant) for the
    number of rotation classes of patterns with b black and w white stones."""
    def multinomial(n, parts):
        out = math.factorial(n)
        for p in parts:
            out //= math.factorial(p)
        return out

    e = 9 - b - w
    ident = multinomial(9, (b, w, e))
    # a half turn fixes the centre and swaps 4 pairs of cells
    half = sum(multinomial(4, (bb, ww, 4 - bb - ww))
               for bb in range(5) for ww in range(5 - bb)
               if b - 2 * bb in (0, 1) and w - 2 * ww in (0, 1) and (b - 2 * bb) + (w - 2 * ww) <= 1)
    # a quarter turn fixes the centre and cycles 2 groups of 4 cells
    quarter = sum(multinomial(2, (bb, ww, 2 - bb - ww))
                  for bb in range(3) for ww in range(3 - bb)
                  if b - 4 * bb in (0, 1) and w - 4 * ww in (0, 1) and (b - 4 * bb) + (w - 4 * ww) <= 1)
    total = ident + half + 2 * quarter
    assert total % 4 == 0
    return total // 4


def test_rotation_minimal_states_closed_form():
    ms = E.minimal_states()
    # identity fixes 3^9 patterns, the half turn 3^5, each quarter turn 3^3
    assert sum(len(v) for v in ms.values()) == (3 ** 9 + 3 ** 5 + 2 * 3 ** 3) // 4 == 4995
    for (b, w), codes in ms.items():
        assert len(codes) == _orbits_with_counts(b, w), (b, w)
        assert codes == sorted(codes)
    assert max(len(v) for v in ms.values()) == 420  # (3,3): C(9,3) C(6,3) / 4


def test_rotation_is_a_quarter_turn():
    # top row "X . ." turns into left column bottom cell (anticlockwise):
    # local (0,0) -> (2,0)
    code = E.quadrant_code([1, 0, 0, 0, 0, 0, 0, 0, 0])
    assert E.quadrant_digits(E.rotate_quadrant_code(code)) == [0, 0, 0, 0, 0, 0, 1, 0, 0]
    for code in range(0, 3 ** 9, 97):
        c = code
        for _ in range(4):
            c = E.rotate_quadrant_code(c)
        assert c == code


def test_states_modulo_symmetry():
    # paper, Introduction: 3,009,081,623,421,558 states with symmetries removed
    assert E.all_states_mod_d4() == 3009081623421558


def test_branching_factor():
    # paper, Introduction: average branching factor 97.3 with rotations,
    # 12.2 once rotations are abstracted (8 rotation choices per placement)
    b = E.average_empty_cells()
    assert round(b, 1) == 12.2
    assert round(8 * b, 1) == 97.3


@pytest.fixture(scope="module")
def totals():
    return E.layout_totals()


def test_blocks_lines_and_sections(totals):
    # paper, "Deterministic pseudorandom partitioning": 3,654,002,393 blocks,
    # 996,084,744 block lines, at most 8239 sections per slice
    assert totals["blocks"] == 3654002393
    assert totals["lines"] == 996084744
    assert totals["max_sections"] == 8239


def test_overcounts(totals):
    # paper, "Data layout and distribution": abstracting over rotations costs
    # 5.4%, removing symmetry only per section a further 9.3%, 15.2% in all
    states = E.all_states_mod_d4()
    rot = totals["rot_entries"] * 256 / 8 / states
    sec = totals["sec_entries"] * 256 / states
    assert round(100 * (rot - 1), 1) == 5.4
    assert round(100 * (sec / rot - 1), 1) == 9.3
    assert round(100 * (sec - 1), 1) == 15.2


def test_section_board_counts():
    for n in (34, 35, 36):
        B, W = E.slice_colours(n)
        for t in E.sections(n)[::37]:
            assert sum(x[0] for x in t) == B and sum(x[1] for x in t) == W
            board = E.section_board(t, (0, 0, 0, 0))
            for q in range(4):
                d = E.quadrant_digits((board >> (16 * q)) & 0xFFFF)
                assert (d.count(1), d.count(2)) == t[q]
