"""Planted mistakes in the oracle must fail its pins.

Each case copies oracle/pentago_oracle.c, plants one plausible mistake by
text substitution, compiles the copy into a temporary folder on the CPU and
checks that the hand positions, brute force against retrograde, or the
invariants reject it.  Nothing here touches the real oracle build.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.golden.fixtures import hand_positions

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "pentago_oracle.c")

MUTANTS = {
    # quarter turn clockwise instead of anticlockwise (both O1 and O2 use it)
    "turn_clockwise": ("b->c[6 * (R0 + 2 - c) + C0 + r] = old[r][c];",
                       "b->c[6 * (R0 + c) + C0 + 2 - r] = old[r][c];"),
    # retrograde forgets the immediate win by placement
    "no_placement_win": ("if (has_five(&A, c)) {\n          value = 1;",
                         "if (0) {\n          value = 1;"),
    # negamax sign dropped in the retrograde
    "child_sign": ("int h = -V[", "int h = V["),
    # simultaneous fives scored for the mover instead of a tie
    "simultaneous_win": ("value = fc - fcb; /* terminal", "value = fc ? 1 : -fcb; /* terminal"),
    # child fill gets the other colour's digit
    "child_colour": ("int child_idx = idx + c * pow3(i);",
                     "int child_idx = idx + other(c) * pow3(i);"),
    # beta packed with quadrants 0 and 1 transposed when bits are written
    "beta_transposed": ("if (value == 1) out[beta >> 6] |= 1ull << (beta & 63);",
                        "beta = (beta & 0xf0) | ((beta & 3) << 2) | ((beta >> 2) & 3);\n"
                        "  if (value == 1) out[beta >> 6] |= 1ull << (beta & 63);"),
    # wrong side to move
    "mover_swapped": ("if (nb == nw) return BLACK;\n  if (nb == nw + 1) return WHITE;",
                      "if (nb == nw) return WHITE;\n  if (nb == nw + 1) return BLACK;"),
    # a full board scored as a win for the mover
    "full_board_win": ("if (fc || fcb || full) return fc - fcb;",
                       "if (fc || fcb || full) return (fc || fcb) ? fc - fcb : 1;"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation site for {name} not found"
    mutant = tmp_path / f"{name}.c"
    mutant.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", str(so), str(mutant)])
    L = ctypes.CDLL(str(so))
    u64, i32, p64 = ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)
    L.oracle_brute_force.argtypes = [u64, i32, p64]
    L.oracle_midgame.argtypes = [u64, i32, i32, p64, ctypes.POINTER(ctypes.c_int8)]
    L.oracle_rotate.argtypes = [u64, i32]
    L.oracle_rotate.restype = u64
    return L


def _call(fn, board, *extra):
    out = np.zeros(8, dtype=np.uint64)
    rc = fn(ctypes.c_uint64(int(board)), *extra, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
            *([None] if fn.__name__ == "oracle_midgame" else []))
    return rc, out


def _pins_pass(L):
    """The oracle's pins, run against a compiled variant.  False = caught."""
    def brute(b):
        return _call(L.oracle_brute_force, b, 8)

    def retro(b):
        return _call(L.oracle_midgame, b, 13, 0)

    for case in hand_positions():
        board = inputs.pack_cells(case["cells"])
        for solve in (brute, retro):
            rc, sv = solve(board)
            if rc:
                return False
            for beta, win, notlose in case["expect"]:
                if (int(sv[beta >> 6]) >> (beta & 63)) & 1 != win:
                    return False
                if (int(sv[4 + (beta >> 6)]) >> (beta & 63)) & 1 != notlose:
                    return False
    for k in (1, 2, 3, 4):
        for board in inputs.midgame_boards(3, k, 0xFACE + k):
            rc1, a = brute(board)
            rc2, b = retro(board)
            if rc1 or rc2 or not (a == b).all():
                return False
            # L-equivariance for one h
            h = 1 + 4 * 3  # g = (1, 3, 0, 0)
            rc3, c = retro(L.oracle_rotate(ctypes.c_uint64(int(board)), h))
            for beta in range(256):
                g = [(beta >> (2 * q)) & 3 for q in range(4)]
                g2 = [(g[0] + 1) % 4, (g[1] + 3) % 4, g[2], g[3]]
                b2 = g2[0] + 4 * g2[1] + 16 * g2[2] + 64 * g2[3]
                if ((int(c[beta >> 6]) >> (beta & 63)) & 1) != ((int(b[b2 >> 6]) >> (b2 & 63)) & 1):
                    return False
    return True


def test_unmutated_copy_passes(tmp_path):
    src = open(SRC).read()
    L = _build(tmp_path, "identity", src[:40], src[:40])
    assert _pins_pass(L)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_build(tmp_path, name, old, new))
