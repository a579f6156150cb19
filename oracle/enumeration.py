"""Plain enumeration of the paper's data layout -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this module; the product builds its own tables independently.

What is enumerated (paper, Section "Data layout and distribution"):

* quadrant states: 3x3 patterns, digit weight 3^(3r+c), 0 empty / 1 black /
  2 white, so 3^9 = 19683 states per quadrant;
* rotation-minimal states: a state is kept when its code is the smallest of
  the four codes of its anticlockwise rotations; the states of one
  (black, white) count pair are listed in increasing code order (the paper's
  reflected-pair ordering only matters for D4-reduced sections, which are not
  computed here; the block counts below do not depend on it);
* sections of slice n: per-quadrant (black, white) counts with ceil(n/2)
  black and floor(n/2) white stones in total; a section is a 4-D array with
  dimension q = number of minimal states of quadrant q's counts;
* D4 on sections: global board symmetries permute the quadrant positions;
  a section is D4-minimal when its count tuple is the smallest of its 8
  images.

Each count printed in the paper is reproduced by a function here and pinned
in tests/test_enumeration.py.
"""
from __future__ import annotations

import functools
import itertools
import math

NQ = 4
QSTATES = 3 ** 9


def quadrant_digits(code: int) -> list[int]:
    return [(code // 3 ** i) % 3 for i in range(9)]


def quadrant_code(digits) -> int:
    return sum(int(d) * 3 ** i for i, d in enumerate(digits))


def rotate_quadrant_code(code: int) -> int:
    """One anticlockwise quarter turn: local (r, c) moves to (2 - c, r)."""
    d = quadrant_digits(code)
    n = [0] * 9
    for r in range(3):
        for c in range(3):
            n[3 * (2 - c) + r] = d[3 * r + c]
    return quadrant_code(n)


@functools.lru_cache(maxsize=None)
def minimal_states() -> dict[tuple[int, int], list[int]]:
    """(black, white) -> increasing list of rotation-minimal quadrant codes."""
    out: dict[tuple[int, int], list[int]] = {}
    for code in range(QSTATES):
        orbit = [code]
        for _ in range(3):
            orbit.append(rotate_quadrant_code(orbit[-1]))
        if code == min(orbit):
            d = quadrant_digits(code)
            out.setdefault((d.count(1), d.count(2)), []).append(code)
    return out


def dims() -> dict[tuple[int, int], int]:
    return {k: len(v) for k, v in minimal_states().items()}


QUAD_COUNTS = [(b, w) for b in range(10) for w in range(10) if b + w <= 9]


def slice_colours(n: int) -> tuple[int, int]:
    """Black and white stones in slice n: black moves first."""
    return (n + 1) // 2, n // 2


def sections(n: int) -> list[tuple[tuple[int, int], ...]]:
    """All count tuples ((b0,w0),...,(b3,w3)) of slice n, lexicographic order."""
    B, W = slice_colours(n)
    out = []
    for t in itertools.product(QUAD_COUNTS, repeat=3):
        b = B - sum(x[0] for x in t)
        w = W - sum(x[1] for x in t)
        if 0 <= b and 0 <= w and b + w <= 9:
            out.append(t + ((b, w),))
    return sorted(out)


# Global symmetries as permutations of quadrant positions (q0 top-left,
# q1 top-right, q2 bottom-left, q3 bottom-right).  A quarter turn of the
# whole board anticlockwise carries top-left to bottom-left, bottom-left to
# bottom-right, bottom-right to top-right and top-right to top-left; a
# left-right mirror swaps the columns of quadrants.
_ROT = (2, 0, 3, 1)  # image position of quadrant q under one quarter turn
_MIRROR = (1, 0, 3, 2)


def _compose(p, q):
    return tuple(p[q[i]] for i in range(4))


def d4_quadrant_perms() -> list[tuple[int, ...]]:
    perms = [(0, 1, 2, 3)]
    for _ in range(3):
        perms.append(_compose(_ROT, perms[-1]))
    perms += [_compose(p, _MIRROR) for p in perms[:4]]
    return perms


def section_images(t):
    out = []
    for p in d4_quadrant_perms():
        img = [None] * 4
        for q in range(4):
            img[p[q]] = t[q]
        out.append(tuple(img))
    return out


def is_d4_minimal(t) -> bool:
    return tuple(t) == min(section_images(t))


def section_size(t) -> int:
    d = dims()
    return math.prod(d[x] for x in t)


def layout_totals():
    """Blocks, block lines, maximum D4-minimal sections per slice, and the
    rotation / section overcount numerators (paper, "Data layout")."""
    d = dims()
    blocks = lines = max_sections = 0
    rot_entries = sec_entries = 0
    for n in range(37):
        count = 0
        for t in sections(n):
            size = math.prod(d[x] for x in t)
            rot_entries += size
            if is_d4_minimal(t):
                count += 1
                sec_entries += size
                bl = [math.ceil(d[x] / 8) for x in t]
                blocks += math.prod(bl)
                lines += sum(math.prod(bl[:q] + bl[q + 1:]) for q in range(4))
        max_sections = max(max_sections, count)
    return dict(blocks=blocks, lines=lines, max_sections=max_sections,
                rot_entries=rot_entries, sec_entries=sec_entries)


# Global symmetries of the 6x6 board as maps of (R, C).
_BOARD_SYMS = [
    lambda R, C: (R, C),
    lambda R, C: (5 - C, R),
    lambda R, C: (5 - R, 5 - C),
    lambda R, C: (C, 5 - R),
    lambda R, C: (R, 5 - C),
    lambda R, C: (5 - R, C),
    lambda R, C: (C, R),
    lambda R, C: (5 - C, 5 - R),
]


def board_symmetries():
    """The 8 elements of D4 as cell permutations: perm[i] = image of cell i."""
    out = []
    for f in _BOARD_SYMS:
        perm = []
        for R in range(6):
            for C in range(6):
                R2, C2 = f(R, C)
                perm.append(6 * R2 + C2)
        out.append(perm)
    return out


def _cycle_lengths(perm):
    seen = [False] * len(perm)
    out = []
    for i in range(len(perm)):
        if not seen[i]:
            n, j = 0, i
            while not seen[j]:
                seen[j] = True
                j = perm[j]
                n += 1
            out.append(n)
    return out


def _fixed_colourings(cycles, B, W) -> int:
    """Colourings constant on every cycle with exactly B black, W white."""
    poly = {(0, 0): 1}
    for L in cycles:
        nxt: dict[tuple[int, int], int] = {}
        for (b, w), v in poly.items():
            for db, dw in ((0, 0), (L, 0), (0, L)):
                k = (b + db, w + dw)
                if k[0] <= B and k[1] <= W:
                    nxt[k] = nxt.get(k, 0) + v
        poly = nxt
    return poly.get((B, W), 0)


def states_mod_d4(n: int) -> int:
    """Positions with n stones up to global symmetry (Burnside's lemma)."""
    B, W = slice_colours(n)
    total = sum(_fixed_colourings(_cycle_lengths(p), B, W) for p in board_symmetries())
    assert total % 8 == 0
    return total // 8


def all_states_mod_d4() -> int:
    return sum(states_mod_d4(n) for n in range(37))


def average_empty_cells() -> float:
    """Average number of empty cells over all symmetry-reduced states, i.e. the
    branching factor once rotations are abstracted away."""
    num = sum(states_mod_d4(n) * (36 - n) for n in range(37))
    return num / all_states_mod_d4()


def section_board(t, index) -> int:
    """Packed board at 4-D index (i0..i3) of section t."""
    ms = minimal_states()
    return sum(ms[t[q]][index[q]] << (16 * q) for q in range(4))
