"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no step of the method: it only draws boards.  Random
numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), one independent stream per
board seeded with ``base + i``.

Board encoding (the library's input format): cell (R, C) lies in quadrant
q = 2*[R>=3] + [C>=3] at local (r, c) = (R mod 3, C mod 3); quadrant q's
16-bit field of the uint64 holds sum digit * 3^(3r+c), digit 0 empty,
1 black, 2 white.

Workload recipes (the paper's own workload is the game's state space, so
every input is synthetic):

* plain midgame: 64 boards, seed 0x14040743 + i, 15 black + 15 white on
  uniformly shuffled cells (6 empty, black to move);
* batched midgame: 1024 boards, seed 0x14040743 + 1000 + i, 12 + 12 stones
  (12 empty, black to move);
* serving: seed 0x14040743 + 5000 + i, k = 8 + (draw mod 9) empty cells,
  ceil((36-k)/2) black and floor((36-k)/2) white (black moves when k is even).

A drawn board that already shows five in a row for either colour as given
(no quadrant turned) is rejected and the same stream draws again.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
SEED_BASE = 0x14040743
SEED_PLAIN = SEED_BASE
SEED_BATCHED = SEED_BASE + 1000
SEED_SERVING = SEED_BASE + 5000
SEED_SECTIONS = SEED_BASE + 7000


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        return self.next() % n

    def uniform(self) -> float:
        """Uniform in (0, 1], 53 random bits."""
        return ((self.next() >> 11) + 1) / float(1 << 53)


def pack_cells(cells) -> int:
    packed = 0
    for R in range(6):
        for C in range(6):
            q = 2 * (R >= 3) + (C >= 3)
            r, c = R % 3, C % 3
            packed += int(cells[6 * R + C]) * 3 ** (3 * r + c) << (16 * q)
    return packed


def unpack_cells(packed: int) -> list[int]:
    out = [0] * 36
    for R in range(6):
        for C in range(6):
            q = 2 * (R >= 3) + (C >= 3)
            r, c = R % 3, C % 3
            code = (packed >> (16 * q)) & 0xFFFF
            out[6 * R + C] = (code // 3 ** (3 * r + c)) % 3
    return out


def _shows_five(cells) -> bool:
    """Input filter: a run of five equal stones as the board is given."""
    for R in range(6):
        for C in range(6):
            for dr, dc in ((0, 1), (1, 0), (1, 1), (1, -1)):
                R4, C4 = R + 4 * dr, C + 4 * dc
                if not (0 <= R4 < 6 and 0 <= C4 < 6):
                    continue
                v = cells[6 * R + C]
                if v and all(cells[6 * (R + i * dr) + C + i * dc] == v for i in range(5)):
                    return True
    return False


def random_board(rng: SplitMix64, n_black: int, n_white: int) -> int:
    """Shuffle the 36 cells (Fisher-Yates), put black on the first n_black and
    white on the next n_white; redraw while the board shows a five."""
    while True:
        order = list(range(36))
        for i in range(35, 0, -1):
            j = rng.below(i + 1)
            order[i], order[j] = order[j], order[i]
        cells = [0] * 36
        for p in order[:n_black]:
            cells[p] = 1
        for p in order[n_black:n_black + n_white]:
            cells[p] = 2
        if not _shows_five(cells):
            return pack_cells(cells)


def midgame_boards(count: int, empties: int, seed: int) -> np.ndarray:
    """``count`` boards with ``empties`` empty cells and balanced colours."""
    stones = 36 - empties
    out = np.zeros(count, dtype=np.uint64)
    for i in range(count):
        out[i] = random_board(SplitMix64(seed + i), (stones + 1) // 2, stones // 2)
    return out


def plain_midgame_boards(count: int = 64) -> np.ndarray:
    return midgame_boards(count, 6, SEED_PLAIN)


def batched_midgame_boards(count: int = 1024) -> np.ndarray:
    return midgame_boards(count, 12, SEED_BATCHED)


def serving_queries(count: int = 10000, kmin: int = 8, kmax: int = 16):
    """(boards, empties) for the serving workload."""
    boards = np.zeros(count, dtype=np.uint64)
    ks = np.zeros(count, dtype=np.int32)
    for i in range(count):
        rng = SplitMix64(SEED_SERVING + i)
        k = kmin + rng.below(kmax - kmin + 1)
        stones = 36 - k
        boards[i] = random_board(rng, (stones + 1) // 2, stones // 2)
        ks[i] = k
    return boards, ks


def poisson_arrivals(count: int, rate_per_s: float, seed: int = SEED_SERVING + 999) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = SplitMix64(seed)
    t = 0.0
    out = np.zeros(count, dtype=np.float64)
    for i in range(count):
        t += -math.log(rng.uniform()) / rate_per_s
        out[i] = t
    return out


def sample_indices(rng: SplitMix64, dims) -> tuple[int, ...]:
    return tuple(rng.below(int(d)) for d in dims)
