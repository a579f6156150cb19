"""Device building blocks against plain definitions and the oracle.

* rotated five-in-a-row masks against the oracle's explicit line scan of the
  rotated board, for all 256 rotations (paper, "Abstracting over rotations");
* rmax against its definition, OR over the 8 single-quadrant quarter turns;
* the quadrant-axis shift against index arithmetic.
All comparisons are exact.
"""
import numpy as np
import pytest

import oracle
from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import beta, bits_to_bool, bool_to_bits, digits, ready, to_dev, to_host

pytestmark = pytest.mark.gpu


def _random_boards(count, seed):
    rng = inputs.SplitMix64(seed)
    out = []
    for _ in range(count):
        cells = [rng.below(3) for _ in range(36)]
        out.append(inputs.pack_cells(cells))
    return np.array(out, dtype=np.uint64)


def test_five_masks_match_oracle_scan():
    import torch
    pp = ready()
    boards = np.concatenate([_random_boards(96, 11), inputs.midgame_boards(32, 4, 12),
                             inputs.midgame_boards(32, 0, 13)])
    out = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
    pp.five_masks(to_dev(boards), out)
    got = bits_to_bool(to_host(out))
    for i, b in enumerate(boards):
        for bt in range(256):
            assert got[i, 0, bt] == oracle.has_five(int(b), bt, 1), (i, bt, "black")
            assert got[i, 1, bt] == oracle.has_five(int(b), bt, 2), (i, bt, "white")


def _rmax_reference(bb):
    out = np.zeros_like(bb)
    for bt in range(256):
        g = digits(bt)
        for q in range(4):
            for d in (1, 3):
                g2 = list(g)
                g2[q] = (g2[q] + d) % 4
                out[:, :, bt] |= bb[:, :, beta(g2)]
    return out


def _random_values(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 2 ** 63, size=(n, 8), dtype=np.int64).astype(np.uint64)
    v ^= rng.integers(0, 2, size=(n, 8), dtype=np.int64).astype(np.uint64) << np.uint64(63)
    return v


def test_rmax_matches_definition():
    import torch
    pp = ready()
    vals = _random_values(300, 5)
    # sparse inputs as well: single bits
    sparse = np.zeros((512, 8), dtype=np.uint64)
    for i in range(512):
        sparse[i, (i // 64) % 8] = np.uint64(1) << np.uint64(i % 64)
    vals = np.concatenate([vals, sparse])
    out = torch.zeros((len(vals), 8), dtype=torch.int64, device="cuda")
    pp.rmax(to_dev(vals), out)
    assert (to_host(out) == bool_to_bits(_rmax_reference(bits_to_bool(vals)))).all()


def test_rmax_flips_parity():
    # paper, "Open source and data": rmax maps tables on one parity class of
    # Z4^4 (sum of g_q even or odd) to the other
    import torch
    pp = ready()
    bb = bits_to_bool(_random_values(64, 6))
    even = np.array([sum(digits(b)) % 2 == 0 for b in range(256)])
    bb[:, :, ~even] = False
    out = torch.zeros((64, 8), dtype=torch.int64, device="cuda")
    pp.rmax(to_dev(bool_to_bits(bb)), out)
    r = bits_to_bool(to_host(out))
    assert not r[:, :, even].any()


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_shift_matches_index_arithmetic(q):
    import torch
    pp = ready()
    vals = _random_values(64, 7 + q)
    bb = bits_to_bool(vals)
    for u in range(4):
        out = torch.zeros((64, 8), dtype=torch.int64, device="cuda")
        pp.shift(to_dev(vals), q, u, out)
        want = np.zeros_like(bb)
        for bt in range(256):
            g = digits(bt)
            g[q] = (g[q] + u) % 4
            want[:, :, bt] = bb[:, :, beta(g)]
        assert (to_host(out) == bool_to_bits(want)).all(), (q, u)
