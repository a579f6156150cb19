"""The seeded input generators (no step of the method): SplitMix64 against
its published reference outputs, the board encoding, and each workload's
recipe (stone counts, side to move, no five as given, one stream per board,
Poisson inter-arrival mean).  The five check uses the oracle."""
import numpy as np

import oracle
from paper_1404_0743_gb300 import inputs


def test_splitmix64_reference_outputs():
    """First outputs for seed 1234567 of the reference SplitMix64 (Steele,
    Lea and Flood, OOPSLA 2014; the widely published test values)."""
    r = inputs.SplitMix64(1234567)
    assert [r.next() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                            4593380528125082431, 16408922859458223821]


def test_pack_unpack_round_trip():
    rng = inputs.SplitMix64(99)
    for _ in range(200):
        cells = [rng.below(3) for _ in range(36)]
        b = inputs.pack_cells(cells)
        assert inputs.unpack_cells(b) == cells
        for q in range(4):
            assert (b >> (16 * q)) & 0xFFFF < 3 ** 9


def _check(boards, empties):
    for b in boards:
        cells = inputs.unpack_cells(int(b))
        nb, nw = cells.count(1), cells.count(2)
        assert 36 - nb - nw == empties
        assert nb - nw == (1 if empties % 2 else 0)  # black moves when the counts are equal
        assert not oracle.has_five(int(b), 0, 1) and not oracle.has_five(int(b), 0, 2)


def test_workload_recipes():
    plain = inputs.plain_midgame_boards(64)
    _check(plain, 6)
    batched = inputs.batched_midgame_boards(64)
    _check(batched, 12)
    assert len(set(int(b) for b in batched)) == 64
    # one stream per board: board i depends on its own seed only
    assert int(inputs.midgame_boards(1, 12, inputs.SEED_BATCHED + 17)[0]) == int(batched[17])
    assert (inputs.batched_midgame_boards(8) == batched[:8]).all()


def test_serving_recipe():
    boards, ks = inputs.serving_queries(300)
    assert set(int(k) for k in ks) == set(range(8, 17))
    for b, k in zip(boards, ks):
        _check([b], int(k))


def test_poisson_mean_gap():
    t = inputs.poisson_arrivals(20000, 1000.0, seed=5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1e-3) < 3e-5  # mean 1/rate, within about 4 standard errors
