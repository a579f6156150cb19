"""The stored expected values of the batched midgame workload match what
they claim to be: every stored board is the generator's board of that
index, and the first stored value is recomputed by the oracle as it stands
(about 30 s), so the GPU tests that read the file compare against the
committed oracle."""
import os

import numpy as np

import oracle
from paper_1404_0743_gb300 import inputs

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batched_midgame_k12.txt")


def _rows():
    rows = []
    for line in open(PATH):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((int(f[0]), int(f[1], 16), [int(w, 16) for w in f[2:]]))
    return rows


def test_stored_boards_are_the_workload():
    rows = _rows()
    boards = inputs.batched_midgame_boards(1024)
    assert [i for i, _, _ in rows] == list(range(0, 1024, 16))
    for i, b, words in rows:
        assert b == int(boards[i]) and len(words) == 8


def test_first_stored_value_recomputed():
    i, b, words = _rows()[0]
    got = oracle.midgame(b)
    assert (np.asarray(got, dtype=np.uint64) == np.array(words, dtype=np.uint64)).all()
