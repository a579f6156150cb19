"""The stored expected values match what they claim to be.

* batched_midgame_k12.txt: every stored board is the generator's board of
  that index (all 1024), and three stored values, first, middle and last,
  are recomputed by the oracle as it stands (a few seconds each on all host
  threads);
* serving_deep_k14_16.txt: every stored board is the serving stream's query
  of that index with the stated number of empty cells, and the fastest of
  the 14-empty values is recomputed (about half a minute on 8 threads).

So the GPU tests that read these files compare against the committed
oracle."""
import os

import numpy as np

import oracle
from paper_1404_0743_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
K12 = os.path.join(HERE, "batched_midgame_k12.txt")
DEEP = os.path.join(HERE, "serving_deep_k14_16.txt")


def _rows(path, key_fields):
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        head = [int(x) for x in f[:key_fields - 1]]
        rows.append((*head, int(f[key_fields - 1], 16), [int(w, 16) for w in f[key_fields:]]))
    return rows


def test_stored_boards_are_the_workload():
    rows = _rows(K12, 2)
    boards = inputs.batched_midgame_boards(1024)
    assert [i for i, _, _ in rows] == list(range(1024))
    for i, b, words in rows:
        assert b == int(boards[i]) and len(words) == 8


def test_stored_values_recomputed():
    rows = _rows(K12, 2)
    for i in (0, 511, 1023):
        _, b, words = rows[i]
        got = oracle.midgame(b, threads=os.cpu_count() or 1)
        assert (np.asarray(got, dtype=np.uint64) == np.array(words, dtype=np.uint64)).all(), i


def test_deep_boards_are_the_serving_queries():
    rows = _rows(DEEP, 3)
    boards, ks = inputs.serving_queries(max(i for i, _, _, _ in rows) + 1)
    assert sorted({k for _, k, _, _ in rows}) == [14, 15, 16]
    for i, k, b, words in rows:
        assert int(boards[i]) == b and int(ks[i]) == k and len(words) == 8
        assert sum(1 for c in oracle.cells(b) if c == 0) == k


def test_one_deep_value_recomputed():
    i, k, b, words = next(r for r in _rows(DEEP, 3) if r[0] == 23)
    assert k == 14
    got = oracle.midgame(b, threads=os.cpu_count() or 1)
    assert (np.asarray(got, dtype=np.uint64) == np.array(words, dtype=np.uint64)).all()

