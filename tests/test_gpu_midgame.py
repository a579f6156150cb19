"""Midgame solver (paper, "Open source and data") against the oracle, bit for bit.

Sizes the oracle finishes in seconds cover several thread blocks and ragged
tails (mixed numbers of empty cells in one launch); the full batched workload
(1024 boards with 12 empty cells, one launch sequence) is checked on stored
oracle values of every board (tests/golden/make_golden.py), and the serving
stream's queries with 14, 15 and 16 empty cells on theirs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import midgame_oracle, ready, to_dev, to_host

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batched_midgame_k12.txt")


def _solve(pp, boards, max_empty):
    import torch
    ws = torch.empty(pp.midgame_workspace_bytes(len(boards), max_empty), dtype=torch.uint8, device="cuda")
    out = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve(to_dev(boards), out, max_empty, ws)
    torch.cuda.synchronize()
    return to_host(out)


def test_plain_midgame_workload():
    """64 seeded 30-stone boards, 6 empty cells, black to move."""
    pp = ready()
    boards = inputs.plain_midgame_boards(64)
    assert (_solve(pp, boards, 6) == midgame_oracle(boards)).all()


def test_mixed_empties_one_launch():
    """Boards with 0..9 empty cells (both movers) in one call: ragged levels."""
    pp = ready()
    boards = np.concatenate([inputs.midgame_boards(7, k, 0x5150 + k) for k in range(10)])
    order = np.random.default_rng(3).permutation(len(boards))
    boards = boards[order]
    got = _solve(pp, boards, 9)
    assert (got == midgame_oracle(boards)).all()


def test_max_empty_larger_than_needed():
    pp = ready()
    boards = inputs.midgame_boards(5, 5, 0xABC)
    assert (_solve(pp, boards, 8) == midgame_oracle(boards)).all()


def test_ten_empty_cells():
    pp = ready()
    boards = inputs.midgame_boards(3, 10, 0x10E)
    assert (_solve(pp, boards, 10) == midgame_oracle(boards)).all()


def test_hand_positions_through_midgame():
    from tests.golden.fixtures import hand_positions
    pp = ready()
    for case in hand_positions():
        board = inputs.pack_cells(case["cells"])
        cells = case["cells"]
        shows = False
        try:
            got = _solve(pp, np.array([board], dtype=np.uint64), 2)[0]
        except pp.PentagoError:
            shows = True  # boards with a five as given are rejected by design
        if shows:
            continue
        for b, win, notlose in case["expect"]:
            assert oracle.bit(got, 0, b) == win and oracle.bit(got, 1, b) == notlose, case["name"]


def test_deterministic_and_host_path():
    import torch
    pp = ready()
    boards = inputs.midgame_boards(40, 7, 0xD0D0)
    a = _solve(pp, boards, 7)
    b = _solve(pp, boards, 7)
    assert (a == b).all()
    ws = torch.empty(pp.midgame_workspace_bytes(len(boards), 7), dtype=torch.uint8, device="cuda")
    out = torch.zeros((len(boards), 8), dtype=torch.int64).pin_memory()
    pp.midgame_solve_host(torch.from_numpy(boards.view(np.int64)), out, 7, ws)
    assert (out.numpy().view(np.uint64) == a).all()


def test_plan_rerun_and_empty_batch():
    import torch
    pp = ready()
    boards = inputs.midgame_boards(9, 6, 0x9)
    plan = pp.MidgamePlan(boards, 6)
    ws = torch.empty(pp.midgame_workspace_bytes(9, 6), dtype=torch.uint8, device="cuda")
    out = torch.zeros((9, 8), dtype=torch.int64, device="cuda")
    plan.run(ws, out)
    first = to_host(out).copy()
    out.zero_()
    plan.run(ws, out)
    torch.cuda.synchronize()
    assert (to_host(out) == first).all()
    assert (first == midgame_oracle(boards)).all()
    empty = pp.MidgamePlan(np.zeros(0, dtype=np.uint64), 6)
    empty.run(ws, out)


def test_invalid_inputs_rejected_before_launch():
    import torch
    pp = ready()
    good = inputs.midgame_boards(1, 6, 1)[0]
    ws = torch.empty(pp.midgame_workspace_bytes(1, 6), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 8), dtype=torch.int64, device="cuda")
    bad_digit = np.uint64(int(good) | 0xFFFF)  # quadrant 0 field >= 3^9
    cells = inputs.unpack_cells(int(good))
    cells[cells.index(0)] = 1  # one black stone too many
    bad_counts = inputs.pack_cells([1 if c == 2 else c for c in cells])
    five = inputs.pack_cells([1] * 5 + [2] * 5 + [0] * 26)
    before = pp.launch_count()
    for b in (bad_digit, bad_counts, five):
        with pytest.raises(pp.PentagoError) as e:
            pp.midgame_solve(to_dev(np.array([b], dtype=np.uint64)), out, 6, ws)
        assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:  # too many empty cells for max_empty
        pp.midgame_solve(to_dev(inputs.midgame_boards(1, 8, 2)), out, 6, ws)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:  # workspace too small
        pp.midgame_solve(to_dev(np.array([good])), out, 6, ws[:1000])
    assert e.value.code == 2
    assert pp.launch_count() == before


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        parts = line.split()
        rows.append((int(parts[0]), int(parts[1], 16), [int(x, 16) for x in parts[2:]]))
    return rows


def test_batched_workload_full_size():
    """All 1024 boards with 12 empty cells in one plan run, as the benchmark
    launches them; every board against stored oracle values."""
    import torch
    pp = ready()
    boards = inputs.batched_midgame_boards(1024)
    rows = _golden()
    assert len(rows) == 1024
    for i, b, _ in rows:
        assert int(boards[i]) == b
    plan = pp.MidgamePlan(boards, 12)
    ws = torch.empty(pp.midgame_workspace_bytes(1024, 12), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1024, 8), dtype=torch.int64, device="cuda")
    plan.run(ws, out)
    torch.cuda.synchronize()
    got = to_host(out)
    for i, _, words in rows:
        assert [int(x) for x in got[i]] == words, i
    # every result satisfies win => not lose
    assert ((got[:, :4] & ~got[:, 4:]) == 0).all()


def _rmax_bits(a):
    """rmax over a [256] bool table (paper, "Abstracting over rotations"):
    out[g] = OR over the 8 single-quadrant quarter turns r of a[g + r]."""
    out = np.zeros(256, dtype=bool)
    for beta in range(256):
        g = [(beta >> (2 * q)) & 3 for q in range(4)]
        for q in range(4):
            for d in (1, 3):
                h = list(g)
                h[q] = (h[q] + d) % 4
                out[beta] |= a[h[0] + 4 * h[1] + 16 * h[2] + 64 * h[3]]
    return out


def _bits(words):
    w = np.asarray(words, dtype=np.uint64)
    return np.array([(int(w[b >> 6]) >> (b & 63)) & 1 for b in range(256)], dtype=bool)


@pytest.mark.parametrize("seed", [0x16A, 0x16B])
def test_maximum_size_against_its_children(seed):
    """16 empty cells (the largest size; beyond the oracle's reach): the
    root's value equals the recursion of "Problem definition" applied to its
    children's values, each solved separately with 15 empty cells, and to
    the root's own five-in-a-row sets from the oracle's line scan:
    win = I | rmax(OR ~notlose'), notlose = I | rmax(OR ~win'), overridden
    where either colour has five.  The half-table solve agrees on its class."""
    import torch
    from tests.test_gpu_parity import class_mask
    pp = ready()
    rng = np.random.default_rng(seed)
    while True:  # a root none of whose children shows five as given
        root = int(inputs.midgame_boards(1, 16, int(rng.integers(1 << 30)))[0])
        cells = oracle.cells(root)
        mover = 1 if cells.count(1) == cells.count(2) else 2
        empties = [i for i in range(36) if cells[i] == 0]
        kids = []
        for e in empties:
            c = list(cells)
            c[e] = mover
            kids.append(oracle.pack(c))
        if not any(oracle.has_five(k, 0, 1) or oracle.has_five(k, 0, 2) for k in kids):
            break
    root_v = _solve(pp, np.array([root], dtype=np.uint64), 16)[0]
    kid_v = _solve(pp, np.array(kids, dtype=np.uint64), 15)
    aw = np.zeros(256, dtype=bool)
    an = np.zeros(256, dtype=bool)
    imm = np.zeros(256, dtype=bool)
    for k, v in zip(kids, kid_v):
        aw |= ~_bits(v[4:])
        an |= ~_bits(v[:4])
        imm |= np.array([oracle.has_five(k, b, mover) for b in range(256)])
    fc = np.array([oracle.has_five(root, b, mover) for b in range(256)])
    fo = np.array([oracle.has_five(root, b, 3 - mover) for b in range(256)])
    t = fc | fo
    win = np.where(t, fc & ~fo, imm | _rmax_bits(aw))
    notlose = np.where(t, fc | ~fo, imm | _rmax_bits(an))
    assert (_bits(root_v[:4]) == win).all()
    assert (_bits(root_v[4:]) == notlose).all()
    ws = torch.empty(pp.midgame_parity_workspace_bytes(1, 16), dtype=torch.uint8, device="cuda")
    half = torch.zeros((1, 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve_parity(to_dev(np.array([root], dtype=np.uint64)), half, 16, 0, ws)
    assert (to_host(half)[0] == (root_v & class_mask(0))).all()


DEEP = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "serving_deep_k14_16.txt")


def deep_rows():
    """(query index, empty cells, board, 8 words) of the stored oracle values
    for the serving stream's first queries with 14, 15 and 16 empty cells."""
    rows = []
    for line in open(DEEP):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((int(f[0]), int(f[1]), int(f[2], 16), [int(w, 16) for w in f[3:]]))
    return rows


def test_deep_queries_against_stored_oracle_values():
    """14, 15 and 16 empty cells (the largest size the solver accepts), in one
    call with max_empty 16, bit for bit against the oracle; the parity-class
    solve agrees on each class."""
    import torch
    from tests.test_gpu_parity import class_mask
    pp = ready()
    rows = deep_rows()
    assert sorted({k for _, k, _, _ in rows}) == [14, 15, 16]
    boards = np.array([b for _, _, b, _ in rows], dtype=np.uint64)
    got = _solve(pp, boards, 16)
    for (i, k, b, words), g in zip(rows, got):
        assert [int(x) for x in g] == words, (i, k)
    for parity in (0, 1):
        ws = torch.empty(pp.midgame_parity_workspace_bytes(len(boards), 16), dtype=torch.uint8, device="cuda")
        half = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
        pp.midgame_solve_parity(to_dev(boards), half, 16, parity, ws)
        assert (to_host(half) == (got & class_mask(parity))).all(), parity
