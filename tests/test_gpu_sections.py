"""Retrograde step over sections (paper, "Data layout and distribution") against
the oracle, bit for bit.

* slice 36 (values from five in a row or a tie), whole slice, sampled boards
  plus every board of the smallest sections;
* slice 35 from slice 36: every board of all small sections, and the full
  slice (8.11e8 boards, 51.9 GB, the launch the benchmark times) on sampled
  boards;
* slice 34 (two stones to place) on a streamed batch of sections;
* cross-path: a section board's value equals the midgame solver's value of
  the same board (the two paths share the value definition but not the
  standardisation code).
"""
import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import (midgame_oracle, oracle_section_value, ready, section_key, section_size, to_dev,
                               to_host, unravel)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    return ready()


@pytest.fixture(scope="module")
def slice36(pp):
    import torch
    secs, total = pp.slice_sections(36)
    out = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, out)
    torch.cuda.synchronize()
    return secs, out


def _sample(secs, rng, count):
    sizes = np.array([section_size(s) for s in secs], dtype=np.int64)
    picks = []
    for _ in range(count):
        si = rng.below(len(secs))
        picks.append((si, rng.below(int(sizes[si]))))
    return picks


def test_slice36_sampled_and_small_sections(pp, slice36):
    secs, out = slice36
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 36)
    picks = _sample(secs, rng, 400)
    order = np.argsort([section_size(s) for s in secs])
    for si in order[:6]:
        picks += [(int(si), L) for L in range(section_size(secs[si]))]
    host = {}
    for si, L in picks:
        row = int(secs[si]["offset"]) + L
        got = to_host(out[row:row + 1])[0]
        assert (got == oracle_section_value(36, secs[si], L)).all(), (si, L)


@pytest.mark.parametrize("d4", [False, True])
def test_slice36_lines_equal_per_board(pp, slice36, d4):
    """Slice 36 by lines (the default) equals the one-thread-per-board kernel
    (stage_children 2) on every board, in the full and the D4 layout."""
    import torch
    if d4:
        _, total = pp.slice_sections(36, d4=True)
        lines = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
        pp.slice_step(36, None, lines, d4=True)
    else:
        lines = slice36[1]
    per_board = torch.full_like(lines, 7)
    pp.slice_step(36, None, per_board, opts=(0, 0, 0, 2), d4=d4)
    torch.cuda.synchronize()
    assert torch.equal(lines, per_board)


def test_slice36_invariants(pp, slice36):
    import torch
    secs, out = slice36
    win, notlose = out[:, :4], out[:, 4:]
    assert int(torch.count_nonzero(win & ~notlose)) == 0


def _children(secs_child, sec, n):
    keys = {section_key(s): s for s in secs_child}
    mover = 1 if n % 2 == 0 else 2
    out = []
    for q in range(4):
        bw = [list(x) for x in section_key(sec)]
        if bw[q][0] + bw[q][1] == 9:
            out.append(None)
            continue
        bw[q][mover - 1] += 1
        out.append(keys[tuple(tuple(x) for x in bw)])
    return out


def test_slice35_small_sections_exhaustive(pp, slice36):
    import torch
    secs36, v36 = slice36
    secs, _ = pp.slice_sections(35)
    sizes = np.array([section_size(s) for s in secs])
    keep = sizes <= 600
    out = torch.zeros((int(sizes[keep].sum()), 8), dtype=torch.int64, device="cuda")
    pp.slice_step(35, v36, out, filter=keep.astype(np.uint8))
    torch.cuda.synchronize()
    got = to_host(out)
    row = 0
    checked = 0
    for si in np.nonzero(keep)[0]:
        for L in range(int(sizes[si])):
            assert (got[row] == oracle_section_value(35, secs[si], L)).all(), (si, L)
            row += 1
            checked += 1
    assert checked > 10000


def test_section_compute_matches_slice_step(pp, slice36):
    import torch
    secs36, v36 = slice36
    secs, total = pp.slice_sections(35)
    sizes = np.array([section_size(s) for s in secs])
    # a few sections of different shapes
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), len(secs) // 2, 17]
    for si in picks:
        sec = secs[si]
        kids = []
        for c in _children(secs36, sec, 35):
            kids.append(None if c is None else v36[int(c["offset"]):int(c["offset"]) + section_size(c)])
        one = torch.zeros((section_size(sec), 8), dtype=torch.int64, device="cuda")
        pp.section_compute(35, sec, kids, one)
        filt = np.zeros(len(secs), dtype=np.uint8)
        filt[si] = 1
        two = torch.zeros_like(one)
        pp.slice_step(35, v36, two, filter=filt)
        torch.cuda.synchronize()
        assert torch.equal(one, two)
        rng = inputs.SplitMix64(si)
        for _ in range(20):
            L = rng.below(section_size(sec))
            assert (to_host(one[L:L + 1])[0] == oracle_section_value(35, sec, L)).all()


def test_section_compute_with_child_descriptors(pp, slice36):
    """pp_section_compute_desc: with the child sections' descriptors the
    result is the same as without; a descriptor with other counts or dims is
    rejected (PP_EINVAL) before anything is written."""
    import torch
    secs36, v36 = slice36
    secs, _ = pp.slice_sections(35)
    sizes = np.array([section_size(s) for s in secs])
    sec = secs[int(np.argsort(sizes)[len(sizes) // 3])]
    cds = _children(secs36, sec, 35)
    kids = [None if c is None else v36[int(c["offset"]):int(c["offset"]) + section_size(c)] for c in cds]
    ref = torch.zeros((section_size(sec), 8), dtype=torch.int64, device="cuda")
    pp.section_compute(35, sec, kids, ref)
    got = torch.zeros_like(ref)
    pp.section_compute(35, sec, kids, got, child_descs=cds)
    torch.cuda.synchronize()
    assert torch.equal(ref, got)
    q = next(i for i, c in enumerate(cds) if c is not None)  # the one quadrant with an empty cell
    wrong_counts = cds[q].copy()
    wrong_counts["bw"] = sec["bw"]  # the parent's counts: the stone placed is missing
    wrong_dims = cds[q].copy()
    wrong_dims["dim"][q] += 1
    for bad in (wrong_counts, wrong_dims, None):
        descs = list(cds)
        descs[q] = bad
        sentinel = torch.full_like(ref, 7)
        with pytest.raises(pp.PentagoError) as e:
            pp.section_compute(35, sec, kids, sentinel, child_descs=descs)
        assert e.value.code == 1
        torch.cuda.synchronize()
        assert bool((sentinel == 7).all())


def test_section_compute_slice34_by_lines(pp, slice36):
    """pp_section_compute below slice 35 runs by lines: a few slice-34
    sections (two 8-stone quadrants, one 7-stone quadrant) built alone from
    their child sections (each a slice-35 section built alone from slice 36)
    agree with the oracle on sampled boards."""
    import torch
    secs36, v36 = slice36
    secs35, _ = pp.slice_sections(35)
    secs, _ = pp.slice_sections(34)
    sizes = np.array([section_size(s) for s in secs])
    counts = np.array([sorted(int(x[0]) + int(x[1]) for x in s["bw"]) for s in secs])
    two8 = np.nonzero((counts == [8, 8, 9, 9]).all(axis=1))[0]
    one7 = np.nonzero((counts == [7, 9, 9, 9]).all(axis=1))[0]
    picks = [int(two8[np.argmin(sizes[two8])]), int(one7[np.argmin(sizes[one7])]), int(two8[len(two8) // 2])]
    for si in picks:
        sec = secs[si]
        kids = []
        for c in _children(secs35, sec, 34):
            if c is None:
                kids.append(None)
                continue
            grand = []
            for g in _children(secs36, c, 35):
                grand.append(None if g is None else v36[int(g["offset"]):int(g["offset"]) + section_size(g)])
            t = torch.zeros((section_size(c), 8), dtype=torch.int64, device="cuda")
            pp.section_compute(35, c, grand, t)
            kids.append(t)
        lines = torch.zeros((section_size(sec), 8), dtype=torch.int64, device="cuda")
        pp.section_compute(34, sec, kids, lines)
        torch.cuda.synchronize()
        rng = inputs.SplitMix64(0x340 + si)
        for _ in range(40):
            L = rng.below(section_size(sec))
            assert (to_host(lines[L:L + 1])[0] == oracle_section_value(34, sec, L)).all(), (si, L)
        assert int(torch.count_nonzero(lines[:, :4] & ~lines[:, 4:])) == 0


def test_slice35_full_slice_sampled(pp, slice36):
    """The whole 36 -> 35 step in one call (the benchmarked launch)."""
    import torch
    secs36, v36 = slice36
    secs, total = pp.slice_sections(35)
    out = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(35, v36, out)
    torch.cuda.synchronize()
    win, notlose = out[:, :4], out[:, 4:]
    assert int(torch.count_nonzero(win & ~notlose)) == 0
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 35)
    picks = _sample(secs, rng, 3000)
    rows = torch.tensor([int(secs[si]["offset"]) + L for si, L in picks], device="cuda")
    got = to_host(out[rows])
    for (si, L), g in zip(picks, got):
        assert (g == oracle_section_value(35, secs[si], L)).all(), (si, L)
    # cross-path: the midgame solver on the same boards (one empty cell);
    # boards that show a five as given are not midgame inputs
    sel = [j for j, (si, L) in enumerate(picks[:800]) if not _shows_five(_board(secs[si], L))]
    boards = np.array([_board(*[secs[picks[j][0]], picks[j][1]]) for j in sel], dtype=np.uint64)
    ws = torch.empty(pp.midgame_workspace_bytes(len(boards), 1), dtype=torch.uint8, device="cuda")
    mg = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve(to_dev(boards), mg, 1, ws)
    assert (to_host(mg) == got[sel]).all()
    del out


def _board(sec, L):
    from oracle import enumeration as E
    return E.section_board(section_key(sec), unravel(L, [int(d) for d in sec["dim"]]))


def _shows_five(b):
    return inputs._shows_five(inputs.unpack_cells(int(b)))


def test_slice34_streamed_batch(pp, slice36):
    """Slice 34 from the full slice 35: a batch of (9,9,8,8)-type sections
    streamed into a compact buffer."""
    import torch
    secs36, v36 = slice36
    secs35, total35 = pp.slice_sections(35)
    v35 = torch.zeros((total35, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(35, v36, v35)
    secs, _ = pp.slice_sections(34)
    sizes = np.array([section_size(s) for s in secs])
    counts = np.array([[int(x[0]) + int(x[1]) for x in s["bw"]] for s in secs])
    two_axes = (counts >= 8).all(axis=1) & ((counts == 8).sum(axis=1) == 2)
    one_axis = (counts == 7).any(axis=1)
    keep = (two_axes | one_axis) & (sizes <= 20000)
    keep[np.nonzero(two_axes)[0][np.argsort(sizes[two_axes])][-3:]] = True  # three big ones
    out = torch.zeros((int(sizes[keep].sum()), 8), dtype=torch.int64, device="cuda")
    pp.slice_step(34, v35, out, filter=keep.astype(np.uint8))
    per_board = torch.zeros_like(out)
    pp.slice_step(34, v35, per_board, filter=keep.astype(np.uint8), opts=(0, 0, 0, 2))
    torch.cuda.synchronize()
    assert torch.equal(out, per_board)  # lines and one thread per board agree
    del per_board
    starts = np.concatenate([[0], np.cumsum(sizes[keep])])
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 34)
    idx = np.nonzero(keep)[0]
    for _ in range(1500):
        j = rng.below(len(idx))
        si = idx[j]
        L = rng.below(int(sizes[si]))
        got = to_host(out[int(starts[j]) + L:int(starts[j]) + L + 1])[0]
        assert (got == oracle_section_value(34, secs[si], L)).all(), (si, L)
    del v35


def test_slice35_line_kernel_equals_per_board_kernel(pp, slice36):
    """The staged line kernel and the one-thread-per-board kernel agree on
    every one of the 8.11e8 boards of slice 35."""
    import torch
    secs36, v36 = slice36
    secs, total = pp.slice_sections(35)
    a = torch.empty((total, 8), dtype=torch.int64, device="cuda")
    b = torch.empty((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(35, v36, a, opts=(0, 0, 0, 1))
    pp.slice_step(35, v36, b, opts=(0, 0, 0, 2))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    del a, b


def test_slice35_with_slice36_on_demand(pp, slice36):
    """Slice 36 on demand (paper, "Data layout and distribution": the last
    slice is computed when needed, not stored): slice 35 with no slice-36
    input equals slice 35 from the stored slice 36 on all 8.11e8 boards,
    through pp_slice_step and through a plan."""
    import torch
    secs36, v36 = slice36
    secs, total = pp.slice_sections(35)
    stored = torch.empty((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(35, v36, stored)
    fly = torch.empty_like(stored)
    pp.slice_step(35, None, fly)
    torch.cuda.synchronize()
    assert torch.equal(stored, fly)
    fly.zero_()
    plan = pp.SlicePlan(35, None, fly)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(stored, fly)
    plan.close()
    del stored, fly


def _period(code):
    """Smallest p in {1, 2, 4} with rot^p(code) = code."""
    from oracle import enumeration as E
    r1 = E.rotate_quadrant_code(code)
    if r1 == code:
        return 1
    return 2 if E.rotate_quadrant_code(r1) == code else 4


def _shift_bits(bits, q, p):
    """[n, 2, 256] bool -> values at g + p e_q."""
    idx = np.arange(256)
    g = (idx >> (2 * q)) & 3
    src = idx - (g << (2 * q)) + (((g + p) % 4) << (2 * q))
    return bits[:, :, src]


@pytest.mark.parametrize("n", [36, 35])
def test_symmetric_quadrant_tie_break_is_free(pp, slice36, n):
    """A child whose quadrant pattern is symmetric (period p < 4) can be
    standardised with any of its turns; the choice (here the smallest turn)
    cannot change any value because every stored value is periodic there:
    V(g + p e_q) = V(g) for all g, on every sampled board with such a
    quadrant."""
    import torch
    from oracle import enumeration as E
    from tests.gpu_helpers import bits_to_bool
    secs36, v36 = slice36
    if n == 36:
        secs, vals = secs36, v36
    else:
        secs, total = pp.slice_sections(35)
        vals = torch.empty((total, 8), dtype=torch.int64, device="cuda")
        pp.slice_step(35, None, vals)
        torch.cuda.synchronize()
    ms = E.minimal_states()
    rng = inputs.SplitMix64(0x7E + n)
    rows, checks = [], []
    for _ in range(6000):
        si = rng.below(len(secs))
        s = secs[si]
        L = rng.below(section_size(s))
        idx = unravel(L, [int(d) for d in s["dim"]])
        for q in range(4):
            code = ms[section_key(s)[q]][idx[q]]
            p = _period(code)
            if p < 4:
                rows.append(int(s["offset"]) + L)
                checks.append((q, p))
    assert len(rows) > 200
    got = bits_to_bool(to_host(vals[torch.tensor(rows, device="cuda")]))
    for (q, p) in set(checks):
        sel = [i for i, c in enumerate(checks) if c == (q, p)]
        b = got[sel]
        assert (b == _shift_bits(b, q, p)).all(), (n, q, p)
    if n == 35:
        del vals
