"""D4-reduced retrograde steps (paper, "Data layout and distribution": only
sections whose counts are least under D4 are computed; Fig. "lines": input
lines are turned before use) and the f_b -> f_{gb} transform they rest on
("Abstracting over rotations").

* the transform against its definition, bit for bit, for all eight
  symmetries and random turns;
* the transform reads a stored board for its preimage: f_c is the transform
  of the oracle's f_{c*}, c* the standardised image of c;
* slices 36, 35 and 34 of the D4-reduced chain equal the full layout on every
  stored board (the full layout is pinned to the oracle in
  test_gpu_sections), and sampled boards equal the oracle directly.
"""
import numpy as np
import pytest

import oracle
from oracle import enumeration as E
from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import (bits_to_bool, bool_to_bits, oracle_section_value, ready, section_key, section_size,
                               to_dev, to_host)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    return ready()


def _phi_plus_t(sym, turns, qmap, reflects):
    """src[beta(g)] = beta(phi_sym(g) + t)."""
    src = np.zeros(256, dtype=np.int64)
    for b in range(256):
        g = [(b >> (2 * q)) & 3 for q in range(4)]
        y = [0] * 4
        for q in range(4):
            y[qmap[q]] = (-g[q]) % 4 if reflects else g[q]
        y = [(y[p] + turns[p]) % 4 for p in range(4)]
        src[b] = y[0] + 4 * y[1] + 16 * y[2] + 64 * y[3]
    return src


def test_symmetry_transform_definition(pp):
    import torch
    rng = np.random.default_rng(7)
    vals = rng.integers(0, 2 ** 63, size=(96, 8), dtype=np.uint64) ^ rng.integers(0, 2, size=(96, 8), dtype=np.uint64) << np.uint64(63)
    d_in = to_dev(vals)
    bb = bits_to_bool(vals)
    for sym in range(8):
        qmap, reflects = pp.symmetry_info(sym)
        for turns in ([0, 0, 0, 0], [1, 2, 3, 0], [3, 1, 0, 2], list(rng.integers(0, 4, 4))):
            out = torch.empty_like(d_in)
            pp.symmetry_transform(d_in, sym, turns, out)
            want = bool_to_bits(bb[:, :, _phi_plus_t(sym, turns, qmap, reflects)])
            assert (to_host(out) == want).all(), (sym, turns)


def _standardise(code):
    """(minimal code m, turns t) with code = rot^t(m)."""
    orbit = [code]
    for _ in range(3):
        orbit.append(E.rotate_quadrant_code(orbit[-1]))
    m = min(orbit)
    # orbit[s] = rot^s(code) = m  =>  code = rot^(4 - s)(m)
    return m, (4 - orbit.index(m)) % 4


def test_symmetry_transform_reads_stored_board(pp):
    """f_c(g) = f_{c*}(phi_s(g) + t) where c* is s c with every quadrant
    standardised (t: its turns), on oracle values."""
    import torch
    boards = np.concatenate([inputs.midgame_boards(4, k, 0xD4A0 + k) for k in (3, 5)])
    stored, want, syms, turns = [], [], [], []
    for i, c in enumerate(boards):
        sym = i % 8
        sc = pp.symmetry_board(int(c), sym)
        t, cstar = [], 0
        for q in range(4):
            m, u = _standardise((sc >> (16 * q)) & 0xFFFF)
            cstar |= m << (16 * q)
            t.append(u)
        stored.append(oracle.midgame(cstar))
        want.append(oracle.midgame(int(c)))
        syms.append(sym)
        turns.append(t)
    for j in range(len(boards)):
        out = torch.empty((1, 8), dtype=torch.int64, device="cuda")
        pp.symmetry_transform(to_dev(np.array([stored[j]])), syms[j], turns[j], out)
        assert (to_host(out)[0] == want[j]).all(), j


def _child_symmetries(secs, n):
    """Symmetries through which the sections of slice n read their children
    (the first one reaching the child's least image)."""
    mover = 0 if n % 2 == 0 else 1
    used = set()
    for s in secs:
        for q in range(4):
            bw = [list(x) for x in section_key(s)]
            if bw[q][0] + bw[q][1] == 9:
                continue
            bw[q][mover] += 1
            imgs = E.section_images(tuple(tuple(x) for x in bw))
            used.add(imgs.index(min(imgs)))
    return used


def _full_rows(secs_full, secs_d4):
    """Row offsets in the full layout of every D4-minimal section."""
    at = {section_key(s): int(s["offset"]) for s in secs_full}
    return [at[section_key(s)] for s in secs_d4]


def _equal_on_minimal(full, secs_full, red, secs_d4):
    import torch
    for s, row in zip(secs_d4, _full_rows(secs_full, secs_d4)):
        n, o = section_size(s), int(s["offset"])
        if not torch.equal(red[o:o + n], full[row:row + n]):
            return section_key(s)
    return None


@pytest.fixture(scope="module")
def chain(pp):
    """D4-reduced slices 36 and 35, and the full layout's 36 and 35."""
    import torch
    out = {}
    for n in (36, 35):
        secs, total = pp.slice_sections(n, d4=True)
        v = torch.empty((total, 8), dtype=torch.int64, device="cuda")
        pp.slice_step(n, out.get(("d4", n + 1), (None,))[0] if n < 36 else None, v, d4=True)
        out[("d4", n)] = (v, secs)
        fsecs, ftotal = pp.slice_sections(n)
        fv = torch.empty((ftotal, 8), dtype=torch.int64, device="cuda")
        pp.slice_step(n, out.get(("full", n + 1), (None,))[0] if n < 36 else None, fv)
        out[("full", n)] = (fv, fsecs)
    torch.cuda.synchronize()
    return out


def test_d4_slice36_equals_full_layout(pp, chain):
    v, secs = chain[("d4", 36)]
    fv, fsecs = chain[("full", 36)]
    assert v.shape[0] == 9397647
    assert _equal_on_minimal(fv, fsecs, v, secs) is None


def test_d4_slice35_equals_full_layout(pp, chain):
    """Every one of the 1.20e8 stored boards of slice 35, read from the
    D4-reduced slice 36 through the symmetries."""
    v, secs = chain[("d4", 35)]
    fv, fsecs = chain[("full", 35)]
    assert v.shape[0] == 119704992
    assert _equal_on_minimal(fv, fsecs, v, secs) is None
    assert _child_symmetries(secs, 35) == {0, 1, 4}


def test_d4_slice35_line_path_equals_per_board(pp, chain):
    """Slice 35 by lines (sections whose child is stored as itself) plus one
    thread per board (the seven sections read through a symmetry) equals
    one thread per board everywhere; the plan equals the step."""
    import torch
    v36, _ = chain[("d4", 36)]
    v, secs = chain[("d4", 35)]
    b = torch.empty_like(v)
    pp.slice_step(35, v36, b, opts=(0, 0, 0, 2), d4=True)
    c = torch.empty_like(v)
    plan = pp.SlicePlan(35, v36, c, d4=True)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(v, b)
    assert torch.equal(v, c)
    plan.close()
    del b, c


def test_d4_slice35_oracle_samples(pp, chain):
    v, secs = chain[("d4", 35)]
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 350)
    for _ in range(400):
        si = rng.below(len(secs))
        L = rng.below(section_size(secs[si]))
        row = int(secs[si]["offset"]) + L
        assert (to_host(v[row:row + 1])[0] == oracle_section_value(35, secs[si], L)).all(), (si, L)


@pytest.fixture(scope="module")
def d4_34(pp, chain):
    """The whole D4-reduced slice 34 (9.85e8 boards, 63 GB) from the
    D4-reduced slice 35, through an autotuned plan."""
    import torch
    v35, _ = chain[("d4", 35)]
    secs, total = pp.slice_sections(34, d4=True)
    v = torch.empty((total, 8), dtype=torch.int64, device="cuda")
    plan = pp.SlicePlan(34, v35, v, d4=True)
    plan.autotune()
    plan.run()
    torch.cuda.synchronize()
    plan.close()
    return v, secs


def test_d4_slice34_equals_full_layout(pp, chain, d4_34):
    """The whole D4-reduced slice 34 (9.85e8 boards, 63 GB) from the
    D4-reduced slice 35, against the full layout's slice 34 computed section
    batch by section batch from the full slice 35, and against the oracle.
    Its children are read through seven of the eight symmetries (all but
    symmetry 6, which the transform tests cover)."""
    import torch
    v, secs = d4_34
    assert v.shape[0] == 985287494
    assert _child_symmetries(secs, 34) == {0, 1, 2, 3, 4, 5, 7}
    fv35, _ = chain[("full", 35)]
    fsecs, _ = pp.slice_sections(34)
    key_to_full = {section_key(s): i for i, s in enumerate(fsecs)}
    order = list(range(len(secs)))
    batch_cap = 160_000_000  # boards per comparison batch (10 GB)
    i = 0
    while i < len(order):
        sel, boards = [], 0
        while i < len(order) and (not sel or boards + section_size(secs[order[i]]) <= batch_cap):
            sel.append(order[i])
            boards += section_size(secs[order[i]])
            i += 1
        keep = np.zeros(len(fsecs), dtype=np.uint8)
        for j in sel:
            keep[key_to_full[section_key(secs[j])]] = 1
        buf = torch.empty((boards, 8), dtype=torch.int64, device="cuda")
        pp.slice_step(34, fv35, buf, filter=keep)  # compact, in full-layout section order
        fidx = sorted(key_to_full[section_key(secs[j])] for j in sel)
        at, o = {}, 0
        for f in fidx:
            at[f] = o
            o += section_size(fsecs[f])
        for j in sel:
            s = secs[j]
            n, off = section_size(s), int(s["offset"])
            r = at[key_to_full[section_key(s)]]
            assert torch.equal(v[off:off + n], buf[r:r + n]), section_key(s)
        del buf
    win, notlose = v[:, :4], v[:, 4:]
    assert int(torch.count_nonzero(win & ~notlose)) == 0
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 340)
    for _ in range(300):
        si = rng.below(len(secs))
        L = rng.below(section_size(secs[si]))
        row = int(secs[si]["offset"]) + L
        assert (to_host(v[row:row + 1])[0] == oracle_section_value(34, secs[si], L)).all(), (si, L)


def test_d4_slice34_lines_equal_per_board(pp, chain, d4_34):
    """Slice 34 by lines along a non-full quadrant (section_line_kernel,
    sections whose children need a symmetry left to one thread per board)
    and wholly one thread per board agree on every board, batch by batch."""
    import torch
    v35, _ = chain[("d4", 35)]
    v, secs = d4_34
    sizes = np.array([section_size(s) for s in secs])
    cap = 160_000_000
    i = 0
    while i < len(secs):
        sel, boards = [], 0
        while i < len(secs) and (not sel or boards + sizes[i] <= cap):
            sel.append(i)
            boards += int(sizes[i])
            i += 1
        keep = np.zeros(len(secs), dtype=np.uint8)
        keep[sel] = 1
        for stage in (1, 2):
            buf = torch.empty((boards, 8), dtype=torch.int64, device="cuda")
            pp.slice_step(34, v35, buf, filter=keep, opts=(0, 0, 0, stage), d4=True)
            o = 0
            for j in sel:
                n, off = int(sizes[j]), int(secs[j]["offset"])
                assert torch.equal(buf[o:o + n], v[off:off + n]), (stage, section_key(secs[j]))
                o += n
            del buf


def test_d4_slice34_ready_plan(pp, chain, d4_34):
    """A D4 slice-34 plan over ready records of the D4 slice 35
    (pp_prepare_children_ready, d4) writes the values of the plan over the
    raw slice 35, on a batch of sections about 1.2e8 boards in all, children
    read through symmetries included."""
    import torch
    v35, _ = chain[("d4", 35)]
    v, secs = d4_34
    sizes = np.array([section_size(s) for s in secs])
    keep = np.zeros(len(secs), dtype=np.uint8)
    acc = 0
    for i in np.argsort(-sizes):
        if acc + sizes[i] <= 120_000_000:
            keep[i] = 1
            acc += int(sizes[i])
    assert _child_symmetries([secs[i] for i in np.flatnonzero(keep)], 34) - {0}
    ready = torch.empty_like(v35)
    pp.prepare_children_ready(34, v35, ready, d4=True)
    out = torch.empty((acc, 8), dtype=torch.int64, device="cuda")
    plan = pp.SlicePlan(34, ready, out, filter=keep, d4=True)
    plan.set_prepared(2)
    plan.run()
    torch.cuda.synchronize()
    o = 0
    for j in np.flatnonzero(keep):
        n, off = int(sizes[j]), int(secs[j]["offset"])
        assert torch.equal(out[o:o + n], v[off:off + n]), section_key(secs[j])
        o += n
    plan.close()
    del ready, out


def _board(sec, L):
    return E.section_board(section_key(sec), [int(x) for x in _unravel(L, sec["dim"])])


def _unravel(L, dims):
    out = []
    for d in dims:
        out.append(L % int(d))
        L //= int(d)
    return out


def test_d4_slice33_batch(pp, d4_34):
    """D4-reduced slice 33 (three stones to place; 338 GB in all, produced
    in section batches) from the resident D4 slice 34: a batch of the
    smallest sections and three large ones, against the oracle on samples
    and against the midgame solver (which shares no standardisation or
    symmetry code with the section path) on 20000 boards."""
    import torch
    v34, _ = d4_34
    secs, total = pp.slice_sections(33, d4=True)
    assert len(secs) == 1343 and total == sum(section_size(s) for s in secs)
    sizes = np.array([section_size(s) for s in secs])
    order = np.argsort(sizes)
    keep = np.zeros(len(secs), dtype=np.uint8)
    keep[order[:400]] = 1
    keep[order[-3:]] = 1
    boards = int(sizes[keep == 1].sum())
    out = torch.empty((boards, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(33, v34, out, filter=keep, d4=True)
    other = torch.empty_like(out)
    pp.slice_step(33, v34, other, filter=keep, opts=(0, 0, 0, 2), d4=True)  # one thread per board
    torch.cuda.synchronize()
    assert torch.equal(out, other)
    del other
    idx = np.nonzero(keep)[0]
    starts = np.concatenate([[0], np.cumsum(sizes[idx])])
    win, notlose = out[:, :4], out[:, 4:]
    assert int(torch.count_nonzero(win & ~notlose)) == 0
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 330)
    picks = []
    for _ in range(20000):
        j = rng.below(len(idx))
        picks.append((j, rng.below(int(sizes[idx[j]]))))
    rows = torch.tensor([int(starts[j]) + L for j, L in picks], device="cuda")
    got = to_host(out[rows])
    for (j, L), g in list(zip(picks, got))[:200]:
        assert (g == oracle_section_value(33, secs[idx[j]], L)).all(), (idx[j], L)
    bl = np.array([_board(secs[idx[j]], L) for j, L in picks], dtype=np.uint64)
    ok = np.array([not inputs._shows_five(inputs.unpack_cells(int(b))) for b in bl])
    ws = torch.empty(pp.midgame_workspace_bytes(int(ok.sum()), 3), dtype=torch.uint8, device="cuda")
    mg = torch.zeros((int(ok.sum()), 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve(to_dev(bl[ok]), mg, 3, ws)
    assert (to_host(mg) == got[ok]).all()
    del out


def test_d4_step_rejects_bad_arguments(pp):
    import torch
    out = torch.empty((4, 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PentagoError):
        pp.slice_step(35, None, out, d4=True)
    with pytest.raises(pp.PentagoError):
        pp.symmetry_transform(out, 8, [0, 0, 0, 0], out)
    with pytest.raises(pp.PentagoError):
        pp.symmetry_transform(out, 1, [0, 4, 0, 0], out)
