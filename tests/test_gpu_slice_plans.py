"""Batched section steps (slice plans): every execution mode and the
autotuner's choice give the same values as the one-shot step, bit for bit,
and a plan replays inside a captured CUDA graph.  The digest kernel agrees
with numpy."""
import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import oracle_section_value, ready, section_size, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slices():
    import torch
    pp = ready()
    s36, t36 = pp.slice_sections(36)
    s35, t35 = pp.slice_sections(35)
    v36 = torch.empty((t36, 8), dtype=torch.int64, device="cuda")
    v35 = torch.empty((t35, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, v36)
    pp.slice_step(35, v36, v35)
    torch.cuda.synchronize()
    return pp, v36, v35


def _batch34(pp, max_boards=3_000_000):
    secs, _ = pp.slice_sections(34)
    sizes = np.array([section_size(s) for s in secs])
    counts = np.array([[int(x[0]) + int(x[1]) for x in s["bw"]] for s in secs])
    eligible = (counts >= 8).all(axis=1)
    keep = np.zeros(len(secs), dtype=np.uint8)
    acc = 0
    for i in np.nonzero(eligible)[0]:
        if acc + sizes[i] <= max_boards:
            keep[i] = 1
            acc += sizes[i]
    return secs, sizes, keep, acc


@pytest.mark.parametrize("opts", [(2, 0, 0, 0, 0), (2, 0, 0, 0, 1), (1, 0, 0, 0, 1), (1, 0, 1, 0, 0)])
def test_slice34_plan_modes(slices, opts):
    import torch
    pp, v36, v35 = slices
    secs, sizes, keep, total = _batch34(pp)
    ref = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(34, v35, ref, filter=keep)
    out = torch.zeros_like(ref)
    plan = pp.SlicePlan(34, v35, out, filter=keep, opts=opts)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # sampled parity against the oracle
    idx = np.nonzero(keep)[0]
    starts = np.concatenate([[0], np.cumsum(sizes[keep.astype(bool)])])
    rng = inputs.SplitMix64(inputs.SEED_SECTIONS + 340)
    for _ in range(200):
        j = rng.below(len(idx))
        L = rng.below(int(sizes[idx[j]]))
        row = int(starts[j]) + L
        assert (to_host(out[row:row + 1])[0] == oracle_section_value(34, secs[idx[j]], L)).all()


def test_plan_autotune_and_graph_replay(slices):
    import torch
    pp, v36, v35 = slices
    secs, sizes, keep, total = _batch34(pp, 1_000_000)
    ref = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(34, v35, ref, filter=keep)
    out = torch.zeros_like(ref)
    plan = pp.SlicePlan(34, v35, out, filter=keep)
    chosen = plan.autotune()
    assert chosen[0] in (1, 2)
    out.zero_()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.run(stream=s)  # warm
    torch.cuda.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_slice35_plan_line_kernel(slices):
    import torch
    pp, v36, v35 = slices
    out = torch.empty_like(v35)
    plan = pp.SlicePlan(35, v36, out)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(out, v35)
    del out


def test_digest_matches_numpy(slices):
    import torch
    pp, v36, v35 = slices
    vals = v36[:100003]
    acc = torch.zeros(4, dtype=torch.int64, device="cuda")
    pp.super_digest(vals, acc)
    acc2 = torch.zeros(4, dtype=torch.int64, device="cuda")
    pp.super_digest(vals, acc2)
    torch.cuda.synchronize()
    host = to_host(vals)
    bits = np.unpackbits(host.view(np.uint8), axis=1).reshape(len(host), 2, 256)
    a = acc.cpu().numpy()
    assert a[0] == bits[:, 0].sum() and a[1] == bits[:, 1].sum() and a[3] == len(host)
    assert torch.equal(acc, acc2)
    flipped = vals.clone()
    flipped[12345, 3] ^= 1 << 7
    acc3 = torch.zeros(4, dtype=torch.int64, device="cuda")
    pp.super_digest(flipped, acc3)
    torch.cuda.synchronize()
    assert int(acc3[2]) != int(acc[2])


def _rmax_bool(bb):
    """rmax over [n, 256] bool tables (paper, "Abstracting over rotations"):
    out[g] = OR over the 8 single-quadrant quarter turns r of bb[g + r]."""
    x = bb.reshape(-1, 4, 4, 4, 4)  # axes g3, g2, g1, g0 (beta = g0 + 4 g1 + 16 g2 + 64 g3)
    out = np.zeros_like(x)
    for ax in (1, 2, 3, 4):
        out |= np.roll(x, 1, axis=ax) | np.roll(x, -1, axis=ax)
    return out.reshape(-1, 256)


def test_prepare_children_definition(slices):
    """Prepared form of slice-35 values: win slot ~rmax(~win), not-lose slot
    ~rmax(~notlose), in place too."""
    import torch
    from tests.gpu_helpers import bits_to_bool, bool_to_bits
    pp, v36, v35 = slices
    vals = v35[:30011].clone()
    prep = torch.empty_like(vals)
    pp.prepare_children(vals, prep)
    torch.cuda.synchronize()
    bb = bits_to_bool(to_host(vals))
    want = np.stack([~_rmax_bool(~bb[:, 0]), ~_rmax_bool(~bb[:, 1])], axis=1)
    assert (to_host(prep) == bool_to_bits(want)).all()
    pp.prepare_children(vals, vals)  # in place
    torch.cuda.synchronize()
    assert torch.equal(vals, prep)


@pytest.mark.parametrize("opts", [(2, 0, 0, 1, 0), (2, 0, 0, 2, 0), (1, 0, 0, 2, 1)])
def test_prepared_plan_equals_raw(slices, opts):
    """A slice-34 plan reading prepared slice-35 values (by lines, one
    thread per board, persistent) writes the same values, bit for bit, as
    the step reading the values as they are."""
    import torch
    pp, v36, v35 = slices
    secs, sizes, keep, total = _batch34(pp, 2_000_000)
    ref = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(34, v35, ref, filter=keep, opts=(2, 0, 0, 2, 0))
    prep = torch.empty_like(v35)
    pp.prepare_children(v35, prep)
    out = torch.zeros_like(ref)
    plan = pp.SlicePlan(34, prep, out, filter=keep, opts=opts)
    plan.set_prepared(True)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # and back: the same plan told the input is raw, on the raw values
    plan2 = pp.SlicePlan(34, v35, out, filter=keep, opts=opts)
    plan2.set_prepared(True)
    plan2.set_prepared(False)
    out.zero_()
    plan2.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    del prep


def test_ready_children_definition(slices):
    """Ready records of slice-35 values for slice 34 (black to move): each
    slot is the prepared slot with black's five-in-a-row set cleared (win
    slot ~(F_b | rmax(~win)) = ~rmax(~win) & ~F_b), in place too; F_b from
    the oracle's boards of each section through pp_five_masks."""
    import torch
    from oracle import section_boards
    from tests.gpu_helpers import section_key
    pp, v36, v35 = slices
    secs, _ = pp.slice_sections(35)
    sizes = np.array([section_size(s) for s in secs])
    picks = [int(i) for i in np.argsort(sizes)[[0, 7, 40, len(sizes) // 2]]]
    prep = torch.empty_like(v35)
    pp.prepare_children(v35, prep)
    ready = torch.empty_like(v35)
    pp.prepare_children_ready(34, v35, ready)
    torch.cuda.synchronize()
    for si in picks:
        sec = secs[si]
        lo, n = int(sec["offset"]), section_size(sec)
        if n > 200_000:
            continue
        boards = torch.from_numpy(section_boards(section_key(sec)).view(np.int64)).cuda()
        masks = torch.empty((n, 8), dtype=torch.int64, device="cuda")
        pp.five_masks(boards, masks)
        fb = masks[:, :4]
        want = prep[lo:lo + n].clone()
        want[:, :4] &= ~fb
        want[:, 4:] &= ~fb
        assert torch.equal(ready[lo:lo + n], want), si
    pp.prepare_children_ready(34, v35, prep)  # in place over a copy
    torch.cuda.synchronize()
    assert torch.equal(prep, ready)
    del prep, ready


def test_ready_children_rejects(slices):
    """Input shorter than the slice's layout, a section offset past the
    values, and a slice with no children below it: PP_EINVAL, nothing
    written."""
    import torch
    pp, v36, v35 = slices
    out = torch.full((1024, 8), 7, dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PentagoError) as e:
        pp.prepare_children_ready(34, v35[:1024], out)
    assert e.value.code == 1
    secs35, _ = pp.slice_sections(35)
    offs = np.full(len(secs35), pp.PP_ABSENT, dtype=np.uint64)
    offs[int(np.argmin([section_size(x) for x in secs35]))] = 1023  # every section holds 3 values or more
    with pytest.raises(pp.PentagoError) as e:
        pp.prepare_children_ready(34, v35[:1024], out, in_offsets=offs)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:
        pp.prepare_children_ready(35, v36[:1024], out)
    assert e.value.code == 1
    sizes35 = np.array([section_size(x) for x in secs35])
    small = np.argsort(sizes35)[:2]
    offs = np.full(len(secs35), pp.PP_ABSENT, dtype=np.uint64)
    offs[small[0]], offs[small[1]] = 0, 1  # the second starts inside the first
    with pytest.raises(pp.PentagoError) as e:
        pp.prepare_children_ready(34, v35[:1024], out, in_offsets=offs)
    assert e.value.code == 1
    torch.cuda.synchronize()
    assert bool((out == 7).all())


@pytest.mark.parametrize("opts", [(2, 0, 0, 1, 0), (2, 0, 0, 2, 0), (1, 0, 0, 2, 1)])
def test_ready_plan_equals_raw(slices, opts):
    """A slice-34 plan reading ready slice-35 records (by lines, one thread
    per board, persistent) writes the same values as the step reading the
    values as they are; so does a sparse step over a subset of slice 35."""
    import torch
    pp, v36, v35 = slices
    secs, sizes, keep, total = _batch34(pp, 2_000_000)
    ref = torch.zeros((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(34, v35, ref, filter=keep, opts=(2, 0, 0, 2, 0))
    ready = torch.empty_like(v35)
    pp.prepare_children_ready(34, v35, ready)
    out = torch.zeros_like(ref)
    plan = pp.SlicePlan(34, ready, out, filter=keep, opts=opts)
    plan.set_prepared(2)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    # sparse: only the slice-35 sections the kept sections read, back to back
    kids = np.flatnonzero(pp.slice_children(34, keep))
    secs35, _ = pp.slice_sections(35)
    offs = np.full(len(secs35), pp.PP_ABSENT, dtype=np.uint64)
    parts, at = [], 0
    for i in kids:
        lo, n = int(secs35[i]["offset"]), section_size(secs35[i])
        offs[i] = at
        parts.append(v35[lo:lo + n])
        at += n
    sub = torch.cat(parts)
    pp.prepare_children_ready(34, sub, sub, in_offsets=offs)
    out.zero_()
    sp = pp.SlicePlan(34, sub, out, filter=keep, opts=opts, in_offsets=offs)
    sp.set_prepared(2)
    sp.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    del ready, sub


def test_prepared_only_below_slice35(slices):
    import torch
    pp, v36, v35 = slices
    out = torch.empty((16, 8), dtype=torch.int64, device="cuda")
    plan = pp.SlicePlan(35, v36, out, filter=_one_section(pp, 35))
    with pytest.raises(pp.PentagoError) as e:
        plan.set_prepared(True)
    assert e.value.code == 1


def _one_section(pp, n):
    secs, _ = pp.slice_sections(n)
    sizes = np.array([section_size(s) for s in secs])
    keep = np.zeros(len(secs), dtype=np.uint8)
    keep[int(np.argmin(sizes))] = 1
    return keep
