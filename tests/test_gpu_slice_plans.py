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
