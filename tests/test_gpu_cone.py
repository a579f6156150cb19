"""Slices below 34 through dependency cones (paper, "Data layout and
distribution": slice n reads only slice n+1, one child section per quadrant
that can take a stone).  Chosen D4 sections of slice 32 are computed from
the top down: the whole D4 slice 36, then at each slice only the sections
the next slice down reads, each step's compact output serving as the sparse
input of the step below.

Checks: slice-32 values against the oracle (every board of the small
sections, samples of a larger one); the sparse step at slice 34 equals the
step from the whole D4 slice 35, by lines and one thread per board, as a
step and as a plan; a section read but absent, or an input too short, is
rejected before any launch.
"""
import numpy as np
import pytest

from tests.gpu_helpers import oracle_section_value, ready, section_size, to_host

pytestmark = pytest.mark.gpu

D4 = True
TARGETS = [501, 293, 137, 1206]  # D4 slice-32 sections: three small cones, one of 1.7e6 values


def _filters(pp, targets):
    f = np.zeros(pp.section_count(32, D4), dtype=np.uint8)
    f[targets] = 1
    filters = {32: f}
    for n in (32, 33, 34):
        filters[n + 1] = pp.slice_children(n, filters[n], d4=D4)
    return filters


@pytest.fixture(scope="module")
def cone():
    import torch
    pp = ready()
    filters = _filters(pp, TARGETS)
    _, total36 = pp.slice_sections(36, D4)
    s36 = torch.empty((total36, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, s36, d4=D4)
    _, n35 = pp.compact_offsets(35, filters[35], D4)
    vals = {35: torch.empty((n35, 8), dtype=torch.int64, device="cuda")}
    pp.slice_step(35, s36, vals[35], filter=filters[35], d4=D4)
    for n in (34, 33, 32):
        offs, _ = pp.compact_offsets(n + 1, filters[n + 1], D4)
        _, count = pp.compact_offsets(n, filters[n], D4)
        vals[n] = torch.empty((count, 8), dtype=torch.int64, device="cuda")
        pp.slice_step_sparse(n, vals[n + 1], offs, vals[n], filter=filters[n], d4=D4)
    torch.cuda.synchronize()
    return pp, filters, s36, vals


def test_slice32_against_oracle(cone):
    pp, filters, _, vals = cone
    secs, _ = pp.slice_sections(32, D4)
    offs, _ = pp.compact_offsets(32, filters[32], D4)
    got = to_host(vals[32])
    rng = np.random.default_rng(32)
    checked = 0
    for i in TARGETS:
        size = section_size(secs[i])
        picks = range(size) if size <= 100 else rng.choice(size, 40, replace=False)
        for L in picks:
            want = oracle_section_value(32, secs[i], int(L))
            assert (got[int(offs[i]) + int(L)] == want).all(), (i, int(L))
            checked += 1
    assert checked >= 300


@pytest.mark.parametrize("stage", [1, 2])
def test_sparse_equals_whole_input_at_slice34(cone, stage):
    """Slice 34 on the cone's sections: from the compact slice-35 cone (sparse)
    and from the whole D4 slice 35, by lines (1) and one thread per board (2)."""
    import torch
    pp, filters, s36, vals = cone
    _, total35 = pp.slice_sections(35, D4)
    whole35 = torch.empty((total35, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(35, s36, whole35, d4=D4)
    want = torch.empty_like(vals[34])
    pp.slice_step(34, whole35, want, filter=filters[34], opts=(0, 0, 0, stage, 0), d4=D4)
    got = torch.empty_like(vals[34])
    offs, _ = pp.compact_offsets(35, filters[35], D4)
    pp.slice_step_sparse(34, vals[35], offs, got, filter=filters[34], opts=(0, 0, 0, stage, 0), d4=D4)
    plan_out = torch.empty_like(vals[34])
    plan = pp.SlicePlan(34, vals[35], plan_out, filter=filters[34], opts=(0, 0, 0, stage, 0), d4=D4,
                        in_offsets=offs)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(got, want) and torch.equal(vals[34], want) and torch.equal(plan_out, want)
    del whole35


def test_sparse_input_errors(cone):
    import torch
    pp, filters, _, vals = cone
    offs, _ = pp.compact_offsets(33, filters[33], D4)
    out = torch.empty_like(vals[32])
    read = np.flatnonzero(filters[33])
    bad = offs.copy()
    bad[read[0]] = np.uint64(pp.PP_ABSENT)  # a section the step reads
    with pytest.raises(pp.PentagoError) as e:
        pp.slice_step_sparse(32, vals[33], bad, out, filter=filters[32], d4=D4)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:  # input shorter than the offsets say
        pp.slice_step_sparse(32, vals[33][:-1], offs, out, filter=filters[32], d4=D4)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:
        pp.SlicePlan(32, vals[33], out, filter=filters[32], d4=D4, in_offsets=bad)
    assert e.value.code == 1
    offs35 = np.zeros(pp.section_count(36, D4), dtype=np.uint64)
    with pytest.raises(pp.PentagoError) as e:  # slice 35 reads slice 36 whole
        pp.slice_step_sparse(35, vals[35], offs35, out, d4=D4)
    assert e.value.code == 1
    pp.slice_step_sparse(32, vals[33], offs, out, filter=filters[32], d4=D4)  # still usable
    torch.cuda.synchronize()
    assert torch.equal(out, vals[32])
