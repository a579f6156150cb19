"""Degenerate section batches: a filter that keeps no section launches
nothing and writes nothing, through the one-shot step, a plan (run and
autotuned) and the sparse step, in both layouts; a one-board section
computes its value.  The output array is a sentinel row that must stay
untouched."""
import numpy as np
import pytest

from tests.gpu_helpers import oracle_section_value, ready, section_size, to_host

pytestmark = pytest.mark.gpu

SENTINEL = 0x5A5A5A5A5A5A5A5A


def _sentinel():
    import torch
    return torch.full((1, 8), SENTINEL, dtype=torch.int64, device="cuda")


@pytest.mark.parametrize("d4", [False, True])
@pytest.mark.parametrize("n", [36, 35, 34, 33])
def test_empty_filter_writes_nothing(n, d4):
    import torch
    pp = ready()
    none = np.zeros(pp.section_count(n, d4), dtype=np.uint8)
    child = None
    if n == 35 and d4:
        # slice 35 turns its whole slice-36 input into the line kernel's forms
        # whatever the filter keeps, so the input must be the whole slice
        child = torch.empty((pp.slice_sections(36, d4)[1], 8), dtype=torch.int64, device="cuda")
        pp.slice_step(36, None, child, d4=True)
    elif n <= 34:
        # sparse input with every section absent: nothing may be read
        child = torch.zeros((8, 8), dtype=torch.int64, device="cuda")
    out = _sentinel()
    if n <= 34:
        offs = np.full(pp.section_count(n + 1, d4), pp.PP_ABSENT, dtype=np.uint64)
        pp.slice_step_sparse(n, child, offs, out, filter=none, d4=d4)
        plan = pp.SlicePlan(n, child, out, filter=none, d4=d4, in_offsets=offs)
    else:
        pp.slice_step(n, child, out, filter=none, d4=d4)
        plan = pp.SlicePlan(n, child, out, filter=none, d4=d4)
    plan.run()
    plan.autotune()
    plan.close()
    torch.cuda.synchronize()
    assert (to_host(out) == np.uint64(SENTINEL)).all()


def test_one_board_sections():
    """Slice-36 sections of one board: each value equals the oracle's."""
    import torch
    pp = ready()
    secs, _ = pp.slice_sections(36)
    ones = [i for i, s in enumerate(secs) if section_size(s) == 1]
    assert ones
    keep = np.zeros(len(secs), dtype=np.uint8)
    keep[ones] = 1
    out = torch.empty((len(ones), 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, out, filter=keep)
    torch.cuda.synchronize()
    got = to_host(out)
    for row, i in enumerate(ones):
        assert (got[row] == oracle_section_value(36, secs[i], 0)).all()
