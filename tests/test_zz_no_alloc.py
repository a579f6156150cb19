"""The allocation-free midgame entry point against the allocating one.

pp_midgame_solve_noalloc serves callers that may not allocate device memory;
it keeps all scratch in the library's fixed 64 MiB device array.  This file
is collected last so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process and after the others.
Two calls in a row (different batches, so the second overwrites the shared
array left by the first) must each match pp_midgame_solve bit for bit, the
tolerance of every parity test here.
"""
import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import ready, to_dev, to_host

pytestmark = pytest.mark.gpu


def _reference(pp, boards, max_empty):
    import torch
    ws = torch.empty(pp.midgame_workspace_bytes(len(boards), max_empty), dtype=torch.uint8, device="cuda")
    out = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve(to_dev(boards), out, max_empty, ws)
    torch.cuda.synchronize()
    return to_host(out)


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    pp = ready()
    first = np.concatenate([inputs.midgame_boards(24, 7, 0x7A11), inputs.midgame_boards(8, 4, 0x7A12)])
    second = inputs.midgame_boards(40, 9, 0x7A13)  # larger tables: overwrites the first call's scratch
    for boards, max_empty in ((first, 8), (second, 9)):
        out = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
        pp.midgame_solve_noalloc(to_dev(boards), out, max_empty)
        torch.cuda.synchronize()
        assert (to_host(out) == _reference(pp, boards, max_empty)).all()


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    import torch
    pp = ready()
    # 8 x 12 empty cells: 8 x (143,365 fills x 64 B + 2^13 masks x 32 B) > 64 MiB
    boards = inputs.midgame_boards(8, 12, 0x7A14)
    out = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PentagoError) as e:
        pp.midgame_solve_noalloc(to_dev(boards), out, 12)
    assert e.value.code == 2 and "64 MiB" in str(e.value)
