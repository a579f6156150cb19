"""Arguments the library rejects on the host, before any launch: value arrays
of the section and slice calls, midgame workspaces and server arenas must be
32-byte aligned (they are read and written 256 bits at a time); parity
classes are -1, 0 or 1.  Each rejection is PP_EINVAL and leaves the context
usable (a valid call follows)."""
import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import midgame_oracle, ready, to_dev, to_host

pytestmark = pytest.mark.gpu


def _off16(nbytes):
    """A device buffer whose start is 16-byte but not 32-byte aligned."""
    import torch
    raw = torch.empty(nbytes + 64, dtype=torch.uint8, device="cuda")
    base = raw.data_ptr() % 32
    view = raw[(16 - base) % 32:][:nbytes] if base != 16 else raw[:nbytes]
    assert view.data_ptr() % 32 == 16
    return raw, view


def test_slice_step_needs_32_byte_arrays():
    import torch
    pp = ready()
    _, total = pp.slice_sections(36, d4=True)
    keep, view = _off16(total * 64)
    out = view.view(torch.int64).view(total, 8)
    with pytest.raises(pp.PentagoError) as e:
        pp.slice_step(36, None, out, d4=True)
    assert e.value.code == 1
    good = torch.empty((total, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, good, d4=True)  # still works
    torch.cuda.synchronize()


def test_midgame_workspace_needs_32_bytes():
    import torch
    pp = ready()
    boards = inputs.midgame_boards(4, 5, 0x5A1)
    plan = pp.MidgamePlan(boards, 5)
    nb = pp.midgame_workspace_bytes(4, 5)
    keep, ws = _off16(nb)
    out = torch.zeros((4, 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PentagoError) as e:
        plan.run(ws, out)
    assert e.value.code == 1
    good = torch.empty(nb, dtype=torch.uint8, device="cuda")
    plan.run(good, out)
    plan.status()
    assert (to_host(out) == midgame_oracle(boards)).all()


def test_server_arena_needs_32_bytes():
    pp = ready()
    keep, arena = _off16(1 << 20)
    with pytest.raises(pp.PentagoError) as e:
        pp.Server(arena, max_slots=4, max_empty=8)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError):
        import torch
        pp.Server(torch.empty(1 << 20, dtype=torch.uint8, device="cuda"), max_slots=4, max_empty=8, parity=3)


def test_parity_arguments():
    import torch
    pp = ready()
    boards = inputs.midgame_boards(2, 4, 0x5A2)
    ws = torch.empty(pp.midgame_parity_workspace_bytes(2, 4), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 8), dtype=torch.int64, device="cuda")
    for bad in (-1, 2):
        with pytest.raises(pp.PentagoError) as e:
            pp.midgame_solve_parity(to_dev(boards), out, 4, bad, ws)
        assert e.value.code == 1
    pp.midgame_solve_parity(to_dev(boards), out, 4, 1, ws)
    torch.cuda.synchronize()
    got = to_host(out)
    assert ((got[:, :4] & ~got[:, 4:]) == 0).all()
