"""Midgame solves on one parity class of the rotations (paper, "Open source
and data": rmax flips the parity of g0 + g1 + g2 + g3, so such a solve needs
one class per level and stores 32 bytes per position instead of 64).

The result on the wanted class equals the oracle's value there, bit for
bit; the other class is zero.  Both classes, every batching mode, the
1024-board workload against stored oracle values, mixed numbers of empty
cells, and the half-size workspace (which is too small for a full solve).
"""
import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import midgame_oracle, ready, to_dev, to_host
from tests.test_gpu_midgame import _golden

pytestmark = pytest.mark.gpu


def class_mask(parity):
    """[8] uint64 words: bit beta set iff beta(g) has g0+g1+g2+g3 = parity (mod 2)."""
    words = np.zeros(4, dtype=np.uint64)
    for beta in range(256):
        par = (beta ^ (beta >> 2) ^ (beta >> 4) ^ (beta >> 6)) & 1
        if par == parity:
            words[beta >> 6] |= np.uint64(1) << np.uint64(beta & 63)
    return np.concatenate([words, words])


def _solve(pp, boards, max_empty, parity):
    import torch
    ws = torch.empty(pp.midgame_parity_workspace_bytes(len(boards), max_empty), dtype=torch.uint8, device="cuda")
    out = torch.full((len(boards), 8), -1, dtype=torch.int64, device="cuda")
    pp.midgame_solve_parity(to_dev(boards), out, max_empty, parity, ws)
    torch.cuda.synchronize()
    return to_host(out)


def test_class_masks_split_the_rotations():
    a, b = class_mask(0), class_mask(1)
    assert ((a & b) == 0).all() and ((a | b) == np.uint64(2 ** 64 - 1)).all()
    assert int(a[0]) & 1  # g = 0 (the position as given) is in class 0


@pytest.mark.parametrize("parity", [0, 1])
def test_plain_workload_on_one_class(parity):
    pp = ready()
    boards = inputs.plain_midgame_boards(64)
    got = _solve(pp, boards, 6, parity)
    want = midgame_oracle(boards)
    m = class_mask(parity)
    assert (got == (want & m)).all()


@pytest.mark.parametrize("parity", [0, 1])
def test_mixed_empties_on_one_class(parity):
    pp = ready()
    boards = np.concatenate([inputs.midgame_boards(5, k, 0x9A00 + k) for k in range(10)])
    boards = boards[np.random.default_rng(9).permutation(len(boards))]
    got = _solve(pp, boards, 9, parity)
    assert (got == (midgame_oracle(boards) & class_mask(parity))).all()


@pytest.fixture(scope="module")
def workload():
    import torch
    pp = ready()
    boards = inputs.batched_midgame_boards(1024)
    plan = pp.MidgamePlan(boards, 12)
    ws = torch.empty(pp.midgame_parity_workspace_bytes(1024, 12), dtype=torch.uint8, device="cuda")
    return pp, boards, plan, ws


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("parity", [0, 1])
def test_batched_workload_every_mode(workload, mode, parity):
    """The 1024 x 12 workload in a half-size workspace, against the stored
    oracle values (every 16th board) masked to the class."""
    import torch
    pp, boards, plan, ws = workload
    plan.configure(mode)
    plan.set_parity(parity)
    out = torch.full((1024, 8), -1, dtype=torch.int64, device="cuda")
    plan.run(ws, out)
    plan.status()
    got = to_host(out)
    m = class_mask(parity)
    for i, _, words in _golden():
        assert (got[i] == (np.array(words, dtype=np.uint64) & m)).all(), (mode, parity, i)
    assert ((got & ~m) == 0).all()


def test_half_workspace_is_half(workload):
    """The parity workspace holds the half-size fill tables; a full solve
    does not fit in it."""
    import torch
    pp, boards, plan, ws = workload
    full = pp.midgame_workspace_bytes(1024, 12)
    half = pp.midgame_parity_workspace_bytes(1024, 12)
    assert half == 1024 * (143365 * 32 + 2 ** 13 * 32 + 64)  # 143,365 fills of 12 empty cells
    assert half < full
    plan.set_parity(-1)
    out = torch.zeros((1024, 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PentagoError) as e:
        plan.run(ws, out)
    assert e.value.code == 2
    with pytest.raises(pp.PentagoError):
        plan.set_parity(2)


def test_full_and_half_agree_on_the_class():
    """The same plan run full, then on class 0: class 0 bits agree."""
    import torch
    pp = ready()
    boards = inputs.midgame_boards(40, 11, 0x11AA)
    plan = pp.MidgamePlan(boards, 11)
    ws = torch.empty(pp.midgame_workspace_bytes(len(boards), 11), dtype=torch.uint8, device="cuda")
    full = torch.zeros((len(boards), 8), dtype=torch.int64, device="cuda")
    plan.run(ws, full)
    plan.set_parity(0)
    half = torch.zeros_like(full)
    plan.run(ws, half)  # a full-size workspace also serves a half plan
    plan.status()
    m = class_mask(0)
    assert (to_host(half) == (to_host(full) & m)).all()
