"""Autotuner cache on the device: a second plan of the same shape takes the
recorded choice and times nothing (a hit); another parity class, board mix
or set of sections is another shape (a miss); PP_AUTOTUNE_CACHE carries the
choices to a later process.  A plan configured from the cache computes the
oracle's values."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import midgame_oracle, ready, section_size, to_dev, to_host

pytestmark = pytest.mark.gpu

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_midgame_second_plan_hits():
    import torch
    pp = ready()
    pp.autotune_cache_clear()
    boards = inputs.midgame_boards(48, 8, 0xCAC)
    ws = torch.empty(pp.midgame_workspace_bytes(48, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros((48, 8), dtype=torch.int64, device="cuda")
    first = pp.MidgamePlan(boards, 8).autotune(ws, out)
    assert pp.autotune_cache_stats() == (1, 0, 1)
    again = boards[::-1].copy()  # same numbers of empty cells, other boards' order
    plan = pp.MidgamePlan(again, 8)
    assert plan.autotune(ws, out) == first
    assert pp.autotune_cache_stats() == (1, 1, 1)
    out.zero_()
    plan.run(ws, out)
    plan.status()
    assert (to_host(out) == midgame_oracle(again)).all()
    plan.set_parity(0)  # another shape
    plan.autotune(ws, out)
    assert pp.autotune_cache_stats() == (2, 1, 2)
    mixed = np.concatenate([boards[:40], inputs.midgame_boards(8, 7, 0xCAD)])  # another board mix
    pp.MidgamePlan(mixed, 8).autotune(ws, out[:48])
    assert pp.autotune_cache_stats() == (3, 1, 3)
    pp.autotune_cache_clear()


def test_slice_plan_second_plan_hits():
    import torch
    pp = ready()
    pp.autotune_cache_clear()
    secs, _ = pp.slice_sections(36)
    order = np.argsort([section_size(s) for s in secs])
    picks = []
    for chosen in (order[:6], order[6:12]):
        f = np.zeros(len(secs), dtype=np.uint8)
        f[chosen] = 1
        total = sum(section_size(secs[i]) for i in chosen)
        picks.append((f, torch.empty((total, 8), dtype=torch.int64, device="cuda")))
    # the per-board slice-36 plans (stage_children 2): the line kernel that
    # slice 36 takes by default has a single configuration and no tuning
    per_board = (0, 0, 0, 2, 0)
    f, out = picks[0]
    first = pp.SlicePlan(36, None, out, filter=f, opts=per_board).autotune()
    assert pp.autotune_cache_stats() == (1, 0, 1)
    want = out.clone()
    out.zero_()
    plan = pp.SlicePlan(36, None, out, filter=f, opts=per_board)
    assert plan.autotune() == first
    assert pp.autotune_cache_stats() == (1, 1, 1)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(out, want)
    lines = torch.zeros_like(out)
    pp.SlicePlan(36, None, lines, filter=f).run()  # by lines: the same values
    torch.cuda.synchronize()
    assert torch.equal(lines, want)
    f2, out2 = picks[1]
    pp.SlicePlan(36, None, out2, filter=f2, opts=per_board).autotune()  # other sections: a miss
    assert pp.autotune_cache_stats() == (2, 1, 2)
    pp.autotune_cache_clear()


CHILD = """
import sys
import torch
sys.path.insert(0, {repo!r})
import paper_1404_0743_gb300 as pp
from paper_1404_0743_gb300 import inputs
pp.init()
boards = inputs.midgame_boards(32, 6, 0xCAE)
plan = pp.MidgamePlan(boards, 6)
ws = torch.empty(pp.midgame_workspace_bytes(32, 6), dtype=torch.uint8, device="cuda")
out = torch.zeros((32, 8), dtype=torch.int64, device="cuda")
print(*plan.autotune(ws, out), *pp.autotune_cache_stats())
"""


def test_cache_file_carries_choices_to_a_later_process(tmp_path):
    ready()  # built
    path = tmp_path / "tune.txt"
    env = dict(os.environ, PP_AUTOTUNE_CACHE=str(path))
    runs = []
    for _ in range(2):
        res = subprocess.run([sys.executable, "-c", CHILD.format(repo=REPO)], env=env, capture_output=True,
                             text=True, timeout=300)
        assert res.returncode == 0, res.stderr
        runs.append([int(v) for v in res.stdout.split()])
    (m1, c1, e1, h1, x1), (m2, c2, e2, h2, x2) = runs
    assert (e1, h1, x1) == (1, 0, 1)  # tuned and written
    assert (e2, h2, x2) == (1, 1, 0)  # read back: no timing
    assert (m1, c1) == (m2, c2)
    lines = [ln for ln in path.read_text().splitlines() if ln and not ln.startswith("#")]
    assert len(lines) == 1 and "midgame parity=-1 max_empty=6 boards=6:32," in lines[0]


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_one_shot_solves_take_the_cached_mode(tmp_path, mode):
    """A one-shot solve of a shape in the cache runs in the cached mode (a
    graph choice keeps the default), counts neither hit nor miss, and
    computes the oracle's values, from device and from host arrays."""
    import torch
    pp = ready()
    pp.autotune_cache_clear()
    boards = inputs.midgame_boards(40, 9, 0xCAF)
    prop = torch.cuda.get_device_properties(0)
    key = f"sm_{prop.major}{prop.minor}x{prop.multi_processor_count} midgame parity=-1 max_empty=9 boards=9:40,"
    f = tmp_path / "one.txt"
    f.write_text(f"{key}\t{mode} 0 0 0 0\n")
    assert pp.autotune_cache_load(f) == 1
    want = midgame_oracle(boards)
    ws = torch.empty(pp.midgame_workspace_bytes(40, 9) + 40 * 64, dtype=torch.uint8, device="cuda")
    out = torch.zeros((40, 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve(to_dev(boards), out, 9, ws)
    torch.cuda.synchronize()
    assert (to_host(out) == want).all()
    hout = torch.zeros((40, 8), dtype=torch.int64).pin_memory()
    pp.midgame_solve_host(torch.from_numpy(boards.view(np.int64)).pin_memory(), hout, 9, ws)
    assert (hout.numpy().view(np.uint64) == want).all()
    assert pp.autotune_cache_stats() == (1, 0, 0)
    pp.autotune_cache_clear()
