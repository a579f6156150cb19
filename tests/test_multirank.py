"""The benchmark's multi-GPU logic on CPU with two gloo ranks: each rank
solves its own, disjoint boards (no collective on the data path), and only
the timing is reduced (max over ranks) to form the whole-job rate."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    boards = bench.rank_boards(rank)[:16]  # the first boards of each rank's block
    slowest = bench.max_over_ranks(1.0 + rank, world, device="cpu")
    rate = bench.whole_job_rate(100, world, slowest)
    out[rank] = (boards.tolist(), slowest, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_boards_and_max_timing():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    b0, s0, r0 = out[0]
    b1, s1, r1 = out[1]
    assert not set(b0) & set(b1)                 # independent problems per rank
    assert s0 == s1 == 2.0                       # max over ranks
    assert r0 == r1 == pytest.approx(2 * 100 / 2.0)
    from paper_1404_0743_gb300 import inputs
    assert b0 == [int(x) for x in inputs.batched_midgame_boards(16)]
