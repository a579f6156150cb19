"""Invariants of the super value checked on the kernels' own results at a size
beyond the oracle's reach (14 empty cells), so they pin the GPU path by
themselves (paper, "Abstracting over rotations"):

* win implies not-lose;
* L-equivariance: super(h s)[g] = super(s)[g + h] for quadrant turns h;
* D4 invariance: super(d s)[phi_d(g)] = super(s)[g] for the 8 board
  symmetries (a reflection reverses the turn direction).

Each board and all its images are solved in one batched call.
"""
import numpy as np
import pytest

import oracle
from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import bits_to_bool, ready, to_dev, to_host

pytestmark = pytest.mark.gpu

TURNS = ([1, 0, 0, 0], [0, 3, 0, 0], [0, 0, 2, 1], [3, 1, 2, 3])


def _beta(g):
    return g[0] + 4 * g[1] + 16 * g[2] + 64 * g[3]


def _g(beta):
    return [(beta >> (2 * q)) & 3 for q in range(4)]


def test_invariants_at_fourteen_empty_cells():
    import torch
    pp = ready()
    roots = inputs.midgame_boards(3, 14, 0x14E)
    batch, jobs = [], []
    for r, s in enumerate(roots):
        s = int(s)
        batch.append(s)
        jobs.append(("root", r, None))
        for h in TURNS:  # h s, unless it shows five as given (not a midgame input)
            hs = oracle.rotate(s, _beta(h))
            if not (oracle.has_five(hs, 0, 1) or oracle.has_five(hs, 0, 2)):
                batch.append(hs)
                jobs.append(("turn", r, h))
        for d in range(8):
            batch.append(pp.symmetry_board(s, d))
            jobs.append(("sym", r, d))
    ws = torch.empty(pp.midgame_workspace_bytes(len(batch), 14), dtype=torch.uint8, device="cuda")
    out = torch.zeros((len(batch), 8), dtype=torch.int64, device="cuda")
    pp.midgame_solve(to_dev(np.array(batch, dtype=np.uint64)), out, 14, ws)
    torch.cuda.synchronize()
    vals = bits_to_bool(to_host(out))  # [n, 2, 256]
    assert not (vals[:, 0] & ~vals[:, 1]).any()  # win => not lose
    root_of = {r: i for i, (kind, r, _) in enumerate(jobs) if kind == "root"}
    turned = symmetric = 0
    for i, (kind, r, arg) in enumerate(jobs):
        base = vals[root_of[r]]
        if kind == "turn":
            for beta in range(256):
                g = _g(beta)
                gh = [(g[q] + arg[q]) % 4 for q in range(4)]
                assert (vals[i][:, beta] == base[:, _beta(gh)]).all(), (r, arg, beta)
            turned += 1
        elif kind == "sym":
            qmap, reflects = pp.symmetry_info(arg)
            for beta in range(256):
                g = _g(beta)
                y = [0] * 4
                for q in range(4):
                    y[qmap[q]] = (-g[q]) % 4 if reflects else g[q]
                assert (vals[i][:, _beta(y)] == base[:, beta]).all(), (r, arg, beta)
            symmetric += 1
    assert turned >= 6 and symmetric == 24
