"""Shared helpers of the GPU tests (device marshalling only)."""
import numpy as np

import oracle
from oracle import enumeration as E


def dev():
    import torch
    return torch.device("cuda:0")


def ready():
    from paper_1404_0743_gb300 import build
    build.build()
    import paper_1404_0743_gb300 as pp
    pp.init()
    return pp


def to_dev(a_u64):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a_u64, dtype=np.uint64).view(np.int64)).to(dev())


def to_host(t):
    return t.cpu().numpy().view(np.uint64)


def section_key(s):
    return tuple(tuple(int(v) for v in row) for row in s["bw"])


def section_size(s):
    return int(np.prod(s["dim"].astype(np.int64)))


def unravel(L, dims):
    idx = []
    for d in dims:
        idx.append(int(L % d))
        L //= d
    return idx


def oracle_section_value(n, s, L):
    return oracle.section_value(n, section_key(s), unravel(L, [int(d) for d in s["dim"]]))


def midgame_oracle(boards, threads=None):
    return oracle.midgame_many([int(b) for b in boards], threads=threads)


def bits_to_bool(sv):
    """[n, 8] uint64 -> [n, 2, 256] bool, bit beta of table t."""
    sv = np.asarray(sv, dtype=np.uint64)
    out = np.zeros((sv.shape[0], 2, 256), dtype=bool)
    for t in range(2):
        for word in range(4):
            w = sv[:, 4 * t + word]
            for b in range(64):
                out[:, t, 64 * word + b] = (w >> np.uint64(b)) & np.uint64(1)
    return out


def bool_to_bits(bb):
    n = bb.shape[0]
    out = np.zeros((n, 8), dtype=np.uint64)
    for t in range(2):
        for word in range(4):
            acc = np.zeros(n, dtype=np.uint64)
            for b in range(64):
                acc |= bb[:, t, 64 * word + b].astype(np.uint64) << np.uint64(b)
            out[:, 4 * t + word] = acc
    return out


def beta(g):
    return g[0] + 4 * g[1] + 16 * g[2] + 64 * g[3]


def digits(b):
    return [(b >> (2 * q)) & 3 for q in range(4)]


E = E
