"""Whole sections of slices 36, 35 and 34 against the oracle, bit for bit:
every section of slice 36, every section of slice 35 with at most 100,000
boards (1,672 of its 2,460 sections) and every section of slice 34 with at
most 30,000 boards (1,860 of 5,660), each digested (set win bits, set
not-lose bits, SHA-256 of its values in layout order) and compared with the
digest of the oracle's values of the same section (tests/golden/
section_digests.txt, written by tests/golden/make_section_digests.py from
the oracle alone).  Slice 35 is checked as the stored step computes it
(from slice 36) and with slice 36 on demand; slice 34 as a filtered step
from slice 35 values as they are and as a plan reading prepared values."""
import os

import numpy as np
import pytest

from tests.golden.digests import digest
from tests.gpu_helpers import ready, to_host

pytestmark = pytest.mark.gpu
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "section_digests.txt")


def _stored():
    rows = {}
    for line in open(PATH):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        n = int(f[0])
        key = tuple((int(f[1 + 2 * q]), int(f[2 + 2 * q])) for q in range(4))
        rows[(n, key)] = (int(f[9]), int(f[10]), int(f[11]), f[12])
    return rows


def _check(pp, n, values, rows, compact=False):
    """Digest every stored section of slice n in values (the whole slice, or
    with compact=True the stored sections back to back in section order)."""
    secs, _ = pp.slice_sections(n)
    host = to_host(values)
    checked, at = 0, 0
    for s in secs:
        key = tuple((int(x[0]), int(x[1])) for x in s["bw"])
        if (n, key) not in rows:
            continue
        size = int(np.prod(s["dim"].astype(np.int64)))
        off = at if compact else int(s["offset"])
        at += size
        boards, w, nl, h = rows[(n, key)]
        assert boards == size, key
        assert digest(host[off:off + size]) == (w, nl, h), (n, key)
        checked += 1
    return checked


def test_slices_36_and_35_against_oracle_digests():
    import torch
    pp = ready()
    rows = _stored()
    _, t36 = pp.slice_sections(36)
    _, t35 = pp.slice_sections(35)
    v36 = torch.empty((t36, 8), dtype=torch.int64, device="cuda")
    v35 = torch.empty((t35, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, v36)
    pp.slice_step(35, v36, v35)
    torch.cuda.synchronize()
    assert _check(pp, 36, v36, rows) == 670
    assert _check(pp, 35, v35, rows) == 1672
    pp.slice_step(35, None, v35)  # slice 36 on demand
    torch.cuda.synchronize()
    assert _check(pp, 35, v35, rows) == 1672
    # slice 34: the stored sections as one filtered step, then as plans on
    # ready and on prepared slice-35 values
    del v36
    secs34, _ = pp.slice_sections(34)
    keep = np.array([(34, tuple((int(x[0]), int(x[1])) for x in s["bw"])) in rows for s in secs34], dtype=np.uint8)
    _, count = pp.compact_offsets(34, keep)
    v34 = torch.empty((count, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(34, v35, v34, filter=keep)
    torch.cuda.synchronize()
    assert _check(pp, 34, v34, rows, compact=True) == 1860
    ready35 = torch.empty_like(v35)
    pp.prepare_children_ready(34, v35, ready35)
    plan = pp.SlicePlan(34, ready35, v34, filter=keep)
    plan.set_prepared(2)
    v34.zero_()
    plan.run()
    torch.cuda.synchronize()
    assert _check(pp, 34, v34, rows, compact=True) == 1860
    plan.close()
    del ready35
    pp.prepare_children(v35, v35)
    plan = pp.SlicePlan(34, v35, v34, filter=keep)
    plan.set_prepared(True)
    v34.zero_()
    plan.run()
    torch.cuda.synchronize()
    assert _check(pp, 34, v34, rows, compact=True) == 1860
