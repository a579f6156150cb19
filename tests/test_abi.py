"""The C-ABI library builds, loads and exports every declared symbol, and its
host-side layout (quadrant lists, sections) equals the oracle's enumeration.
No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import enumeration as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pentago_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1404_0743_gb300 import build
    build.build()
    import paper_1404_0743_gb300 as pp
    return pp.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("pp_init", "pp_midgame_solve", "pp_section_compute", "pp_slice_step",
                     "pp_midgame_plan_create", "pp_midgame_plan_run", "pp_midgame_solve_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_1404_0743_gb300 import _native
    for name in declared_functions():
        assert name in _native._SIGNATURES, f"{name} has no Python binding"


def test_struct_sizes():
    from paper_1404_0743_gb300 import _native
    assert ctypes.sizeof(_native.SectionDesc) == 24
    assert ctypes.sizeof(_native.BatchOpts) == 20


def test_quadrant_lists_match_oracle(lib):
    import paper_1404_0743_gb300 as pp
    ms = E.minimal_states()
    for b in range(10):
        for w in range(10 - b):
            assert list(pp.quadrant_states(b, w)) == ms[(b, w)], (b, w)


@pytest.mark.parametrize("n", [0, 1, 17, 18, 33, 34, 35, 36])
def test_sections_match_oracle(lib, n):
    import paper_1404_0743_gb300 as pp
    secs, total = pp.slice_sections(n)
    want = E.sections(n)
    assert len(secs) == len(want)
    d = E.dims()
    offset = 0
    for s, t in zip(secs, want):
        assert tuple(tuple(int(v) for v in row) for row in s["bw"]) == t
        assert [int(x) for x in s["dim"]] == [d[x] for x in t]
        assert int(s["offset"]) == offset
        offset += int(np.prod([d[x] for x in t]))
    assert total == offset


def test_host_errors_without_gpu(lib):
    import paper_1404_0743_gb300 as pp
    with pytest.raises(pp.PentagoError):
        pp.quadrant_states(5, 5)
    with pytest.raises(pp.PentagoError):
        pp.slice_sections(37)
    with pytest.raises(pp.PentagoError):
        pp.midgame_workspace_bytes(4, 17)


def test_workspace_size(lib):
    import paper_1404_0743_gb300 as pp
    # per board: compact fill table (one 64 B entry per fill of every level:
    # sum_m C(k, m) C(m, ceil(m/2)) fills), five tables of both colours over
    # every subset of the empty cells (2 x 2^k x 32 B), one result
    from math import comb
    fills = {k: sum(comb(k, m) * comb(m, (m + 1) // 2) for m in range(k + 1)) for k in (12, 16)}
    assert fills[12] == 143365 and fills[16] == 10165779
    assert pp.midgame_workspace_bytes(1024, 12) == 1024 * (fills[12] * 64 + 2 ** 13 * 32 + 64)
    assert pp.midgame_workspace_bytes(1, 16) == fills[16] * 64 + 2 ** 17 * 32 + 64


def test_plan_requires_init_or_validates(lib):
    """Plan creation validates boards on the host before touching the GPU."""
    import paper_1404_0743_gb300 as pp
    with pytest.raises(pp.PentagoError):
        pp.MidgamePlan(np.array([0xFFFF], dtype=np.uint64), 16)
