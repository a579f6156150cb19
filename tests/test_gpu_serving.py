"""Continuous-batching server for midgame queries (paper, "Open source and
data": positions beyond the database are solved from scratch on request).

Every result is bit-exact against the oracle, and identical whether the query
ran alone or in a mix that made it share launches with others.  Admission
respects the arena footprint; late arrivals join at level boundaries and
finish while long queries are still running.
"""
import time

import numpy as np
import pytest

from paper_1404_0743_gb300 import inputs
from tests.gpu_helpers import midgame_oracle, ready

pytestmark = pytest.mark.gpu


def _server(pp, arena_bytes, slots=64, max_empty=12, parity=-1):
    import torch
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    return pp.Server(arena, max_slots=slots, max_empty=max_empty, parity=parity)


def _collect(srv, n, timeout=120):
    out = {}
    t = time.time()
    while len(out) < n and time.time() - t < timeout:
        srv.wait(1, 5.0)
        for r in srv.poll():
            out[r["req_id"]] = r
    assert len(out) == n, f"{len(out)} of {n} results"
    return out


def test_results_match_oracle():
    pp = ready()
    boards = np.concatenate([inputs.midgame_boards(5, k, 0x5E00 + k) for k in range(3, 10)])
    srv = _server(pp, 1 << 28)
    for i, b in enumerate(boards):
        srv.submit(int(b), i)
    res = _collect(srv, len(boards))
    want = midgame_oracle(boards)
    for i in range(len(boards)):
        assert res[i]["status"] == 0
        assert (res[i]["value"] == want[i]).all(), i
    srv.close()


def test_server_with_its_own_arena_matches_oracle():
    """pp_server_create_budget: the library allocates the arena from a byte
    budget and frees it on close; results as with a caller's arena."""
    pp = ready()
    boards = np.concatenate([inputs.midgame_boards(3, k, 0x5F00 + k) for k in (4, 7, 9)])
    srv = pp.Server(budget=1 << 27, max_slots=16, max_empty=10)
    for i, b in enumerate(boards):
        srv.submit(int(b), i)
    res = _collect(srv, len(boards))
    want = midgame_oracle(boards)
    for i in range(len(boards)):
        assert res[i]["status"] == 0
        assert (res[i]["value"] == want[i]).all(), i
    assert srv.stats()["arena_free_largest"] == 1 << 27
    srv.close()
    with pytest.raises(pp.PentagoError) as e:  # more than the device holds
        pp.Server(budget=1 << 50, max_slots=4, max_empty=8)
    assert e.value.code == 2
    with pytest.raises(ValueError):
        pp.Server(max_slots=4)


def test_same_result_alone_and_in_the_mix():
    pp = ready()
    probe = inputs.midgame_boards(1, 9, 0xA10E)[0]
    srv = _server(pp, 1 << 28)
    srv.submit(int(probe), 0)
    alone = _collect(srv, 1)[0]["value"]
    # the mix: the probe is submitted between waves of other queries, so it
    # shares launches with queries at other levels
    others = np.concatenate([inputs.midgame_boards(6, k, 0xB000 + k) for k in (6, 8, 10, 11)])
    rng = np.random.default_rng(0)
    order = rng.permutation(len(others))
    for j in order[:12]:
        srv.submit(int(others[j]), 100 + int(j))
    time.sleep(0.002)
    srv.submit(int(probe), 1)
    for j in order[12:]:
        srv.submit(int(others[j]), 100 + int(j))
    res = _collect(srv, 1 + len(others))
    assert (res[1]["value"] == alone).all()
    st = srv.stats()
    assert st["max_active"] >= 2
    want = midgame_oracle([probe])[0]
    assert (alone == want).all()
    srv.close()


def test_admission_by_footprint():
    pp = ready()
    boards = inputs.midgame_boards(4, 10, 0xF00D)
    # arena for exactly one query with 10 empty cells (17,303 fills of
    # compact fill table and 2^10 super values of five tables)
    srv = _server(pp, (17303 + 2 ** 10) * 64, slots=8, max_empty=10)
    for i, b in enumerate(boards):
        srv.submit(int(b), i)
    res = _collect(srv, len(boards))
    st = srv.stats()
    assert st["max_active"] == 1
    want = midgame_oracle(boards)
    for i in range(len(boards)):
        assert (res[i]["value"] == want[i]).all()
    # admission is in arrival order
    done = [res[i]["done_s"] for i in range(len(boards))]
    assert done == sorted(done)
    srv.close()


def test_late_arrivals_overlap_long_query():
    pp = ready()
    long_q = inputs.midgame_boards(1, 16, 0x10C)[0]  # 17 levels, 10 million fills
    short = inputs.midgame_boards(20, 5, 0x5C)        # 6 levels
    srv = _server(pp, 1 << 30, max_empty=16)
    srv.submit(int(long_q), 0)
    for i, b in enumerate(short):
        srv.submit(int(b), 1 + i)
    res = _collect(srv, 1 + len(short))
    # short queries admitted while the long one runs finish before it
    running = [i for i in range(len(short)) if res[1 + i]["admit_s"] < res[0]["done_s"]]
    assert running, "every short query arrived after the long one finished"
    assert all(res[1 + i]["done_s"] < res[0]["done_s"] for i in running)
    want = midgame_oracle(short)
    for i in range(len(short)):
        assert (res[1 + i]["value"] == want[i]).all()
    srv.close()


def test_submit_rejections():
    pp = ready()
    srv = _server(pp, 3 ** 8 * 64, slots=4, max_empty=10)
    with pytest.raises(pp.PentagoError) as e:  # five in a row as given
        srv.submit(inputs.pack_cells([1] * 5 + [2] * 5 + [0] * 26), 0)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:  # more empty cells than max_empty
        srv.submit(int(inputs.midgame_boards(1, 12, 1)[0]), 1)
    assert e.value.code == 1
    with pytest.raises(pp.PentagoError) as e:  # footprint larger than the arena
        srv.submit(int(inputs.midgame_boards(1, 10, 1)[0]), 2)
    assert e.value.code == 2
    srv.close()


@pytest.mark.parametrize("parity", [0, 1])
def test_parity_server_matches_oracle_on_its_class(parity):
    """A server on one parity class (half tables): results equal the oracle
    on that class and are zero on the other; the arena admits by the half
    footprint (3^k + 2^(k+1)) x 32 bytes."""
    from tests.test_gpu_parity import class_mask
    pp = ready()
    boards = np.concatenate([inputs.midgame_boards(4, k, 0x7A00 + k) for k in range(3, 11)])
    srv = _server(pp, 1 << 27, parity=parity)
    for i, b in enumerate(boards):
        srv.submit(int(b), i)
    res = _collect(srv, len(boards))
    want = midgame_oracle(boards) & class_mask(parity)
    for i in range(len(boards)):
        assert res[i]["status"] == 0
        assert (res[i]["value"] == want[i]).all(), i
    srv.close()
    # exactly one 10-empty query fits an arena of its half footprint
    # ((17,303 fills + 2^11 masks) x 32 bytes, rounded up to 64)
    qs = inputs.midgame_boards(3, 10, 0x7B10)
    half = (17303 + 2 ** 11 + 1) // 2 * 64
    srv = _server(pp, half, slots=4, max_empty=10, parity=parity)
    for i, b in enumerate(qs):
        srv.submit(int(b), i)
    res = _collect(srv, len(qs))
    assert srv.stats()["max_active"] == 1
    want = midgame_oracle(qs) & class_mask(parity)
    for i in range(len(qs)):
        assert (res[i]["value"] == want[i]).all()
    with pytest.raises(pp.PentagoError):  # the full footprint would not fit
        _server(pp, half, slots=4, max_empty=10).submit(int(qs[0]), 9)
    srv.close()


def test_deep_queries_served_against_stored_oracle_values():
    """The serving stream's queries with 14, 15 and 16 empty cells, served in
    one mix with smaller queries, bit for bit against the stored oracle
    values."""
    from tests.test_gpu_midgame import deep_rows
    pp = ready()
    rows = deep_rows()
    small = inputs.midgame_boards(8, 9, 0xDEE9)
    srv = _server(pp, 6 << 30, slots=64, max_empty=16)
    for i, _, b, _ in rows:
        srv.submit(b, i)
    for j, b in enumerate(small):
        srv.submit(int(b), 1000 + j)
    res = _collect(srv, len(rows) + len(small), timeout=300)
    for i, k, _, words in rows:
        assert res[i]["status"] == 0
        assert [int(x) for x in res[i]["value"]] == words, (i, k)
    want = midgame_oracle(small)
    for j in range(len(small)):
        assert (res[1000 + j]["value"] == want[j]).all()
    srv.close()
