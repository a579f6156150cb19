"""Out-of-core steps (paper, "Data layout and distribution": slice n reads
only slice n+1, which may live outside the device): chosen D4 sections of
slice 32 from a slice 33 held half on the device and half in pinned host
memory, copied in per batch on a second stream through two staging halves.
The values equal the sparse step's from a device-resident input, bit for
bit (raw and prepared input), and a sample matches the oracle; a section
held nowhere and staging room too small are rejected before any launch."""
import numpy as np
import pytest

from tests.gpu_helpers import oracle_section_value, ready, section_size, to_host

pytestmark = pytest.mark.gpu

D4 = True
TARGETS = [501, 293, 137, 77, 1206]


@pytest.fixture(scope="module")
def held():
    """The targets' cone down to slice 33 (compact), the direct slice-32
    values, and slice 33 split between a device base and pinned host."""
    import torch
    pp = ready()
    f = np.zeros(pp.section_count(32, D4), dtype=np.uint8)
    f[TARGETS] = 1
    filters = {32: f}
    for n in (32, 33, 34):
        filters[n + 1] = pp.slice_children(n, filters[n], d4=D4)
    _, total36 = pp.slice_sections(36, D4)
    s36 = torch.empty((total36, 8), dtype=torch.int64, device="cuda")
    pp.slice_step(36, None, s36, d4=D4)
    _, n35 = pp.compact_offsets(35, filters[35], D4)
    vals = {35: torch.empty((n35, 8), dtype=torch.int64, device="cuda")}
    pp.slice_step(35, s36, vals[35], filter=filters[35], d4=D4)
    for n in (34, 33, 32):
        offs, _ = pp.compact_offsets(n + 1, filters[n + 1], D4)
        _, count = pp.compact_offsets(n, filters[n], D4)
        vals[n] = torch.empty((count, 8), dtype=torch.int64, device="cuda")
        pp.slice_step_sparse(n, vals[n + 1], offs, vals[n], filter=filters[n], d4=D4)
    torch.cuda.synchronize()
    secs33, _ = pp.slice_sections(33, D4)
    offs33, _ = pp.compact_offsets(33, filters[33], D4)
    read = np.flatnonzero(filters[33])
    on_device, on_host = read[0::2], read[1::2]
    dev_size = sum(section_size(secs33[i]) for i in on_device)
    stage = 2 * sum(section_size(secs33[i]) for i in on_host)  # each half holds every host section
    base = torch.zeros((dev_size + stage, 8), dtype=torch.int64, device="cuda")
    dev_offsets = np.full(len(secs33), pp.PP_ABSENT, dtype=np.uint64)
    host = [None] * len(secs33)
    at = 0
    for i in on_device:
        size = section_size(secs33[i])
        base[at:at + size] = vals[33][int(offs33[i]):int(offs33[i]) + size]
        dev_offsets[i] = at
        at += size
    for i in on_host:
        size = section_size(secs33[i])
        host[i] = vals[33][int(offs33[i]):int(offs33[i]) + size].cpu().pin_memory()
    torch.cuda.synchronize()
    return pp, filters, vals, base, dev_offsets, host, dev_size, stage


def _batches(pp):
    halves = []
    for part in (TARGETS[:2], TARGETS[2:]):
        f = np.zeros(pp.section_count(32, D4), dtype=np.uint8)
        f[part] = 1
        halves.append(f)
    return halves


def _run(pp, st, filters_):
    import torch
    copy = torch.cuda.Stream()
    outs, staged = [], 0
    for f in filters_:
        _, count = pp.compact_offsets(32, f, D4)
        out = torch.empty((count, 8), dtype=torch.int64, device="cuda")
        staged += st.step(out, filter=f, copy_stream=copy)
        outs.append(out)
    torch.cuda.synchronize()
    return outs, staged


def _want(pp, vals, filters, f):
    import torch
    secs32, _ = pp.slice_sections(32, D4)
    offs, _ = pp.compact_offsets(32, filters[32], D4)
    rows = [vals[32][int(offs[i]):int(offs[i]) + section_size(secs32[i])] for i in np.flatnonzero(f)]
    return torch.cat(rows)


def test_staged_equals_device_resident(held):
    import torch
    pp, filters, vals, base, dev_offsets, host, dev_size, stage = held
    st = pp.Stager(32, base, dev_offsets, host, dev_size, stage, d4=D4)
    batches = _batches(pp)
    outs, staged = _run(pp, st, batches + batches)  # twice: each half reused
    assert staged > 0
    for out, f in zip(outs, batches + batches):
        assert torch.equal(out, _want(pp, vals, filters, f))
    # a sample against the oracle
    secs32, _ = pp.slice_sections(32, D4)
    got = to_host(outs[0])
    i = int(np.flatnonzero(batches[0])[0])
    for L in (0, section_size(secs32[i]) // 2, section_size(secs32[i]) - 1):
        assert (got[L] == oracle_section_value(32, secs32[i], L)).all()


def test_staged_prepared(held):
    import torch
    pp, filters, vals, base, dev_offsets, host, dev_size, stage = held
    pbase = base.clone()
    pp.prepare_children(pbase[:dev_size], pbase[:dev_size])
    phost = []
    for t in host:
        if t is None:
            phost.append(None)
            continue
        d = t.cuda()
        pp.prepare_children(d, d)
        phost.append(d.cpu().pin_memory())
    torch.cuda.synchronize()
    st = pp.Stager(32, pbase, dev_offsets, phost, dev_size, stage, prepared=True, d4=D4)
    outs, _ = _run(pp, st, _batches(pp))
    for out, f in zip(outs, _batches(pp)):
        assert torch.equal(out, _want(pp, vals, filters, f))


def test_staged_ready(held):
    """The same with ready records (prepared = 2): the device part made
    ready in place through its offsets, each host section on its own."""
    import torch
    pp, filters, vals, base, dev_offsets, host, dev_size, stage = held
    rbase = base.clone()
    pp.prepare_children_ready(32, rbase[:dev_size], rbase[:dev_size], d4=D4, in_offsets=dev_offsets)
    rhost = []
    for i, t in enumerate(host):
        if t is None:
            rhost.append(None)
            continue
        d = t.cuda()
        offs = np.full(len(host), pp.PP_ABSENT, dtype=np.uint64)
        offs[i] = 0
        pp.prepare_children_ready(32, d, d, d4=D4, in_offsets=offs)
        rhost.append(d.cpu().pin_memory())
    torch.cuda.synchronize()
    st = pp.Stager(32, rbase, dev_offsets, rhost, dev_size, stage, prepared=2, d4=D4)
    outs, _ = _run(pp, st, _batches(pp))
    for out, f in zip(outs, _batches(pp)):
        assert torch.equal(out, _want(pp, vals, filters, f))


def test_stager_rejects(held):
    import torch
    pp, filters, vals, base, dev_offsets, host, dev_size, stage = held
    nowhere = list(host)
    i = next(j for j, t in enumerate(host) if t is not None)
    nowhere[i] = None
    st = pp.Stager(32, base, dev_offsets, nowhere, dev_size, stage, d4=D4)
    out = torch.empty((vals[32].shape[0], 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PentagoError) as e:
        st.step(out, filter=filters[32])
    assert e.value.code == 1
    small = pp.Stager(32, base, dev_offsets, host, dev_size, 2, d4=D4)  # one value per half
    with pytest.raises(pp.PentagoError) as e:
        small.step(out, filter=filters[32])
    assert e.value.code == 2
    with pytest.raises(pp.PentagoError) as e:  # a device section inside the staging room
        pp.Stager(32, base, dev_offsets, host, 0, stage, d4=D4)
    assert e.value.code == 1
