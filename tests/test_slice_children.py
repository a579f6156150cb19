"""Child sections read by a set of sections (paper, "Data layout and
distribution": slice n needs only slice n+1, one child section per quadrant
that can take a stone), on the host: the library's marks equal the rule
applied to the oracle's enumeration, with least images under D4 taken from
the oracle's section images; every section of slice n+1 has a parent; the
compact offsets of a filtered step place kept sections back to back.  No
kernel is launched here."""
import numpy as np
import pytest

from oracle import enumeration as E


@pytest.fixture(scope="module")
def pp():
    from paper_1404_0743_gb300 import build
    build.build()
    import paper_1404_0743_gb300 as pp
    return pp


def _children(n, t, d4):
    """Sections of slice n+1 read by section t of slice n."""
    mover = 0 if n % 2 == 0 else 1  # black moves when the counts are equal
    out = set()
    for q in range(4):
        if sum(t[q]) >= 9:
            continue
        c = [list(x) for x in t]
        c[q][mover] += 1
        c = tuple(tuple(x) for x in c)
        out.add(min(E.section_images(c)) if d4 else c)
    return out


@pytest.mark.parametrize("d4", [False, True])
@pytest.mark.parametrize("n", [0, 1, 17, 26, 31, 32, 33, 34, 35])
def test_children_follow_the_rule(pp, n, d4):
    parents = [t for t in E.sections(n) if not d4 or E.is_d4_minimal(t)]
    kids = [t for t in E.sections(n + 1) if not d4 or E.is_d4_minimal(t)]
    index = {t: i for i, t in enumerate(kids)}
    rng = np.random.default_rng(n + 100 * d4)
    for trial in range(4):
        keep = rng.random(len(parents)) < 0.05 * (trial + 1)
        got = pp.slice_children(n, keep.astype(np.uint8), d4=d4)
        want = np.zeros(len(kids), dtype=np.uint8)
        for t, k in zip(parents, keep):
            if k:
                for c in _children(n, t, d4):
                    want[index[c]] = 1
        assert (got == want).all()


@pytest.mark.parametrize("d4", [False, True])
@pytest.mark.parametrize("n", [0, 9, 30, 33, 35])
def test_every_child_section_has_a_parent(pp, n, d4):
    assert pp.slice_children(n, None, d4=d4).all()


def test_compact_offsets(pp):
    secs, _ = pp.slice_sections(33, d4=True)
    keep = np.zeros(len(secs), dtype=np.uint8)
    keep[[3, 10, 11, 500]] = 1
    offs, total = pp.compact_offsets(33, keep, d4=True)
    sizes = [int(np.prod(secs[i]["dim"].astype(np.int64))) for i in (3, 10, 11, 500)]
    assert [int(offs[i]) for i in (3, 10, 11, 500)] == [0, sizes[0], sizes[0] + sizes[1], sum(sizes[:3])]
    assert total == sum(sizes)
    assert int((offs != np.uint64(pp.PP_ABSENT)).sum()) == 4


def test_children_errors(pp):
    with pytest.raises(pp.PentagoError):
        pp.slice_children(36)
    with pytest.raises(ValueError):
        pp.slice_children(30, np.ones(3, dtype=np.uint8))


@pytest.mark.parametrize("d4", [False, True])
def test_no_parents_no_children(pp, d4):
    none = np.zeros(pp.section_count(30, d4), dtype=np.uint8)
    assert not pp.slice_children(30, none, d4=d4).any()
