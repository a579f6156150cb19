"""The stored oracle digests of whole sections (tests/golden/
section_digests.txt) cover what they claim: every section of slice 36,
every slice-35 section of at most 100,000 boards and every slice-34 section
of at most 30,000 boards, each with its size; one small section of each
slice is recomputed by the oracle as it stands."""
import os

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


SECTIONS = os.path.join(HERE, "section_digests.txt")


def test_section_digests_cover_what_they_claim():
    """Every slice-36 section, every slice-35 section of at most 100,000
    boards and every slice-34 section of at most 30,000, with its size; one
    small section of each slice recomputed by the oracle."""
    from oracle import enumeration as E
    from tests.golden.digests import digest
    rows = {}
    for line in open(SECTIONS):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        key = tuple((int(f[1 + 2 * q]), int(f[2 + 2 * q])) for q in range(4))
        rows[(int(f[0]), key)] = (int(f[9]), int(f[10]), int(f[11]), f[12])
    want = ({(36, t) for t in E.sections(36)} |
            {(35, t) for t in E.sections(35) if E.section_size(t) <= 100_000} |
            {(34, t) for t in E.sections(34) if E.section_size(t) <= 30_000})
    assert set(rows) == want
    for (n, t), (size, _, _, _) in rows.items():
        assert size == E.section_size(t)
    for n in (36, 35, 34):
        t = min((t for (m, t) in rows if m == n), key=lambda t: (E.section_size(t), t))
        vals = oracle.midgame_batch(oracle.section_boards(t))
        assert digest(vals) == rows[(n, t)][1:]
