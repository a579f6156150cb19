"""Write the oracle's digests of whole sections of slices 36, 35 and 34.

Calls only the CPU oracle (oracle/) and the board generator of the section
layout (oracle.enumeration); nothing here touches the CUDA library.  For
every section of slice 36, every section of slice 35 with at most 100,000
boards and every section of slice 34 with at most 30,000 boards, every
board of the section is valued by the oracle (O3: the section's board
decoded through the plain minimal-state lists and valued by the
rotation-separate retrograde), and the digest of the section's values in
layout order (tests/golden/digests.py) is written, one line per section:
    <slice> <b0 w0 b1 w1 b2 w2 b3 w3> <boards> <win bits> <not-lose bits> <sha256 prefix>
About 5e7 + 3e7 + 1.6e7 oracle evaluations: about an hour on 8 host
threads.  --slices recomputes only the given slices and keeps the file's
lines of the others.
Run:  python tests/golden/make_section_digests.py [--threads N] [--slices 36,35,34]
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import enumeration as E  # noqa: E402
from tests.golden.digests import digest  # noqa: E402

OUT = os.path.join(HERE, "section_digests.txt")
MAX_BOARDS = {36: None, 35: 100_000, 34: 30_000}  # None: every section


def sections(n):
    """Count tuples of slice n's sections and their sizes."""
    return [(t, E.section_size(t)) for t in E.sections(n)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--slices", default="36,35,34")
    args = ap.parse_args()
    todo = [int(x) for x in args.slices.split(",")]
    keep = []
    if os.path.exists(OUT):
        keep = [line.rstrip("\n") for line in open(OUT)
                if not line.startswith("#") and line.strip() and int(line.split()[0]) not in todo]
    rows = list(keep)
    for n in todo:
        for t, size in sections(n):
            if MAX_BOARDS[n] is not None and size > MAX_BOARDS[n]:
                continue
            t0 = time.time()
            vals = oracle.midgame_batch(oracle.section_boards(t), threads=args.threads)
            w, nl, h = digest(vals)
            rows.append(f"{n} " + " ".join(f"{b} {c}" for b, c in t) + f" {size} {w} {nl} {h}")
            if size > 200_000:
                print(f"slice {n} section {t}: {size} boards, {time.time() - t0:.1f} s", flush=True)
    rows.sort(key=lambda r: (-int(r.split()[0]), tuple(int(x) for x in r.split()[1:9])))
    with open(OUT, "w") as f:
        f.write("# oracle digests of whole sections: slice 36 (every section), slice 35 (every section of\n")
        f.write("# at most 100000 boards), slice 34 (every section of at most 30000 boards); slice, (black,\n")
        f.write("# white) per quadrant, boards, set win bits, set not-lose bits, first 16 hex digits of the\n")
        f.write("# SHA-256 of the values (tests/golden/digests.py)\n")
        for r in rows:
            f.write(r + "\n")
    print(f"wrote {len(rows)} sections to {OUT}")


if __name__ == "__main__":
    main()
