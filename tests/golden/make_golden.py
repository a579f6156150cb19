"""Write stored expected values of the midgame workloads.

Calls only the CPU oracle (oracle/); nothing here touches the CUDA library.
Two sets, each one text file in this folder:

* ``--set k12``: batched_midgame_k12.txt, every one of the 1024 seeded
  12-empty boards of the batched workload (about 35 s of oracle time each,
  one board per host thread), one line per board:
      <board index> <packed board hex> <8 super-value words hex>
* ``--set deep``: serving_deep_k14_16.txt, the first queries of the serving
  stream with 14, 15 and 16 empty cells (4, 3 and 2 of them; up to 11 GB of
  oracle table and several minutes of all host threads each), one line per
  query:
      <query index> <empty cells> <packed board hex> <8 super-value words hex>

Run:  python tests/golden/make_golden.py --set k12|deep [--threads N]
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1404_0743_gb300 import inputs  # noqa: E402

K12 = os.path.join(HERE, "batched_midgame_k12.txt")
DEEP = os.path.join(HERE, "serving_deep_k14_16.txt")
DEEP_COUNTS = {14: 4, 15: 3, 16: 2}


def deep_queries():
    """(query index, k, board) of the serving stream's first queries with
    14, 15 and 16 empty cells, in stream order."""
    boards, ks = inputs.serving_queries(10000)
    want = dict(DEEP_COUNTS)
    out = []
    for i, (b, k) in enumerate(zip(boards, ks)):
        k = int(k)
        if want.get(k, 0) > 0:
            want[k] -= 1
            out.append((i, k, int(b)))
        if not any(want.values()):
            break
    return out


def _words(v):
    return " ".join(f"{int(w):016x}" for w in v)


def write_k12(threads):
    boards = inputs.batched_midgame_boards(1024)
    vals = oracle.midgame_many([int(b) for b in boards], threads=threads)
    with open(K12, "w") as f:
        f.write("# batched midgame workload (seed 0x14040743 + 1000 + i, 12 empty cells), every board:\n")
        f.write("# board index, packed board, oracle super value (win[4], notlose[4])\n")
        for i, v in enumerate(vals):
            f.write(f"{i} {int(boards[i]):016x} {_words(v)}\n")
    print(f"wrote 1024 boards to {K12}")


def write_deep(threads):
    rows = []
    for i, k, b in deep_queries():
        t = time.time()
        v = oracle.midgame(b, threads=threads)
        print(f"query {i}: {k} empty cells, {time.time() - t:.0f} s", flush=True)
        rows.append((i, k, b, v))
    with open(DEEP, "w") as f:
        f.write("# serving workload (seed 0x14040743 + 5000 + i): the first queries with 14, 15 and 16\n")
        f.write("# empty cells; query index, empty cells, packed board, oracle super value\n")
        f.write("# (win[4], notlose[4])\n")
        for i, k, b, v in rows:
            f.write(f"{i} {k} {b:016x} {_words(v)}\n")
    print(f"wrote {len(rows)} queries to {DEEP}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--set", choices=["k12", "deep"], required=True)
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    (write_k12 if args.set == "k12" else write_deep)(args.threads)


if __name__ == "__main__":
    main()
