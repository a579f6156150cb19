"""Write stored expected values for the batched midgame workload.

Calls only the CPU oracle (oracle/); nothing here touches the CUDA library.
Output: batched_midgame_k12.txt, one line per sampled board:
    <board index> <packed board hex> <8 super-value words hex>
for every 16th of the 1024 seeded 12-empty boards (64 boards, about 30 s of
oracle time each).  Run:  python tests/golden/make_golden.py [--threads N]
"""
import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1404_0743_gb300 import inputs  # noqa: E402

STRIDE = 16
OUT = os.path.join(HERE, "batched_midgame_k12.txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    boards = inputs.batched_midgame_boards(1024)
    idx = list(range(0, 1024, STRIDE))
    vals = oracle.midgame_many([boards[i] for i in idx], threads=args.threads)
    with open(OUT, "w") as f:
        f.write("# batched midgame workload (seed 0x14040743 + 1000 + i, 12 empty cells):\n")
        f.write("# board index, packed board, oracle super value (win[4], notlose[4])\n")
        for i, v in zip(idx, vals):
            words = " ".join(f"{int(w):016x}" for w in v)
            f.write(f"{i} {int(boards[i]):016x} {words}\n")
    print(f"wrote {len(idx)} boards to {OUT}")


if __name__ == "__main__":
    main()
