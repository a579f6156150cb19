"""Small, self-contained cases for profiling one kernel at a time.

    python -m paper_1404_0743_gb300.profile_cases --case midgame [--boards 64] [--empty 12]
    python -m paper_1404_0743_gb300.profile_cases --case slice36 [--stage 2] [--d4]
    python -m paper_1404_0743_gb300.profile_cases --case slice35 [--max-boards 20000000]
        [--stage 2] [--d4]
    python -m paper_1404_0743_gb300.profile_cases --case section34 [--sparse]

midgame: one plan run over seeded boards (fill tables 3^empty x 64 B per
board), repeated --repeat times.
slice36: the whole slice 36 (4.8e7 boards, 3.1 GB; --d4: 0.6 GB), by lines
or with --stage 2 one thread per board, repeated --repeat times.
slice35: slice 36 in full (3.1 GB; with --d4 the D4-reduced slice 36, 0.6
GB), then the smallest (or --pick largest) slice-35 sections whose boards add
up to at most --max-boards, back to back; --stage 2 runs them one thread per
board (the section kernel) instead of by lines.
section34: the largest slice-34 section with two 8-stone quadrants (29.6M
boards, by lines), built alone from its two child sections of slice 35 and
their slice-36 children, each through pp_section_compute (about 3 GB); with
--sparse the section is then computed again through pp_slice_step_sparse
from its two child sections (which prepares them first).
Each case prints its wall time per repeat (not a benchmark number).
"""
import argparse
import time

import numpy as np


def main():
    import torch

    import paper_1404_0743_gb300 as pp
    from paper_1404_0743_gb300 import build, inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["midgame", "slice36", "slice35", "slice34", "section34"], required=True)
    ap.add_argument("--boards", type=int, default=64)
    ap.add_argument("--empty", type=int, default=12)
    ap.add_argument("--max-boards", type=int, default=20_000_000)
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--mode", type=int, default=2,
                    help="midgame plan mode: 1 persistent, 2 one launch per level, 3 CUDA graph")
    ap.add_argument("--pick", choices=["smallest", "largest"], default="smallest",
                    help="which sections fill the --max-boards budget")
    ap.add_argument("--stage", type=int, default=0, help="slice35: 1 by lines (default), 2 one thread per board")
    ap.add_argument("--d4", action="store_true", help="slice35: the D4-reduced layouts")
    ap.add_argument("--sparse", action="store_true",
                    help="section34: through pp_slice_step_sparse (children prepared by the step)")
    args = ap.parse_args()
    build.build()
    pp.init()
    dev = torch.device("cuda:0")
    if args.case == "section34":
        # the largest slice-34 section with two 8-stone quadrants, built alone
        # from its own children (each through pp_section_compute)
        def key(s):
            return tuple(tuple(int(v) for v in row) for row in s["bw"])

        def size(s):
            return int(np.prod(s["dim"].astype(np.int64)))

        tables = {n: {key(s): s for s in pp.slice_sections(n)[0]} for n in (34, 35, 36)}
        cands = [s for s in tables[34].values() if sorted(int(x[0]) + int(x[1]) for x in s["bw"]) == [8, 8, 9, 9]]
        top = max(cands, key=size)
        made = {}

        def build_section(n, k):
            if (n, k) in made:
                return made[(n, k)]
            desc = tables[n][k]
            mover = 0 if n % 2 == 0 else 1
            kids = []
            for q in range(4):
                bw = [list(x) for x in k]
                if n == 36 or bw[q][0] + bw[q][1] == 9:
                    kids.append(None)
                    continue
                bw[q][mover] += 1
                kids.append(build_section(n + 1, tuple(tuple(x) for x in bw)))
            out = torch.empty((size(desc), 8), dtype=torch.int64, device=dev)
            pp.section_compute(n, desc, kids, out)
            made[(n, k)] = out
            return out

        for n_kid in (35,):
            for q in range(4):
                bw = [list(x) for x in key(top)]
                if bw[q][0] + bw[q][1] < 9:
                    bw[q][0] += 1
                    build_section(n_kid, tuple(tuple(x) for x in bw))
        torch.cuda.synchronize()
        if args.sparse:
            # the same section through pp_slice_step_sparse: its two child
            # sections back to back as the sparse input (prepared by the step,
            # since the section outnumbers its children)
            secs35, _ = pp.slice_sections(35)
            kids = [i for i, s in enumerate(secs35) if (35, key(s)) in made]
            cat = torch.cat([made[(35, key(secs35[i]))] for i in kids])
            offs = np.full(len(secs35), pp.PP_ABSENT, dtype=np.uint64)
            at = 0
            for i in kids:
                offs[i] = at
                at += size(secs35[i])
            secs34, _ = pp.slice_sections(34)
            f = np.array([key(s) == key(top) for s in secs34], dtype=np.uint8)
            out = torch.empty((size(top), 8), dtype=torch.int64, device=dev)
            for _ in range(args.repeat):
                t = time.perf_counter()
                pp.slice_step_sparse(34, cat, offs, out, filter=f)
                torch.cuda.synchronize()
                print(f"section {key(top)} (sparse step): {size(top)} boards: {1e3 * (time.perf_counter() - t):.2f} ms")
            return
        for _ in range(args.repeat):
            t = time.perf_counter()
            made.pop((34, key(top)), None)
            build_section(34, key(top))
            torch.cuda.synchronize()
            print(f"section {key(top)}: {size(top)} boards: {1e3 * (time.perf_counter() - t):.2f} ms")
        return
    if args.case == "slice36":
        _, total36 = pp.slice_sections(36, d4=args.d4)
        v36 = torch.zeros((total36, 8), dtype=torch.int64, device=dev)
        for _ in range(args.repeat):
            t = time.perf_counter()
            pp.slice_step(36, None, v36, opts=(0, 0, 0, args.stage) if args.stage else None, d4=args.d4)
            torch.cuda.synchronize()
            print(f"slice 36: {total36} boards: {1e3 * (time.perf_counter() - t):.2f} ms")
        return
    if args.case == "midgame":
        boards = inputs.midgame_boards(args.boards, args.empty, inputs.SEED_BATCHED)
        plan = pp.MidgamePlan(boards, args.empty)
        plan.configure(args.mode)
        ws = torch.empty(pp.midgame_workspace_bytes(args.boards, args.empty), dtype=torch.uint8, device=dev)
        out = torch.zeros((args.boards, 8), dtype=torch.int64, device=dev)
        for _ in range(args.repeat):
            t = time.perf_counter()
            plan.run(ws, out)
            torch.cuda.synchronize()
            print(f"midgame {args.boards} x {args.empty}: {1e3 * (time.perf_counter() - t):.2f} ms")
    else:
        n = 35 if args.case == "slice35" else 34
        d4 = args.d4 and n == 35
        secs36, total36 = pp.slice_sections(36, d4=d4)
        v36 = torch.zeros((total36, 8), dtype=torch.int64, device=dev)
        pp.slice_step(36, None, v36, d4=d4)
        src = v36
        if n == 34:
            secs35, total35 = pp.slice_sections(35)
            src = torch.zeros((total35, 8), dtype=torch.int64, device=dev)
            pp.slice_step(35, v36, src)
        secs, _ = pp.slice_sections(n, d4=d4)
        sizes = np.array([int(np.prod(s["dim"].astype(np.int64))) for s in secs])
        order = np.argsort(sizes) if args.pick == "smallest" else np.argsort(-sizes)
        keep = np.zeros(len(secs), dtype=np.uint8)
        acc = 0
        for i in order:
            if acc + sizes[i] > args.max_boards:
                continue
            keep[i] = 1
            acc += sizes[i]
        out = torch.zeros((acc, 8), dtype=torch.int64, device=dev)
        for _ in range(args.repeat):
            t = time.perf_counter()
            pp.slice_step(n, src, out, filter=keep, opts=(0, 0, 0, args.stage) if args.stage else None, d4=d4)
            torch.cuda.synchronize()
            print(f"slice {n}: {int(keep.sum())} sections, {acc} boards: {1e3 * (time.perf_counter() - t):.2f} ms")


if __name__ == "__main__":
    main()
