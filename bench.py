"""Benchmark of the pentago retrograde hot path on GB300.

Default workload: the batched midgame solve, 1024 seeded boards with 24
stones (12 empty cells, black to move), every board's compact fill table
(143,365 super values) in HBM, all levels of all boards in one plan run.  A "step" is one
full run.  The metric counts every 256-rotation super value computed (all
143,365 valid fills of each board, 146,805,760 per step).

The JSON line also carries the full terminal retrograde step over sections
(slice 36 from five-in-a-row, then slice 35 from slice 36: 8.59e8 super
values, 55 GB written) as "slice_step", with its own HBM roofline, the
slice-34 stream ("slice34_batched"), the D4-reduced chain 36 -> 35 -> 34
with the D4 slice-33 stream, the out-of-core slice 33 -> 32 stream and the
largest slice-32 section's cone ("d4_chain"), the midgame on one parity
class ("midgame_half") and the serving run ("serving").

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own 1024 boards (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
import weakref

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BOARDS = 1024
EMPTY = 12
FILLS_PER_BOARD = 143365  # sum over m of C(12, m) C(m, ceil(m/2))
METRIC = "boards/s (256-rotation super values)"
# DRAM bytes (read + write) of one step of the 1024 x 12 workload, from one
# single-pass ncu capture of the current kernels (dram__bytes_read.sum +
# dram__bytes_write.sum): the persistent launch, and the 13 level launches of
# the graph and per-level modes (None where a kernel has changed since)
PERSISTENT_TRAFFIC_BYTES = 11.39e9 + 9.39e9
LEVEL_TRAFFIC_BYTES = 10.30e9 + 9.06e9
TRAFFIC_SOURCE = "profiles/midgame_persistent_kernel_1024x12_traffic.md"
# what bounds the midgame kernels instead of DRAM bandwidth (ncu --set full):
# the persistent launch on 128 boards x 12 empty cells, and one level-8
# launch of the level kernel on 32 boards
BINDING_LIMIT = {
    "persistent": {"source": "profiles/midgame_persistent_kernel_128x12.md", "l1tex_throughput_pct": 71.0,
                   "l1tex_data_pipe_pct": 70.7, "alu_pipe_pct": 49.4, "issue_active_pct": 36.2,
                   "warps_active_pct": 49.8,
                   "reading": "the L1 data pipe and the latency of scattered 64-byte child loads "
                              "(long-scoreboard stalls, 12.7 per issue; grid barriers 3.1)"},
    "level": {"source": "profiles/midgame_level_kernel_32x12.md", "l1tex_throughput_pct": 78.1,
              "l1tex_data_pipe_pct": 70.4, "alu_pipe_pct": 53.5, "issue_active_pct": 43.0,
              "warps_active_pct": 67.3,
              "reading": "latency of scattered 64-byte child loads (long-scoreboard stalls, 15.7 per issue) "
                         "and the L1 data pipe"}}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = []
        try:
            with open(self.path) as f:
                lines = f.readlines()
            os.unlink(self.path)
        except Exception:
            pass
        return parse_clocks(lines)


def parse_clocks(lines):
    """Median SM clock, the highest max clock and the throttle reasons seen
    in nvidia-smi rows of ClockSampler.FIELDS (csv, no header, no units);
    rows that do not parse are skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for name, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """The slowest rank's time (timing only; no collective on the data path)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_boards(rank):
    """Each rank's own 1024 boards: rank 0 solves the standard workload, rank r
    the next disjoint block of seeds (weak scaling, independent problems)."""
    from paper_1404_0743_gb300 import inputs
    if rank == 0:
        return inputs.batched_midgame_boards(BOARDS)
    return inputs.midgame_boards(BOARDS, EMPTY, inputs.SEED_BATCHED + rank * BOARDS)


def whole_job_rate(units_per_rank, world, slowest_s):
    return world * units_per_rank / slowest_s


def cpu_baseline(threads=None, boards=None):
    """The oracle as it stands on the host cores: one 12-empty board of the
    workload per core, in parallel.  Returns (boards/s, cores, sample)."""
    import oracle
    from paper_1404_0743_gb300 import inputs
    cores = threads or os.cpu_count() or 1
    sample = boards if boards is not None else inputs.batched_midgame_boards(cores)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.midgame_many(sample, threads=cores)
    dt = time.perf_counter() - t0
    return len(sample) * FILLS_PER_BOARD / dt, cores, (
        f"{len(sample)} of the workload's 12-empty boards (all {FILLS_PER_BOARD} fills each), "
        f"one per host thread, {dt:.1f} s wall")


class PreparedPlan:
    """A slice plan below slice 35 whose input is first turned into ready
    records (pp_prepare_children_ready: one pass over the input) at every
    run, so the timed work includes that pass; its boards then skip their
    rmax and their lines with one more stone."""

    def __init__(self, pp, n, src, out, **kw):
        import torch
        self.pp, self.src, self.n = pp, src, n
        self.d4, self.offs = kw.get("d4", False), kw.get("in_offsets")
        self.prep = torch.empty_like(src)
        self.plan = pp.SlicePlan(n, self.prep, out, **kw)
        self.plan.set_prepared(2)

    def _ready(self, stream):
        self.pp.prepare_children_ready(self.n, self.src, self.prep, d4=self.d4, in_offsets=self.offs, stream=stream)

    def run(self, stream=None):
        self._ready(stream)
        self.plan.run(stream=stream)

    def autotune(self, stream=None):
        self._ready(stream)
        return self.plan.autotune(stream=stream)

    def close(self):
        self.plan.close()
        self.prep = None


def slice34_run(pp, dev, v35, batch_gb):
    """Config 4: all slice-34 sections whose quadrants hold 8 or 9 stones
    (3420 sections, 5.25e9 boards, 336 GB of output), streamed through one
    device buffer in batches, each batch one plan (many sections, one launch)
    followed by a digest of its output; the whole stream is captured in one
    CUDA graph.  Against it: one launch per section (pp_section_compute) on
    the first batch."""
    import torch
    secs, _ = pp.slice_sections(34)
    sizes = np.array([int(np.prod(s["dim"].astype(np.int64))) for s in secs])
    counts = np.array([[int(x[0]) + int(x[1]) for x in s["bw"]] for s in secs])
    eligible = np.nonzero((counts >= 8).all(axis=1))[0]
    cap = int(batch_gb * (1 << 30) // 64)
    batches, cur, acc = [], [], 0
    for i in eligible:
        if acc + sizes[i] > cap and cur:
            batches.append(cur)
            cur, acc = [], 0
        cur.append(int(i))
        acc += int(sizes[i])
    if cur:
        batches.append(cur)
    out = torch.empty((max(int(sizes[b].sum()) for b in batches), 8), dtype=torch.int64, device=dev)
    dig = torch.zeros(4, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream()
    # slice 35 as ready records, once per pass over the stream (51.9 GB)
    prep = torch.empty_like(v35)
    plans = []
    for bt in batches:
        f = np.zeros(len(secs), dtype=np.uint8)
        f[bt] = 1
        plans.append(pp.SlicePlan(34, prep, out, filter=f))
        plans[-1].set_prepared(2)
    pp.prepare_children_ready(34, v35, prep, stream=stream)
    chosen = plans[0].autotune(stream=stream)
    for p in plans[1:]:
        p.configure(chosen)
    torch.cuda.synchronize()

    def stream_once():
        pp.prepare_children_ready(34, v35, prep, stream=stream)
        for p, bt in zip(plans, batches):
            p.run(stream=stream)
            pp.super_digest(out, dig, n=int(sizes[bt].sum()), stream=stream)

    with torch.cuda.stream(stream):
        stream_once()  # warm
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        stream_once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dig.zero_()
    torch.cuda.synchronize()
    e0.record()  # replay() launches the graph on the current stream
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    digest = [int(x) for x in dig.cpu().numpy().view(np.uint64)]
    total = int(sizes[eligible].sum())
    # one launch per section on the first batch
    b0 = batches[0]
    kids = {tuple(tuple(int(v) for v in row) for row in s["bw"]): s for s in pp.slice_sections(35)[0]}
    args = []
    for i in b0:
        s = secs[i]
        ch = []
        for q in range(4):
            bw = [[int(v) for v in row] for row in s["bw"]]
            if bw[q][0] + bw[q][1] == 9:
                ch.append(None)
                continue
            bw[q][0] += 1  # slice 34: black moves
            c = kids[tuple(tuple(x) for x in bw)]
            sz = int(np.prod(c["dim"].astype(np.int64)))
            ch.append(v35[int(c["offset"]):int(c["offset"]) + sz])
        args.append((s, ch))
    off = 0
    e0.record()
    for (s, ch), i in zip(args, b0):
        pp.section_compute(34, s, ch, out[off:off + int(sizes[i])])
        off += int(sizes[i])
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    b0_boards = int(sizes[b0].sum())
    for p in plans:
        p.close()
    del out, prep
    return {
        "workload": "slice 34 from slice 35: the 3420 sections with 8 or 9 stones in every quadrant, "
                    f"streamed in {len(batches)} batches of <= {batch_gb} GB through one buffer, "
                    "each batch one plan launch + a digest, whole stream one CUDA graph; slice 35 "
                    "turned into ready records first (one pass, inside the timed graph)",
        "sections": int(len(eligible)), "boards": total, "output_gb": total * 64 / 1e9,
        "ms": ms, "boards_per_s": total / (ms / 1e3), "chosen_opts": list(chosen),
        "digest": {"win_bits": digest[0], "notlose_bits": digest[1], "hash": hex(digest[2]), "values": digest[3]},
        "per_section_launches": {"sections": len(b0), "boards": b0_boards, "ms": ms_plain,
                                 "boards_per_s": b0_boards / (ms_plain / 1e3)},
    }


def midgame_half_run(pp, plan, ws, out, steps, warmup, stream, hbm_peak, peak_kind):
    """The batched midgame workload on parity class 0 only (the rotations g
    with g0+g1+g2+g3 even, which hold the positions as given): 32-byte half
    fill tables (paper, "Open source and data").  Same plan, autotuned
    again; the values produced are 128-rotation halves of super values."""
    import torch
    plan.set_parity(0)
    mode, ctas = plan.autotune(ws, out)
    for _ in range(warmup):
        plan.run(ws, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.run(ws, out)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.status()
    ms = e0.elapsed_time(e1) / steps
    plan.set_parity(-1)
    per_step = BOARDS * FILLS_PER_BOARD
    alg = BOARDS * (FILLS_PER_BOARD + 596652) * 32  # 32 B per fill stored, 32 B per move loaded
    return {
        "workload": "the batched midgame workload (1024 boards x 12 empty) on parity class 0 of the rotations, "
                    "half fill tables (32 B per position)",
        "ms_per_step": ms, "value": per_step / (ms / 1e3), "unit": "boards/s (128-rotation half super values)",
        "execution": {1: "one persistent cooperative launch", 2: "one launch per level",
                      3: "CUDA graph of level launches"}[mode] + (f", {ctas} CTA/SM" if ctas else ""),
        "workspace_gb": pp.midgame_parity_workspace_bytes(BOARDS, EMPTY) / 1e9,
        "roofline": {"bound": "hbm", "kernel": "midgame_persistent_kernel<half>" if mode == 1 else
                     "midgame_level_kernel<half>", "achieved": alg / (ms / 1e3) / 1e9, "peak": hbm_peak,
                     "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / hbm_peak, "peak_kind": peak_kind,
                     "traffic": None, "alg_bytes_per_step": alg},
    }


def d4_slice33_stream(pp, dev, v34, batch_gb):
    """D4-reduced slice 33 (1343 sections, 5.28e9 boards, 338 GB: more than
    the device holds) from the resident D4 slice 34, streamed through one
    buffer in section batches of at most batch_gb, each batch one plan launch
    and a digest; the whole stream is one CUDA graph, timed once."""
    import torch
    secs, total = pp.slice_sections(33, d4=True)
    sizes = np.array([int(np.prod(s["dim"].astype(np.int64))) for s in secs])
    cap = int(batch_gb * (1 << 30) // 64)
    batches, cur, acc = [], [], 0
    for i in range(len(secs)):
        if acc + sizes[i] > cap and cur:
            batches.append(cur)
            cur, acc = [], 0
        cur.append(i)
        acc += int(sizes[i])
    if cur:
        batches.append(cur)
    out = torch.empty((max(int(sizes[b].sum()) for b in batches), 8), dtype=torch.int64, device=dev)
    dig = torch.zeros(4, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream()
    # D4 slice 34 as ready records, once per pass over the stream (63 GB)
    prep = torch.empty_like(v34)
    plans = []
    for bt in batches:
        f = np.zeros(len(secs), dtype=np.uint8)
        f[bt] = 1
        plans.append(pp.SlicePlan(33, prep, out, filter=f, d4=True))
        plans[-1].set_prepared(2)
    pp.prepare_children_ready(33, v34, prep, d4=True, stream=stream)
    chosen = plans[0].autotune(stream=stream)
    for p in plans[1:]:
        p.configure(chosen)
    torch.cuda.synchronize()

    def stream_once():
        pp.prepare_children_ready(33, v34, prep, d4=True, stream=stream)
        for p, bt in zip(plans, batches):
            p.run(stream=stream)
            pp.super_digest(out, dig, n=int(sizes[bt].sum()), stream=stream)

    with torch.cuda.stream(stream):
        stream_once()  # warm
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        stream_once()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dig.zero_()
    torch.cuda.synchronize()
    e0.record()  # replay() launches the graph on the current stream
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    digest = [int(x) for x in dig.cpu().numpy().view(np.uint64)]
    for p in plans:
        p.close()
    del out, g
    return {
        "workload": f"D4 slice 33 from D4 slice 34: 1343 sections streamed in {len(batches)} batches of "
                    f"<= {batch_gb} GB through one buffer, each batch one plan launch + a digest, one CUDA graph",
        "sections": len(secs), "boards": total, "output_gb": total * 64 / 1e9, "ms": ms,
        "boards_per_s": total / (ms / 1e3), "chosen_opts": list(chosen),
        "digest": {"win_bits": digest[0], "notlose_bits": digest[1], "hash": hex(digest[2]), "values": digest[3]},
    }


def d4_slice32_stream(pp, dev, v34, host_gb, batch_gb):
    """The chain below slice 34 out of core (paper, "Data layout and
    distribution": slice n reads only slice n+1): D4 slice 33 (338 GB, more
    than the device holds) is made in batches from the resident D4 slice 34
    and kept, as ready records, in device memory as far as it fits and in
    pinned host memory after that (up to host_gb); then D4 slice 32 (1.43 TB)
    is made in batches of sections from the slice-33 sections they read:
    those in host memory are copied in on a second stream while the batch
    before computes (pp_stager), and each output batch is digested and copied
    out to a pinned host buffer on a third stream.  Slice-32 sections whose
    slice-33 input was kept nowhere are skipped and counted.  v34 is
    overwritten with its ready records."""
    import torch
    secs33, total33 = pp.slice_sections(33, d4=True)
    secs32, total32 = pp.slice_sections(32, d4=True)
    size33 = np.prod(secs33["dim"].astype(np.int64), axis=1)
    size32 = np.prod(secs32["dim"].astype(np.int64), axis=1)
    # batch buffers, staging halves and the host buffers are powers of two
    # (the pinned host allocator rounds sizes up to one)
    cap = 1 << int(np.log2(batch_gb * (1 << 30) / 64))
    pp.prepare_children_ready(33, v34, v34, d4=True)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    # phase 1 holds v34, the kept slice-33 sections, the staging room (2 cap)
    # and a batch buffer (cap); phase 2 frees v34 and the buffer for two
    # output buffers (2 cap)
    dev_values = max(0, (free - 3 * cap * 64 - (12 << 30)) // 64)
    host_values = 1 << int(np.log2(host_gb * (1 << 30) / 64)) if host_gb >= 1 else 0
    # ---- phase 1: slice 33 in batches, each kept on the device or on the host
    order = list(range(len(secs33)))
    dev_off = np.full(len(secs33), pp.PP_ABSENT, dtype=np.uint64)
    where, d_used, h_used = {}, 0, 0
    for i in order:
        if d_used + size33[i] <= dev_values:
            where[i] = ("dev", d_used)
            d_used += int(size33[i])
        elif h_used + size33[i] <= host_values:
            where[i] = ("host", h_used)
            h_used += int(size33[i])
    stage_values = 2 * cap
    base = torch.empty((d_used + stage_values, 8), dtype=torch.int64, device=dev)
    hstore = torch.empty((host_values, 8), dtype=torch.int64, pin_memory=True) if h_used else None
    buf = torch.empty((cap, 8), dtype=torch.int64, device=dev)
    dig33 = torch.zeros(4, dtype=torch.int64, device=dev)
    stream, copy, out_s = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    batches, cur, acc = [], [], 0
    for i in order:
        if i not in where:
            continue
        kind = where[i][0]
        if cur and (acc + size33[i] > cap or kind != where[cur[0]][0] or
                    (kind == "dev" and where[i][1] != where[cur[-1]][1] + size33[cur[-1]])):
            batches.append(cur)
            cur, acc = [], 0
        cur.append(i)
        acc += int(size33[i])
    if cur:
        batches.append(cur)
    plans = []
    for bt in batches:
        f = np.zeros(len(secs33), dtype=np.uint8)
        f[bt] = 1
        kind, at = where[bt[0]]
        dst = base[at:] if kind == "dev" else buf
        plans.append((pp.SlicePlan(33, v34, dst, filter=f, d4=True), bt, kind, at, dst))
        plans[-1][0].set_prepared(2)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    torch.cuda.synchronize()
    e0.record(stream)
    d2h33 = 0
    for plan, bt, kind, at, dst in plans:
        n = int(size33[bt].sum())
        plan.run(stream=stream)
        pp.super_digest(dst, dig33, n=n, stream=stream)
        # the batch's sections sit back to back in section order
        offs = np.full(len(secs33), pp.PP_ABSENT, dtype=np.uint64)
        offs[sorted(bt)] = np.concatenate([[0], np.cumsum(size33[sorted(bt)])[:-1]]).astype(np.uint64)
        pp.prepare_children_ready(32, dst[:n], dst[:n], d4=True, in_offsets=offs, stream=stream)
        if kind == "host":
            with torch.cuda.stream(stream):
                hstore[at:at + n].copy_(buf[:n], non_blocking=True)
            d2h33 += n * 64
    for i, (kind, at) in where.items():
        if kind == "dev":
            dev_off[i] = at
    e1.record(stream)
    torch.cuda.synchronize()
    ms33 = e0.elapsed_time(e1)
    for pl in plans:
        pl[0].close()
    plan = dst = pl = None  # loop variables hold the last plan (and with it v34) and buffer
    gone = weakref.ref(v34)
    del buf, plans, v34
    torch.cuda.empty_cache()
    if gone() is not None:
        raise RuntimeError("slice 34 is still referenced; the out-of-core stream needs its memory")
    # ---- phase 2: slice 32 in batches through the stager
    host = [hstore[where[i][1]:where[i][1] + int(size33[i])] if where.get(i, ("", 0))[0] == "host" else None
            for i in range(len(secs33))]
    st = pp.Stager(32, base, dev_off, host, d_used, stage_values, prepared=2, d4=True)
    kept = set(where)
    batches32, cur, acc, staged_need = [], [], 0, 0
    skipped = 0
    for i in range(len(secs32)):
        f1 = np.zeros(len(secs32), dtype=np.uint8)
        f1[i] = 1
        kids = np.flatnonzero(pp.slice_children(32, f1, d4=True))
        if not all(int(k) in kept for k in kids):
            skipped += 1
            continue
        hneed = sum(int(size33[k]) for k in kids if where[int(k)][0] == "host")
        if size32[i] > cap or hneed > cap:
            skipped += 1
            continue
        if cur and (acc + size32[i] > cap or staged_need + hneed > cap):
            batches32.append(cur)
            cur, acc, staged_need = [], 0, 0
        cur.append(i)
        acc += int(size32[i])
        staged_need += hneed  # an upper bound: sections shared by the batch's sections are counted each time
    if cur:
        batches32.append(cur)
    outs = [torch.empty((cap, 8), dtype=torch.int64, device=dev) for _ in range(2)]
    ring = torch.empty((cap, 8), dtype=torch.int64, pin_memory=True)
    dig32 = torch.zeros(4, dtype=torch.int64, device=dev)
    done_out = [torch.cuda.Event() for _ in range(2)]
    filters = []
    for bt in batches32:
        f = np.zeros(len(secs32), dtype=np.uint8)
        f[bt] = 1
        filters.append(f)
    torch.cuda.synchronize()
    staged = d2h32 = boards32 = 0
    e0.record(stream)
    for j, (bt, f) in enumerate(zip(batches32, filters)):
        o = outs[j % 2]
        n = int(size32[bt].sum())
        if j >= 2:
            stream.wait_event(done_out[j % 2])  # its previous contents are on their way out
        staged += st.step(o, filter=f, stream=stream, copy_stream=copy)
        pp.super_digest(o, dig32, n=n, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        out_s.wait_event(ev)
        with torch.cuda.stream(out_s):
            ring[:n].copy_(o[:n], non_blocking=True)
        done_out[j % 2].record(out_s)
        d2h32 += n * 64
        boards32 += n
    e1.record(stream)
    e2.record(out_s)
    torch.cuda.synchronize()
    ms32 = e0.elapsed_time(e1)
    ms32_out = max(ms32, e0.elapsed_time(e2))
    st.close()
    d33 = [int(x) for x in dig33.cpu().numpy().view(np.uint64)]
    d32 = [int(x) for x in dig32.cpu().numpy().view(np.uint64)]
    del base, hstore, outs, ring
    torch.cuda.empty_cache()
    return {
        "workload": "D4 slice 33 from the resident D4 slice 34, kept as ready records on the device "
                    f"({d_used * 64 / 1e9:.0f} GB) and in pinned host memory ({h_used * 64 / 1e9:.0f} GB); then "
                    f"D4 slice 32 in {len(batches32)} batches of <= {batch_gb} GB from the slice-33 sections they "
                    "read, host ones copied in on a second stream while the batch before computes, each output "
                    "batch digested and copied out to pinned host memory on a third stream",
        "slice33": {"sections_kept": len(kept), "sections": len(secs33), "boards_kept": int(d_used + h_used),
                    "ms": ms33, "d2h_gb": d2h33 / 1e9,
                    "digest": {"win_bits": d33[0], "notlose_bits": d33[1], "hash": hex(d33[2]), "values": d33[3]}},
        "slice32": {"sections": int(sum(len(b) for b in batches32)), "sections_total": len(secs32),
                    "sections_skipped": skipped, "boards": boards32, "boards_total": int(total32),
                    "ms": ms32_out, "boards_per_s": boards32 / (ms32_out / 1e3),
                    "h2d_gb": staged * 64 / 1e9, "h2d_gbs": staged * 64 / 1e9 / (ms32_out / 1e3),
                    "d2h_gb": d2h32 / 1e9, "d2h_gbs": d2h32 / 1e9 / (ms32_out / 1e3),
                    "digest": {"win_bits": d32[0], "notlose_bits": d32[1], "hash": hex(d32[2]), "values": d32[3]}},
    }


def d4_cone_run(pp, dev, steps, warmup):
    """Below slice 33 by dependency cone: the largest D4 slice-32 section
    (4.06e8 boards; slice 32 is 1.43 TB, more than the device holds) from the
    whole D4 slice 36 and, at slices 35, 34 and 33, only the sections the
    slice below reads.  Each level is one autotuned plan whose compact output
    is the sparse input of the next; one step runs the five levels."""
    import torch
    secs32, _ = pp.slice_sections(32, d4=True)
    sizes32 = np.prod(secs32["dim"].astype(np.int64), axis=1)
    target = int(np.argmax(sizes32))
    filters = {32: np.zeros(len(secs32), dtype=np.uint8)}
    filters[32][target] = 1
    for n in (32, 33, 34):
        filters[n + 1] = pp.slice_children(n, filters[n], d4=True)
    _, total36 = pp.slice_sections(36, d4=True)
    vals = {36: torch.empty((total36, 8), dtype=torch.int64, device=dev)}
    plans = {36: pp.SlicePlan(36, None, vals[36], d4=True)}
    plans[36].run()
    for n in (35, 34, 33, 32):
        _, count = pp.compact_offsets(n, filters[n], True)
        vals[n] = torch.empty((count, 8), dtype=torch.int64, device=dev)
        if n == 35:
            plans[n] = pp.SlicePlan(35, vals[36], vals[n], filter=filters[n], d4=True)
        else:
            offs, _ = pp.compact_offsets(n + 1, filters[n + 1], True)
            plans[n] = PreparedPlan(pp, n, vals[n + 1], vals[n], filter=filters[n], d4=True, in_offsets=offs)
        plans[n].run()
        plans[n].autotune()
    levels = (36, 35, 34, 33, 32)
    for _ in range(warmup):
        for n in levels:
            plans[n].run()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(levels) + 1)]
    ms = dict.fromkeys(levels, 0.0)
    for _ in range(steps):
        ev[0].record(stream)
        for j, n in enumerate(levels):
            plans[n].run()
            ev[j + 1].record(stream)
        torch.cuda.synchronize()
        for j, n in enumerate(levels):
            ms[n] += ev[j].elapsed_time(ev[j + 1]) / steps
    dig = torch.zeros(4, dtype=torch.int64, device=dev)
    pp.super_digest(vals[32], dig)
    digest = [int(x) for x in dig.cpu().numpy().view(np.uint64)]
    boards = {n: int(vals[n].shape[0]) for n in levels}
    for p in plans.values():
        p.close()
    del vals
    torch.cuda.empty_cache()
    total_ms = sum(ms.values())
    return {
        "workload": "the largest D4 slice-32 section (counts " + str(secs32[target]["bw"].tolist()) +
                    ") through its dependency cone: D4 slice 36 whole, then the sections of slices 35, 34 and 33 "
                    "that the slice below reads (" + ", ".join(str(int(filters[n].sum())) for n in (35, 34, 33)) +
                    " sections), each level's compact output the next level's sparse input",
        "boards": boards,
        "ms": {str(n): ms[n] for n in levels},
        "ms_per_step": total_ms,
        "slice32_boards_per_s": boards[32] / (ms[32] / 1000.0),
        "value": sum(boards.values()) / (total_ms / 1000.0), "unit": "boards/s (stored D4-reduced super values)",
        "digest": {"win_bits": digest[0], "notlose_bits": digest[1], "hash": hex(digest[2]), "values": digest[3]},
    }


def d4_chain_run(pp, dev, steps, warmup, hbm_peak, peak_kind, batch_gb, host_gb):
    """The D4-reduced retrograde chain: slices 36, 35 and 34 with only the
    sections whose counts are least under the board symmetries (0.6, 7.7 and
    63 GB), each slice read from the one above through the symmetries, one
    autotuned plan per slice.  Times each slice over `steps` runs, then
    streams slice 33 from the resident slice 34 (d4_slice33_stream)."""
    import torch
    stream = torch.cuda.current_stream()
    plans, vals, totals = {}, {}, {}
    prev = None
    for n in (36, 35, 34):
        _, total = pp.slice_sections(n, d4=True)
        v = torch.empty((total, 8), dtype=torch.int64, device=dev)
        plan = PreparedPlan(pp, n, prev, v, d4=True) if n < 35 else pp.SlicePlan(n, prev, v, d4=True)
        plan.run()
        plan.autotune()
        plans[n], vals[n], totals[n] = plan, v, total
        prev = v
    plan = v = prev = None  # only the dicts hold the slices (slice 34 is handed on below)
    for _ in range(warmup):
        for n in (36, 35, 34):
            plans[n].run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ms = {36: 0.0, 35: 0.0, 34: 0.0}
    for _ in range(steps):
        ev[0].record(stream)
        for j, n in enumerate((36, 35, 34)):
            plans[n].run()
            ev[j + 1].record(stream)
        torch.cuda.synchronize()
        for j, n in enumerate((36, 35, 34)):
            ms[n] += ev[j].elapsed_time(ev[j + 1]) / steps
    for p in plans.values():
        p.close()
    p = None
    plans.clear()  # the plans hold their input and output tensors
    del vals[36], vals[35]
    torch.cuda.empty_cache()
    s33 = d4_slice33_stream(pp, dev, vals[34], batch_gb) if batch_gb else None
    torch.cuda.empty_cache()
    # the out-of-core stream takes slice 34 over (it is made ready in place and freed)
    s32 = d4_slice32_stream(pp, dev, vals.pop(34), host_gb, batch_gb / 2) if batch_gb and host_gb else None
    full = {n: pp.slice_sections(n)[1] for n in (36, 35, 34)}
    # slice 34: one 64 B store per board plus one 64 B child read per move
    # (two moves per board)
    bytes34 = totals[34] * 64 * 3
    achieved = bytes34 / (ms[34] / 1000.0) / 1e9
    total_ms = ms[36] + ms[35] + ms[34]
    boards = totals[36] + totals[35] + totals[34]
    del vals
    return {
        "workload": "D4-reduced slices 36 -> 35 -> 34 (100, 330 and 750 sections; every board of each)",
        "boards_per_step": boards,
        "full_layout_boards_per_step": full[36] + full[35] + full[34],
        "ms_per_step": total_ms,
        "ms_slice36": ms[36], "ms_slice35": ms[35], "ms_slice34": ms[34],
        "value": boards / (total_ms / 1000.0), "unit": "boards/s (stored D4-reduced super values)",
        "roofline": {"bound": "hbm", "kernel": "section_line_kernel (D4 slice 34, ready children)", "achieved": achieved,
                     "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                     "traffic": None, "alg_bytes_per_launch": bytes34},
        "slice33_stream": s33,
        "slice32_stream": s32,
    }


def serving_run(pp, dev, n_queries):
    """Serving: a stream of midgame queries (8-16 empty cells) through the
    continuous-batching server, against the plain form (pp_midgame_solve per
    query, one at a time) on the same GPU.  Closed loop first (every query
    at once: each form's capacity), then Poisson arrivals at 0.5, 0.8 and
    1.0 x the server's capacity and at 0.8 x the plain form's capacity; at
    each load both forms face the same arrival times (the plain form as a
    host thread that solves each query when it has arrived and the one
    before is done).  Every result of every run is compared with the
    server's closed-loop result."""
    import torch
    from paper_1404_0743_gb300 import inputs
    boards, ks = inputs.serving_queries(n_queries)
    n = len(boards)
    fills = {k: sum(__import__("math").comb(k, m) * __import__("math").comb(m, (m + 1) // 2)
                    for m in range(k + 1)) for k in range(8, 17)}
    sub_boards = sum(fills[int(k)] for k in ks)
    arena = torch.empty(64 << 30, dtype=torch.uint8, device=dev)
    srv = pp.Server(arena, max_slots=256, max_empty=16)

    def drain(server, count, timeout=900):
        got = {}
        t = time.time()
        while len(got) < count and time.time() - t < timeout:
            server.wait(1, 1.0)
            for r in server.poll(4096):
                got[r["req_id"]] = r
        return got

    def pct(lat):
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}

    # server, closed loop: everything at once -> capacity
    t0 = time.perf_counter()
    for i, b in enumerate(boards):
        srv.submit(int(b), i)
    res = drain(srv, n)
    cap_s = time.perf_counter() - t0
    capacity = n / cap_s
    want = np.stack([res[i]["value"] for i in range(n)])

    # plain form: pp_midgame_solve per query on device-resident boards (one
    # per 16 bytes: the entry point takes 16-byte aligned board arrays)
    d_boards = torch.zeros((n, 2), dtype=torch.int64, device=dev)
    d_boards[:, 0] = torch.from_numpy(boards.view(np.int64)).to(dev)
    ws = torch.empty(pp.midgame_workspace_bytes(1, 16), dtype=torch.uint8, device=dev)
    one = torch.zeros((1, 8), dtype=torch.int64, device=dev)

    def plain_solve(i):
        pp.midgame_solve(d_boards[i, :1], one, int(ks[i]), ws)
        return one.cpu().numpy().view(np.uint64)[0]

    plain_solve(0)
    t0 = time.perf_counter()
    plain_mism = sum(int(not (plain_solve(i) == want[i]).all()) for i in range(n))
    plain_cap = n / (time.perf_counter() - t0)

    # the arrival loops run with Python's cyclic garbage collector paused: a
    # collection over the results kept so far stalls the submitting thread
    # for tens of milliseconds, which would show up as late arrivals
    def server_load(rate, base):
        arrivals = inputs.poisson_arrivals(n, rate)
        late = np.zeros(n)
        gc.collect()
        gc.disable()
        try:
            t0 = time.perf_counter()
            for i, (b, at) in enumerate(zip(boards, arrivals)):
                while time.perf_counter() - t0 < at:
                    pass
                late[i] = time.perf_counter() - t0 - at
                srv.submit(int(b), base + i)
        finally:
            gc.enable()
        got = drain(srv, n)
        wall = time.perf_counter() - t0
        lat = np.array([got[base + i]["done_s"] - got[base + i]["submit_s"] for i in range(n)]) * 1e3
        mism = sum(int(not (got[base + i]["value"] == want[i]).all()) for i in range(n))
        return arrivals, {"qps": n / wall, "boards_per_s": sub_boards / wall, **pct(lat), "mismatches": mism,
                          "max_submit_lateness_ms": float(late.max() * 1e3)}

    def plain_load(arrivals):
        lat, mism = np.zeros(n), 0
        gc.collect()
        gc.disable()
        try:
            t0 = time.perf_counter()
            for i, at in enumerate(arrivals):
                while time.perf_counter() - t0 < at:
                    pass
                v = plain_solve(i)
                lat[i] = (time.perf_counter() - t0 - at) * 1e3
                mism += int(not (v == want[i]).all())
            wall = time.perf_counter() - t0
        finally:
            gc.enable()
        return {"qps": n / wall, "boards_per_s": sub_boards / wall, **pct(lat), "mismatches": mism}

    loads = {}
    points = [("server", 0.5), ("server", 0.8), ("server", 1.0), ("plain", 0.8)]
    for j, (which, frac) in enumerate(points):
        rate = frac * (capacity if which == "server" else plain_cap)
        arrivals, sv = server_load(rate, (j + 1) * 1_000_000)
        loads[f"load_{frac}x_{which}_capacity"] = {"arrival_rate_qps": rate, "server": sv,
                                                   "plain": plain_load(arrivals)}
    stats = srv.stats()
    srv.close()
    # the same closed loop on parity class 0 (half tables: the positions as
    # given and their even rotations), in the same arena
    hsrv = pp.Server(arena, max_slots=256, max_empty=16, parity=0)
    t0 = time.perf_counter()
    for i, b in enumerate(boards):
        hsrv.submit(int(b), i)
    got_h = drain(hsrv, n)
    half_s = time.perf_counter() - t0
    half_stats = hsrv.stats()
    hsrv.close()
    mask0 = np.zeros(8, dtype=np.uint64)
    for beta in range(256):
        if not (beta ^ (beta >> 2) ^ (beta >> 4) ^ (beta >> 6)) & 1:
            mask0[beta >> 6] |= np.uint64(1) << np.uint64(beta & 63)
            mask0[4 + (beta >> 6)] |= np.uint64(1) << np.uint64(beta & 63)
    half_mism = sum(int(not (got_h[i]["value"] == (want[i] & mask0)).all()) for i in range(n))
    del arena, ws
    return {
        "workload": f"{n} seeded queries (seed 0x14040743+5000+i), k uniform in 8..16 empty cells, "
                    f"Poisson arrivals (separate seeded stream)",
        "queries": n,
        "closed_loop_qps": capacity, "closed_loop_boards_per_s": sub_boards / cap_s,
        "max_active": stats["max_active"],
        "closed_loop_parity0": {"qps": n / half_s, "boards_per_s": sub_boards / half_s,
                                "max_active": half_stats["max_active"], "mismatches_vs_full_on_class": half_mism},
        "plain_sequential": {"qps": plain_cap, "mismatches_vs_server": plain_mism},
        **loads,
    }


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1404_0743_gb300 import inputs
    import oracle
    cores = os.cpu_count() or 1
    warm = inputs.plain_midgame_boards(cores)
    for _ in range(args.warmup):
        oracle.midgame_many(warm, threads=cores)
    boards = inputs.batched_midgame_boards(BOARDS)
    times = []
    for s in range(args.steps):
        sample = [boards[(s * cores + j) % BOARDS] for j in range(cores)]
        t0 = time.perf_counter()
        oracle.midgame_many(sample, threads=cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * cores * FILLS_PER_BOARD / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "boards/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batched midgame solve: 1024 boards x 12 empty cells (one oracle board per host "
                               "thread per step)", "boards": BOARDS, "empty_cells": EMPTY},
        "cpu_baseline": {"value": value, "unit": "boards/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} boards of the workload per step, one per host thread"},
        "e2e": {"value": value, "unit": "boards/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    import paper_1404_0743_gb300 as pp
    from paper_1404_0743_gb300 import build, inputs

    build.build()
    torch.cuda.set_device(local)
    pp.init()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    hbm_peak, peak_kind = peaks()

    # ---- batched midgame -------------------------------------------------
    boards = rank_boards(rank)
    plan = pp.MidgamePlan(boards, EMPTY)
    ws = torch.empty(pp.midgame_workspace_bytes(BOARDS, EMPTY), dtype=torch.uint8, device=dev)
    out = torch.zeros((BOARDS, 8), dtype=torch.int64, device=dev)
    mode, ctas = plan.autotune(ws, out)  # untimed: picks per-level launches, graph or persistent
    for _ in range(args.warmup):
        plan.run(ws, out)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = pp.launch_count()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        plan.run(ws, out)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_total = start.elapsed_time(end)
    launches = pp.launch_count() - launches0
    clk = clocks.stop()
    plan.status()
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    per_step = BOARDS * FILLS_PER_BOARD
    value = whole_job_rate(per_step, world, ms_step / 1000.0)

    # Algorithmic bytes of a step, counted with level reuse: every fill's
    # 64 B value is stored once and read once by the level above (its
    # parents find it in L2 after the first read), so the DRAM minimum is
    # 2 x 64 B per fill.  That count is the roofline's; the gather count
    # (one 64 B child load per move, every one from DRAM) is reported beside
    # it as an effective rate.  A step is the five-table launch and the
    # level work (one persistent launch, or one launch per level).
    gathers_per_board = 596652
    alg_bytes = 2 * BOARDS * FILLS_PER_BOARD * 64
    gather_bytes = BOARDS * (FILLS_PER_BOARD + gathers_per_board) * 64
    launches_per_step = launches / args.steps
    achieved = alg_bytes / (ms_step / 1000.0) / 1e9
    kernel = "midgame_persistent_kernel" if mode == 1 else "midgame_level_kernel"
    traffic = PERSISTENT_TRAFFIC_BYTES if mode == 1 else LEVEL_TRAFFIC_BYTES

    # ---- end to end through the host-array entry point ------------------------
    hb = torch.from_numpy(boards.view(np.int64)).pin_memory()
    ho = torch.zeros((BOARDS, 8), dtype=torch.int64).pin_memory()
    pp.midgame_solve_host(hb, ho, EMPTY, ws)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pp.midgame_solve_host(hb, ho, EMPTY, ws)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
    e2e_value = whole_job_rate(per_step, world, e2e_s)

    # ---- the same workload on one parity class (half tables) ------------------
    half = midgame_half_run(pp, plan, ws, out, args.steps, args.warmup, stream, hbm_peak, peak_kind)
    del ws, out

    # ---- terminal retrograde step: slice 36 then slice 35 ----------------------
    secs36, total36 = pp.slice_sections(36)
    secs35, total35 = pp.slice_sections(35)
    v36 = torch.empty((total36, 8), dtype=torch.int64, device=dev)
    v35 = torch.empty((total35, 8), dtype=torch.int64, device=dev)
    for _ in range(max(1, args.warmup)):
        pp.slice_step(36, None, v36)
        pp.slice_step(35, v36, v35)
    torch.cuda.synchronize()
    e36 = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t36 = t35 = 0.0
    for _ in range(args.steps):
        e36[0].record(stream)
        pp.slice_step(36, None, v36)
        e36[1].record(stream)
        pp.slice_step(35, v36, v35)
        e36[2].record(stream)
        torch.cuda.synchronize()
        t36 += e36[0].elapsed_time(e36[1])
        t35 += e36[1].elapsed_time(e36[2])
    t36 /= args.steps
    t35 /= args.steps
    # slice 35 with slice 36 on demand (no slice-36 array): same values
    pp.slice_step(35, None, v35)
    e36[0].record(stream)
    for _ in range(args.steps):
        pp.slice_step(35, None, v35)
    e36[1].record(stream)
    torch.cuda.synchronize()
    t35_fly = e36[0].elapsed_time(e36[1]) / args.steps
    bytes35 = total35 * 64 + total36 * 64  # write slice 35 + read slice 36 once
    bytes36 = total36 * 64
    slice_step = {
        "workload": "slice 36 (670 sections) then slice 35 (2460 sections) of the full enumeration",
        "boards_per_step": total36 + total35,
        "ms_per_step": t36 + t35,
        "ms_slice36": t36, "ms_slice35": t35,
        "ms_slice35_with_slice36_on_demand": t35_fly,
        "value": (total36 + total35) / ((t36 + t35) / 1000.0), "unit": "boards/s",
        "roofline": {"bound": "hbm", "kernel": "line35_kernel (slice 35)",
                     "achieved": bytes35 / (t35 / 1000.0) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": bytes35 / (t35 / 1000.0) / 1e9 / hbm_peak, "peak_kind": peak_kind,
                     "traffic": None, "alg_bytes_per_launch": bytes35},
        "roofline_slice36": {"bound": "hbm", "kernel": "line36_kernel (slice 36: stores only)",
                             "achieved": bytes36 / (t36 / 1000.0) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": bytes36 / (t36 / 1000.0) / 1e9 / hbm_peak, "peak_kind": peak_kind,
                             "alg_bytes_per_launch": bytes36},
        # the pair: slice 36 written, read back once, slice 35 written
        "roofline_step": {"bound": "hbm", "achieved": (bytes35 + bytes36) / ((t36 + t35) / 1000.0) / 1e9,
                          "peak": hbm_peak, "unit": "GB/s",
                          "frac": (bytes35 + bytes36) / ((t36 + t35) / 1000.0) / 1e9 / hbm_peak,
                          "peak_kind": peak_kind, "alg_bytes": bytes35 + bytes36},
    }
    del v36
    torch.cuda.empty_cache()
    slice34 = slice34_run(pp, dev, v35, args.slice34_batch_gb) if args.slice34_batch_gb else None
    del v35
    torch.cuda.empty_cache()
    d4 = d4_chain_run(pp, dev, args.steps, args.warmup, hbm_peak, peak_kind,
                      args.slice34_batch_gb, args.host_gb) if args.d4 else None
    torch.cuda.empty_cache()
    if d4 is not None:
        d4["slice32_cone"] = d4_cone_run(pp, dev, args.steps, args.warmup)
        torch.cuda.empty_cache()
    serving = serving_run(pp, dev, args.serve_queries) if args.serve_queries else None

    if rank != 0:
        return
    cpu_v, cores, sample = cpu_baseline()
    line = {
        "metric": METRIC, "value": value, "unit": "boards/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batched midgame solve: 1024 boards x 12 empty cells (seed 0x14040743+1000+i), "
                               "compact fill tables (143,365 x 64 B per board) in HBM, one plan run per step",
                   "boards": BOARDS, "empty_cells": EMPTY, "super_values_per_step": per_step,
                   "l2": "working set 9.7 GB of compact fill and five tables, far larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{world}",
                   "execution": {1: "one persistent cooperative launch", 2: "one launch per level",
                                 3: "CUDA graph of level launches"}[mode] + (f", {ctas} CTA/SM" if ctas else ""),
                   "autotuned": True},
        "roofline": {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": traffic,
                     "alg_bytes_per_step": alg_bytes,
                     "alg_bytes_rule": "64 B stored + 64 B read once per fill (143,365 fills per board)",
                     "launches_per_step": launches_per_step,
                     "traffic_source": TRAFFIC_SOURCE,
                     "traffic_achieved": traffic / (ms_step / 1000.0) / 1e9 if traffic else None,
                     "traffic_frac": traffic / (ms_step / 1000.0) / 1e9 / hbm_peak if traffic else None,
                     "gather_bytes_per_step": gather_bytes,
                     "gather_rate_gbs": gather_bytes / (ms_step / 1000.0) / 1e9,
                     "binding_limit": BINDING_LIMIT["persistent" if mode == 1 else "level"]},
        "cpu_baseline": {"value": cpu_v, "unit": "boards/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": e2e_value, "unit": "boards/s", "h2d_bytes_per_step": BOARDS * 8,
                "d2h_bytes_per_step": BOARDS * 64},
        "gpu_launches": launches,
        "clocks": clk,
        "midgame_half": half,
        "slice_step": slice_step,
        "slice34_batched": slice34,
        "d4_chain": d4,
        "serving": serving,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--serve-queries", type=int, default=10000, help="serving stream length (0 = skip)")
    ap.add_argument("--slice34-batch-gb", type=float, default=40.0,
                    help="batch size of the slice-34 and D4 slice-33 streams (0 = skip both)")
    ap.add_argument("--d4", type=int, default=1, help="D4-reduced chain 36 -> 35 -> 34 (0 = skip)")
    ap.add_argument("--host-gb", type=float, default=64.0,
                    help="pinned host memory for the out-of-core D4 slice 33 -> 32 stream (0 = skip it)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
