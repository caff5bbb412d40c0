"""Benchmark of the shuffle + merge hot path on GB300.

Workload: the plain shuffle + merge that emulates 8 workers of the paper's
cuDF merge benchmark (Sec. V-B, Fig. 8: chunk size 1E8, shuffle, fraction
match 0.3): P = 8 hash partitions, 100M left rows (int64 key = seeded
permutation, float64 payload U[0,1)) and 100M right rows (30% of keys drawn
from the left keys), synthetic data.  One step = one mdj_merge call: partition
both tables, join every partition pair, read the output count back, write the
joined rows.  Inputs (3.2 GB) are far larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mdj|reference]

Prints one JSON line.  With N > 1 (launched by torchrun) every rank runs an
independent replica on its own GPU (the path has no exchange between GPUs);
value = all rows merged by all ranks / max-over-ranks time.
The reference arm (--impl reference) times the CPU oracle (shuffle by a stable
counting sort, then a sort-merge join per partition pair) on a bounded sample
of the same workload, on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2101_08878_gb300 import datagen  # noqa: E402

METRIC = "merge input rows/s & HBM-roofline %, batched vs plain; p50/p99 join latency"
UNIT = "rows/s"
N_LEFT = N_RIGHT = 100_000_000
P = 8
FRAC = 0.3
SEED = 1
WORKLOAD = "plain shuffle+merge, P=8 hash partitions, 100M x 100M rows, int64 key + float64 payload, match 0.3"

# algorithmic bytes per row of each kernel (8-byte keys and payloads, 4-byte row ids)
KEY, PAY, RID, OUT_ROW = 8, 8, 4, 32


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.close()

    def summary(self):
        try:
            lines = [ln.strip() for ln in open(self.file.name) if ln.strip()]
            os.unlink(self.file.name)
        except OSError:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------ CPU baseline

def oracle_step(left, right, p, threads: int = 1):
    """The CPU oracle as it stands: stable hash partition of both tables (the
    shuffle), then a sort-merge inner join of every partition pair.  With
    threads > 1 the two partitions and the P partition-pair merges run on a
    thread pool (the oracle's C calls release the GIL); the work is the same."""
    import oracle

    def merge_part(q, loff, lparts, roff, rparts):
        ls = [c[loff[q]:loff[q + 1]] for c in lparts]
        rs = [c[roff[q]:roff[q + 1]] for c in rparts]
        return oracle.merge_table(ls, rs)["key"].size

    if threads <= 1:
        loff, _, lparts = oracle.partition_table(left, 0, p)
        roff, _, rparts = oracle.partition_table(right, 0, p)
        return sum(merge_part(q, loff, lparts, roff, rparts) for q in range(p))
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads) as ex:
        fl = ex.submit(oracle.partition_table, left, 0, p)
        fr = ex.submit(oracle.partition_table, right, 0, p)
        (loff, _, lparts), (roff, _, rparts) = fl.result(), fr.result()
        futs = [ex.submit(merge_part, q, loff, lparts, roff, rparts) for q in range(p)]
        return sum(f.result() for f in futs)


def cpu_baseline(n_sample: int, reps: int = 1):
    """The oracle on this host: single-threaded (the headline CPU number) and
    on a thread pool over all cores (at most 2 + P threads do work)."""
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(n_sample, n_sample, FRAC, seed=SEED + 1000)
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(reps):
        m = oracle_step([lk, lp], [rk, rp], P)
    dt = (time.perf_counter() - t0) / reps
    assert m == math.floor(FRAC * n_sample)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    threads = max(1, min(cores, P))
    t0 = time.perf_counter()
    for _ in range(reps):
        m = oracle_step([lk, lp], [rk, rp], P, threads=threads)
    dt_all = (time.perf_counter() - t0) / reps
    assert m == math.floor(FRAC * n_sample)
    return {"value": 2 * n_sample / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n_sample} x {n_sample} rows of the same generator (seed {SEED + 1000}), P={P}: "
                      f"stable partition of both sides + sort-merge per partition, single thread, "
                      f"{dt:.2f} s per merge",
            "all_cores": {"value": 2 * n_sample / dt_all, "unit": UNIT, "cores": threads,
                          "host_cores": cores, "ms_per_merge": round(dt_all * 1e3, 1)}}


# --------------------------------------------------------------- GPU arm

def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (x itself when there is one rank): the
    job's time is its slowest replica's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(rows_per_rank: int, world: int, seconds: float) -> float:
    """Rows merged by all replicas per second of the slowest one."""
    return rows_per_rank * world / seconds


# Steps of the hot path as the roofline counts them (8-byte keys and
# payloads, 4-byte row ids): the per-side histogram read (a2), the exchange
# (a4: read a row, write it with its row id; a second internal radix pass is
# overhead and adds no algorithmic bytes) and the join (a5-a7: read both
# sides' partitioned rows, write the output rows).
STEP_KERNELS = {
    "hist": ("a2 histogram", ["hist"]),
    "exchange": ("a4 scatter (the exchange)", ["shuffle_pass1", "shuffle_pass2", "scatter_stable",
                                               "scatter_reserve"]),
    "join": ("a5-a7 build + probe + write", ["join_write", "join_write_exact"]),
}


def step_alg_bytes(step: str, n_left: int, n_right: int, m: int) -> int:
    if step == "hist":
        return KEY * (n_left + n_right)
    if step == "exchange":
        return ((KEY + PAY) + (KEY + PAY + RID)) * (n_left + n_right)
    return (KEY + PAY + RID) * (n_left + n_right) + OUT_ROW * m


def step_rooflines(prof: dict, steps: int, n_left: int, n_right: int, m: int, peak: float):
    """Per-step achieved bandwidth: the step's algorithmic bytes per merge over
    the device time of its kernels per merge (CUDA events around every launch,
    on the launch stream)."""
    out = {}
    for step, (label, names) in STEP_KERNELS.items():
        ms = sum(prof[k][1] for k in names if k in prof) / steps
        launches = sum(prof[k][0] for k in names if k in prof) // max(steps, 1)
        if ms <= 0:
            continue
        alg = step_alg_bytes(step, n_left, n_right, m)
        gbs = alg / (ms / 1e3) / 1e9
        out[step] = {"what": label, "kernels": [k for k in names if k in prof], "launches_per_merge": launches,
                     "ms_per_merge": round(ms, 4), "alg_bytes_per_merge": alg, "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / peak, 4)}
    return out


def run_gpu(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08878_gb300 import mdj

    (lk, lp), (rk, rp) = datagen.match_fraction_tables(N_LEFT, N_RIGHT, FRAC, seed=SEED + rank)
    left = [torch.from_numpy(lk).to(dev), torch.from_numpy(lp).to(dev)]
    right = [torch.from_numpy(rk).to(dev), torch.from_numpy(rp).to(dev)]
    m_expect = math.floor(FRAC * N_RIGHT)

    def barrier():
        if dist is not None:
            dist.barrier()

    def step():
        res = mdj.mdj_merge(left, right, P)
        assert res.nrows == m_expect, res.nrows
        return res

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the timed region: K steps without launch tracing (value, ms_per_step)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            res = step()
            del res
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms_total = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    # K more steps with every launch bracketed by CUDA events on its stream:
    # the per-kernel times (rooflines, launch list, launch count)
    mdj.profile_reset()
    mdj.profile_enable(True)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        res = step()
        del res
    t1.record(stream)
    torch.cuda.synchronize()
    mdj.profile_enable(False)
    prof = mdj.profile_collect()
    ms_traced_step = t0.elapsed_time(t1) / args.steps
    ms_step = ms_total / args.steps
    value = whole_job_rate(N_LEFT + N_RIGHT, world, ms_step / 1e3)

    # ---- roofline: the dominant step of the path (by device time inside the
    # timed region), its algorithmic bytes per merge over its kernels' time
    peak, peak_kind = peaks()
    launches = sum(v[0] for v in prof.values())
    steps_roof = step_rooflines(prof, args.steps, N_LEFT, N_RIGHT, m_expect, peak)
    dom_step = max(steps_roof, key=lambda k: steps_roof[k]["ms_per_merge"])
    d = steps_roof[dom_step]
    traffic = measured_traffic(dom_step)
    b_alg_step = step_alg_bytes("hist", N_LEFT, N_RIGHT, m_expect) + \
        step_alg_bytes("exchange", N_LEFT, N_RIGHT, m_expect) + step_alg_bytes("join", N_LEFT, N_RIGHT, m_expect)
    assert b_alg_step == 64 * (N_LEFT + N_RIGHT) + OUT_ROW * m_expect
    roofline = {
        "bound": "hbm", "kernel": f"{dom_step}: {d['what']} ({', '.join(d['kernels'])})",
        "achieved": d["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": d["frac"],
        "traffic": traffic,
        "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6800 GB/s",
        "ms_per_merge": d["ms_per_merge"], "alg_bytes_per_merge": d["alg_bytes_per_merge"],
        "launches_per_merge": d["launches_per_merge"],
    }
    step_roof = {"alg_bytes": b_alg_step, "achieved_gbs": round(b_alg_step / (ms_step / 1e3) / 1e9, 1),
                 "frac": round(b_alg_step / (ms_step / 1e3) / 1e9 / peak, 4), "steps": steps_roof}
    kernels = {k: {"launches": v[0], "ms_per_step": round(v[1] / args.steps, 4),
                   "share": round(v[1] / max(sum(x[1] for x in prof.values()), 1e-9), 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    # ---- the same merge through the streamed-output path, one window of all rows
    stream_plain = None
    if args.stream_windows > 0:
        stream_plain = stream_whole(left, right, m_expect, ms_step, dev)

    # ---- the same join with the key written as two int32 columns
    multi_key = None
    if args.multikey_steps > 0:
        multi_key = multikey_section(args, left, right, m_expect, ms_step, dev)

    # ---- end to end through the C ABI with host buffers: mdj_merge_host takes
    # the pinned host tables, copies them in, merges, and hands the result to
    # a sink that copies it into pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        hl = [torch.from_numpy(lk).pin_memory(), torch.from_numpy(lp).pin_memory()]
        hr = [torch.from_numpy(rk).pin_memory(), torch.from_numpy(rp).pin_memory()]
        del left[:], right[:]
        torch.cuda.empty_cache()
        e2e = e2e_section(args, dev, hl, hr, m_expect, dist, world)
        del hl, hr

    # ---- the same tables merged from host memory under a 1 GiB device budget
    # (after e2e: its host-memory traffic would otherwise sit in e2e's timing)
    host_tables = None
    if args.host_budget_mib > 0:
        torch.cuda.empty_cache()
        host_tables = host_tables_section(args, dev, (lk, lp), (rk, rp), m_expect)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_left": N_LEFT, "n_right": N_RIGHT, "P": P, "match_fraction": FRAC,
                   "output_rows": m_expect, "seed": SEED, "l2": "inputs (3.2 GB) larger than L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "step_roofline": step_roof, "kernels": kernels, "gpu_launches": launches,
        "timing": {"value_from": f"{args.steps} steps without launch tracing",
                   "kernels_from": f"{args.steps} further steps with CUDA events around every launch "
                                   f"({round(ms_traced_step, 4)} ms per step with the tracing)"},
        "e2e": e2e, "clocks": clk.summary(),
    }
    if host_tables is not None:
        line["host_tables"] = host_tables
    if multi_key is not None:
        line["multi_key"] = multi_key

    def section(name, fn):
        # a section that fails reports its error in the line instead of
        # taking the whole line with it
        try:
            torch.cuda.empty_cache()
            line[name] = fn()
        except Exception as e:  # noqa: BLE001
            line[name] = {"error": f"{type(e).__name__}: {e}"}

    if args.latency_calls > 0:
        section("plain_1M", lambda: plain_1m_section(args, dev))
    if args.stream_windows > 0:
        section("streamed", lambda: dict(streamed_section(args, dev), plain_workload_one_window=stream_plain))
    if args.transpose_steps > 0:
        section("transpose_sum", lambda: transpose_section(args, dev))
    if args.batch_pairs > 0:
        section("batched", lambda: batched_section(args, dev))
    if args.serve_requests > 0:
        section("served", lambda: served_section(args, dev))
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def e2e_section(args, dev, hl, hr, m_expect, dist, world):
    """mdj_merge_host (the library's host-table entry point) from pinned host
    tables to pinned host result buffers, timed on the host around each call
    (the call synchronises its stream before it returns)."""
    import torch
    from paper_2101_08878_gb300 import mdj

    budget = 32 << 30  # both tables fit one bucket: copied in once, merged in place
    out = {"key": torch.empty(m_expect, dtype=torch.int64, pin_memory=True),
           "lrow": torch.empty(m_expect, dtype=torch.uint32, pin_memory=True),
           "rrow": torch.empty(m_expect, dtype=torch.uint32, pin_memory=True),
           "lpay": torch.empty(m_expect, dtype=torch.float64, pin_memory=True),
           "rpay": torch.empty(m_expect, dtype=torch.float64, pin_memory=True)}

    def to_host(first, piece):
        n = piece.nrows
        out["key"][first:first + n].copy_(piece.key, non_blocking=True)
        out["lrow"][first:first + n].copy_(piece.left_row, non_blocking=True)
        out["rrow"][first:first + n].copy_(piece.right_row, non_blocking=True)
        out["lpay"][first:first + n].copy_(piece.left_cols[0], non_blocking=True)
        out["rpay"][first:first + n].copy_(piece.right_cols[0], non_blocking=True)

    def call():
        total, _ = mdj.merge_host_chunked(hl, hr, P, budget, on_piece=to_host, device=dev)
        assert total == m_expect, total
        return total

    call()
    call()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        call()
        times.append(time.perf_counter() - t0)
    dt = max_over_ranks(statistics.mean(times), dist, dev)
    # spot check: the host copy holds joined rows (key equals the left key of its left row)
    lk_host = hl[0]
    idx = torch.randint(0, m_expect, (1000,))
    lrow = out["lrow"].view(torch.int32)[idx].to(torch.int64) & 0xFFFFFFFF
    assert torch.equal(out["key"][idx], lk_host[lrow])
    h2d = sum(c.numel() * c.element_size() for c in list(hl) + list(hr))
    d2h = sum(t.numel() * t.element_size() for t in out.values())
    return {"value": whole_job_rate(N_LEFT + N_RIGHT, world, dt), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(dt * 1e3, 3), "steps": args.e2e_steps,
            "api": "mdj_merge_host (C ABI): pinned host tables in, sink copies each result window to pinned "
                   "host buffers; host wall time per call"}


def plain_1m_section(args, dev):
    """The 1M x 1M plain merge with one partition (unique left keys, match
    fraction 0.3): latency of single mdj_merge calls, host-observed (the call
    returns after the output count is read back and the rows are written)
    and on the device (CUDA events around the call)."""
    import torch
    from paper_2101_08878_gb300 import mdj

    (lk, lp), (rk, rp) = datagen.match_fraction_tables(1_000_000, 1_000_000, FRAC, seed=0)
    L = [torch.from_numpy(lk).to(dev), torch.from_numpy(lp).to(dev)]
    R = [torch.from_numpy(rk).to(dev), torch.from_numpy(rp).to(dev)]
    stream = torch.cuda.current_stream(dev)
    for _ in range(20):
        assert mdj.mdj_merge(L, R, 1).nrows == 300_000
    torch.cuda.synchronize()
    host_ms, dev_ms = [], []
    for _ in range(args.latency_calls):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        res = mdj.mdj_merge(L, R, 1)
        e1.record(stream)
        host_ms.append((time.perf_counter() - t0) * 1e3)
        assert res.nrows == 300_000
        del res
        e1.synchronize()
        dev_ms.append(e0.elapsed_time(e1))
    q = (lambda v, f: float(np.percentile(np.array(v), f)))
    return {"workload": "plain inner merge, P=1: 1M x 1M rows, unique left keys, match fraction 0.3, 300,000 rows out",
            "calls": args.latency_calls, "p50_ms": round(q(host_ms, 50), 4), "p99_ms": round(q(host_ms, 99), 4),
            "device_p50_ms": round(q(dev_ms, 50), 4), "device_p99_ms": round(q(dev_ms, 99), 4),
            "value": 2_000_000 / (q(host_ms, 50) / 1e3), "unit": "input rows/s at p50"}


def multikey_section(args, left, right, m_expect, merge_ms, dev):
    """The bench join with each key split into two int32 key columns (high
    and low bits): mdj_merge_multi (tuple surrogate, merge, verification) on
    the pair, against mdj_merge on the single key.  Same rows either way."""
    import torch
    from paper_2101_08878_gb300 import mdj

    def split(k):
        return [(k >> 20).to(torch.int32), (k & 0xFFFFF).to(torch.int32)]

    L = split(left[0]) + [left[1]]
    R = split(right[0]) + [right[1]]
    stream = torch.cuda.current_stream(dev)

    def step():
        res = mdj.mdj_merge_multi(L, R, [0, 1], [0, 1], P)
        assert res.nrows == m_expect
        return res

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.multikey_steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.multikey_steps
    del L, R
    return {"workload": "the bench tables, key written as (key >> 20, key & 0xFFFFF) int32 columns",
            "ms_per_step": round(ms, 3), "value": (N_LEFT + N_RIGHT) / (ms / 1e3), "unit": UNIT,
            "single_key_merge_ms": round(merge_ms, 3), "rows": m_expect}


def host_tables_section(args, dev, left_np, right_np, m_expect):
    """The bench tables held in host memory (3.2 GB, pageable) and merged
    through mdj_merge_host with a device budget smaller than the tables:
    chunked hash partition into host staging, then one stream per bucket pair,
    each window handed to a sink that counts rows (nothing is kept).  Wall
    time of the first full-size call (after a warm-up call on a 1/10 sample)
    and the median of three more: the device's first accesses to host pages
    cost extra on this host, so the first call is reported on its own."""
    import torch
    from paper_2101_08878_gb300 import mdj

    budget = args.host_budget_mib << 20
    L = [torch.from_numpy(c) for c in left_np]
    R = [torch.from_numpy(c) for c in right_np]
    seen = [0]

    def count(first_row, piece):
        seen[0] += piece.nrows

    k = len(L[0]) // 10
    mdj.merge_host_chunked([c[:k] for c in L], [c[:k] for c in R], P, budget, on_piece=count, device=dev)
    walls = []
    for _ in range(4):
        seen[0] = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        total, _ = mdj.merge_host_chunked(L, R, P, budget, on_piece=count, device=dev)
        walls.append(time.perf_counter() - t0)
        assert total == seen[0] == m_expect, (total, seen[0])
    wall = float(np.median(walls[1:]))
    in_bytes = sum(c.numel() * c.element_size() for c in L + R)
    return {"workload": "the bench tables in pageable host memory, inner merge, sink counts rows",
            "device_budget_bytes": budget, "input_bytes": in_bytes, "rows": total,
            "first_call_s": round(walls[0], 3), "wall_s": round(wall, 3), "calls_s": [round(w, 3) for w in walls],
            "value": (len(L[0]) + len(R[0])) / wall, "unit": "input rows/s (median of calls 2-4)"}


def stream_whole(left, right, m_expect, merge_ms, dev):
    """The bench workload through mdj_stream_open + one window of every row,
    against mdj_merge: what the streamed path costs when the result fits."""
    import torch
    from paper_2101_08878_gb300 import mdj

    def once(how="inner"):
        t0 = time.perf_counter()
        st = mdj.MergeStream(left, right, P, how=how)
        t_open = time.perf_counter() - t0
        assert how != "inner" or st.total_rows == m_expect
        rows = st.total_rows
        buf = st.buffers(st.total_rows)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.emit(0, st.total_rows, buf)
        e1.record(stream)
        torch.cuda.synchronize()
        st.close()
        del buf
        return t_open * 1e3, e0.elapsed_time(e1), rows

    once()
    runs = [once() for _ in range(3)]
    open_ms = statistics.median(r[0] for r in runs)
    emit_ms = statistics.median(r[1] for r in runs)
    once("outer")
    o_open, o_emit, o_rows = once("outer")
    return {"open_ms": round(open_ms, 3), "emit_ms": round(emit_ms, 3),
            "total_ms": round(open_ms + emit_ms, 3), "merge_ms": round(merge_ms, 3),
            "rows": m_expect, "note": "open is host-timed (it ends with the count read back); emit by CUDA events",
            "outer_join": {"rows": o_rows, "open_ms": round(o_open, 3), "emit_ms": round(o_emit, 3)}}


def zipf_device(n: int, n_values: int, s: float, gen, dev):
    """n keys in [0, n_values), P(key = k-1) proportional to k^-s, by inverse CDF on the device."""
    import torch
    k = torch.arange(1, n_values + 1, dtype=torch.float64, device=dev)
    cdf = torch.cumsum(k.pow(-s), 0)
    cdf /= cdf[-1].clone()
    u = torch.rand(n, generator=gen, dtype=torch.float64, device=dev)
    return torch.searchsorted(cdf, u, right=True).clamp_(max=n_values - 1).to(torch.int64)


def streamed_section(args, dev):
    """The skewed many-to-many workload (Zipf(1.1) keys over 1e7 values on both
    sides, 50M x 200M rows, P = 64; about 2.0e14 joined rows) through the
    streamed-output path: mdj_stream_open once, then windows of 2^26 rows at
    offsets spread over the whole result, each written by one emit kernel into
    one reused 2.1 GB buffer.  Keys and payloads are drawn on the device
    (seeded torch generator) with the distribution of the test generator."""
    import torch
    from paper_2101_08878_gb300 import mdj

    n_l, nvals, P_z = args.stream_left, 10_000_000, 64
    n_r = 4 * n_l
    g = torch.Generator(device=dev)
    g.manual_seed(2)
    L = [zipf_device(n_l, nvals, 1.1, g, dev), torch.rand(n_l, generator=g, dtype=torch.float64, device=dev)]
    R = [zipf_device(n_r, nvals, 1.1, g, dev), torch.rand(n_r, generator=g, dtype=torch.float64, device=dev)]
    torch.cuda.synchronize()
    mdj.MergeStream(L, R, P_z).close()  # first launches of the stream kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = mdj.MergeStream(L, R, P_z)
    open_s = time.perf_counter() - t0
    m = st.total_rows
    W = min(1 << 26, m)
    buf = st.buffers(W)
    stream = torch.cuda.current_stream(dev)
    k = args.stream_windows
    offsets = [int(i * (m - W) // max(k - 1, 1)) for i in range(k)]
    st.emit(offsets[0], W, buf)  # warm
    ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for q0 in offsets:
        e0.record(stream)
        st.emit(q0, W, buf)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    # a row of every window is checked against its source rows
    li = buf.left_row[-1].view(torch.int32).to(torch.int64)
    ri = buf.right_row[-1].view(torch.int32).to(torch.int64)
    assert int(L[0][li]) == int(R[0][ri]) == int(buf.key[-1])
    st.close()
    # count + checksum mode on the same tables (mdj_count_checksum): its
    # count must equal the stream's row count
    mdj.mdj_count_checksum(L, R, P_z)  # warm
    torch.cuda.synchronize()
    cms = []
    for _ in range(3):
        t1 = time.perf_counter()
        cnt, csum = mdj.mdj_count_checksum(L, R, P_z)
        cms.append((time.perf_counter() - t1) * 1e3)
    assert cnt == m, (cnt, m)
    count_mode = {"rows": cnt, "checksum": csum, "ms": round(statistics.median(cms), 3),
                  "value": (n_l + n_r) / (statistics.median(cms) / 1e3), "unit": "input rows/s",
                  "note": "host wall time per mdj_count_checksum call (ends with the totals read back); "
                          "the count equals the streamed output's row count"}
    peak, _ = peaks()
    med = statistics.median(ms)
    per_row = OUT_ROW + RID + PAY  # written row + the grouped build side's row id and payload read
    achieved = per_row * W / (med / 1e3) / 1e9
    rate = W / (med / 1e3)
    return {"workload": f"Zipf(1.1) over {nvals} values both sides, {n_l} x {n_r} rows, P={P_z}, int64 key + "
                        "float64 payload (drawn on the device, seeded)",
            "total_rows": m, "open_ms": round(open_s * 1e3, 2),
            "open_input_rows_per_s": (n_l + n_r) / open_s,
            "window_rows": W, "windows": k, "window_offsets": offsets, "ms_per_window": [round(x, 4) for x in ms],
            "emit": {"value": rate, "unit": "output rows/s", "ms_per_window": round(med, 4),
                     "roofline": {"bound": "hbm", "kernel": "stream_emit", "achieved": round(achieved, 1),
                                  "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                                  "alg_bytes_per_row": per_row,
                                  "note": "32 B written + 12 B grouped build side read per row; probe-side "
                                          "and entry reads not counted"}},
            "all_rows_estimate_s": round(m / rate, 1), "count_mode": count_mode}


def transpose_section(args, dev):
    """The paper's other application benchmark, y = x + x.T on a float64
    array: 16K x 16K (Fig. 7) and 20E3 x 20E3 (Fig. 9(a)), x drawn U[0,1) on
    the device (seeded).  One step = one mdj_transpose_add call; algorithmic
    bytes = 16 per element (x read once, y written once); arrays of 2-3 GB
    are far larger than L2.  The CPU oracle (numpy x + x.T, one thread) is
    timed on a 4096 x 4096 sample."""
    import torch
    from paper_2101_08878_gb300 import mdj
    import oracle

    peak, _ = peaks()
    stream = torch.cuda.current_stream(dev)
    sizes = []
    for n in (16384, 20000):
        g = torch.Generator(device=dev)
        g.manual_seed(n)
        x = torch.rand((n, n), generator=g, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)
        for _ in range(3):
            mdj.transpose_add(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.transpose_steps):
            mdj.transpose_add(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.transpose_steps
        i, j = 12345 % n, n - 7
        assert float(y[i, j]) == float(x[i, j]) + float(x[j, i])
        alg = 16 * n * n
        achieved = alg / (ms / 1e3) / 1e9
        sizes.append({"n": n, "ms_per_step": round(ms, 4), "elements_per_s": n * n / (ms / 1e3),
                      "roofline": {"bound": "hbm", "kernel": "transpose_add", "achieved": round(achieved, 1),
                                   "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                                   "alg_bytes_per_launch": alg}})
        del x, y
        torch.cuda.empty_cache()
    oracle.build()
    xs = np.random.default_rng(0).random((4096, 4096))
    oracle.transpose_add(xs)
    t0 = time.perf_counter()
    for _ in range(3):
        oracle.transpose_add(xs)
    cpu_s = (time.perf_counter() - t0) / 3
    return {"workload": "y = x + x.T, float64, 16384^2 and 20000^2 (x U[0,1) drawn on the device, seeded)",
            "steps": args.transpose_steps, "sizes": sizes,
            "cpu_baseline": {"value": 4096 * 4096 / cpu_s, "unit": "elements/s", "cores": 1, "kind": "oracle",
                             "sample": "numpy x + x.T on a 4096 x 4096 float64 array, one thread"}}


def batched_section(args, dev):
    """The batched workload: 256 independent partition-pair joins (n_L, n_R log-uniform in
    [1K, 4M], match fraction U[0.1, 0.9]) through mdj_join_batch (tuned) versus
    the plain path, one mdj_join call per pair.  Input rows/s of each."""
    import torch
    from paper_2101_08878_gb300 import mdj
    from paper_2101_08878_gb300.tuner import BatchTuner

    pairs = datagen.batch_pairs(args.batch_pairs, 1_000, 4_000_000, seed=3)
    lo = np.concatenate([[0], np.cumsum([p[0][0].size for p in pairs])]).astype(np.uint64)
    ro = np.concatenate([[0], np.cumsum([p[1][0].size for p in pairs])]).astype(np.uint64)
    L = [torch.from_numpy(np.concatenate([p[0][0] for p in pairs])).to(dev),
         torch.from_numpy(np.concatenate([p[0][1] for p in pairs])).to(dev)]
    R = [torch.from_numpy(np.concatenate([p[1][0] for p in pairs])).to(dev),
         torch.from_numpy(np.concatenate([p[1][1] for p in pairs])).to(dev)]
    rows = int(lo[-1] + ro[-1])
    expect = sum(int(np.count_nonzero(p[1][0] < p[0][0].size)) for p in pairs)
    del pairs
    tuner = BatchTuner()
    tr, fp, jt = tuner.choose(L, R, lo, ro)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def batched():
        res, po = mdj.mdj_join_batch(L, R, lo, ro, 0, 0, tr, fp, jt)
        assert res.nrows == expect

    def plain():
        m = 0
        for i in range(len(lo) - 1):
            a, b, c, d = int(lo[i]), int(lo[i + 1]), int(ro[i]), int(ro[i + 1])
            m += mdj.mdj_join([L[0][a:b], L[1][a:b]], [R[0][c:d], R[1][c:d]]).nrows
        assert m == expect

    ms_b = timed(batched, 5)
    ms_p = timed(plain, 2)
    return {"workload": f"{len(lo) - 1} pairs, sizes log-uniform [1K, 4M] per side, match U[0.1, 0.9], "
                        f"int64 key + float64 payload, {rows} input rows, {expect} output rows",
            "batched": {"value": rows / (ms_b / 1e3), "unit": UNIT, "ms_per_batch": round(ms_b, 3),
                        "tuning": {"table_rows": tr, "fill_pct": fp, "join_threads": jt,
                                   "searched": "table rows {2048, 4096, 8192} x fill {60, 75, 85, 95}% x "
                                               "join block {256, 512} threads, timed on this batch"}},
            "plain_per_pair": {"value": rows / (ms_p / 1e3), "unit": UNIT, "ms_per_batch": round(ms_p, 3)},
            "speedup": round(ms_p / ms_b, 3)}


_FP_M = (1 << 64) - 1


def _fp_mix_np(x):
    x = x ^ (x >> np.uint64(33))
    x = x * np.uint64(0xFF51AFD7ED558CCD)
    x = x ^ (x >> np.uint64(33))
    x = x * np.uint64(0xC4CEB9FE1A85EC53)
    return x ^ (x >> np.uint64(33))


def fingerprint_np(key, lrow, rrow, lpay, rpay):
    """Order-independent fingerprint of a join result: (rows, sum over rows of
    a 64-bit mix of every column's bits, modulo 2^64).  Two results agree on
    it when they hold the same multiset of rows (up to a 2^-64 chance)."""
    with np.errstate(over="ignore"):
        bits = (lambda a: np.ascontiguousarray(a).view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)
                .astype(np.uint64))
        h = _fp_mix_np(bits(key) ^ np.uint64(0x9E3779B97F4A7C15))
        h = _fp_mix_np(h ^ (bits(lrow) * np.uint64(0xBF58476D1CE4E5B9)))
        h = _fp_mix_np(h ^ (bits(rrow) * np.uint64(0x94D049BB133111EB)))
        h = _fp_mix_np(h ^ bits(lpay))
        h = _fp_mix_np(h ^ (bits(rpay) + np.uint64(0x632BE59BD9B4E019)))
        return int(key.size), int(h.sum(dtype=np.uint64))


_FP_CONST = {}


def _fp_consts(dev):
    """The fingerprint's 64-bit constants as int64 device scalars (cached)."""
    import torch
    key = str(dev)
    if key not in _FP_CONST:
        vals = [0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53, 0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9,
                0x94D049BB133111EB, 0x632BE59BD9B4E019]
        _FP_CONST[key] = [torch.tensor(v - (1 << 64) if v >= (1 << 63) else v, dtype=torch.int64, device=dev)
                          for v in vals]
    return _FP_CONST[key]


def _fp_mix_t(x, k):
    lsr = (lambda v, s: (v >> s) & ((1 << (64 - s)) - 1))  # logical shift of int64 bits
    x = x ^ lsr(x, 33)
    x = x * k[0]
    x = x ^ lsr(x, 33)
    x = x * k[1]
    return x ^ lsr(x, 33)


def fingerprint_torch(res):
    """fingerprint_np on a device JoinResult (int64 arithmetic wraps modulo
    2^64 like uint64); returns a device tensor [sum] (the row count is known
    on the host)."""
    import torch

    def bits(t):
        if t.element_size() == 4:
            return t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        return t.view(torch.int64)

    k = _fp_consts(res.key.device)
    h = _fp_mix_t(bits(res.key) ^ k[2], k)
    h = _fp_mix_t(h ^ (bits(res.left_row) * k[3]), k)
    h = _fp_mix_t(h ^ (bits(res.right_row) * k[4]), k)
    h = _fp_mix_t(h ^ bits(res.left_cols[0]), k)
    h = _fp_mix_t(h ^ (bits(res.right_cols[0]) + k[5]), k)
    return h.sum().reshape(1)


def _oracle_fp(args):
    """Worker of the served check: the oracle's join of one request, fingerprinted."""
    lk, lp, rk, rp = args
    import oracle
    want = oracle.merge_table([lk, lp], [rk, rp])
    return fingerprint_np(want["key"], want["left_row"], want["right_row"], want["left_cols"][0],
                          want["right_cols"][0])


def served_requests(n: int, seed: int = 4):
    """The request stream's parameters: P in {1, 8, 32}, n_L and n_R log-uniform
    in [1e4, 2e7], int32 or int64 keys and float32 or float64 payloads (50/50)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nl = int(datagen.log_uniform_sizes(rng, 1, 10_000, 20_000_000)[0])
        nr = int(datagen.log_uniform_sizes(rng, 1, 10_000, 20_000_000)[0])
        kd = "int32" if rng.random() < 0.5 else "int64"
        pd = "float32" if rng.random() < 0.5 else "float64"
        out.append({"i": i, "nl": nl, "nr": nr, "key": kd, "pay": pd, "P": int(rng.choice([1, 8, 32]))})
    return out


def request_tables(spec, dev):
    """One request's tables on the device from its own seed (the match-fraction
    recipe: left keys a permutation of [0, n_L), floor(0.3 n_R) right keys drawn
    from the left keys, the rest from [n_L, 2 n_L), right rows shuffled;
    payloads U[0, 1))."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(4000 + spec["i"])
    kd = getattr(torch, spec["key"])
    pd = getattr(torch, spec["pay"])
    nl, nr = spec["nl"], spec["nr"]
    m = math.floor(FRAC * nr)
    lk = torch.randperm(nl, generator=g, device=dev).to(kd)
    pick = torch.randint(0, nl, (m,), generator=g, device=dev)
    rk = torch.cat([lk[pick], torch.randint(nl, 2 * nl, (nr - m,), generator=g, device=dev).to(kd)])
    rk = rk[torch.randperm(nr, generator=g, device=dev)]
    lp = torch.rand(nl, generator=g, device=dev, dtype=pd)
    rp = torch.rand(nr, generator=g, device=dev, dtype=pd)
    return [lk, lp], [rk, rp], m


def _canonical(res):
    """The rows of a device JoinResult sorted by (key, left_row, right_row), all columns."""
    import torch
    order = torch.argsort(res.right_row.view(torch.int32).to(torch.int64) & 0xFFFFFFFF, stable=True)
    for col in (res.left_row.view(torch.int32).to(torch.int64) & 0xFFFFFFFF, res.key.to(torch.int64)):
        order = order[torch.argsort(col[order], stable=True)]
    as_indexable = (lambda t: t.view(torch.int32) if t.dtype == torch.uint32 else t)
    return [as_indexable(t)[order] for t in [res.key, res.left_row, res.right_row, *res.left_cols, *res.right_cols]]


def served_canonical_check(work, dev, max_batch_rows, groups: int = 8, per_group: int = 4):
    """Seeded groups of requests with one dtype class are served together
    (MergeServer, batching on) and every result is compared, column by column
    and bit for bit after the canonical sort, with the request run alone."""
    import asyncio
    import torch
    from paper_2101_08878_gb300 import mdj
    from paper_2101_08878_gb300.server import MergeServer, run_poisson

    rng = np.random.default_rng(47)
    by_cls = {}
    for i, (L, R, P_, m) in enumerate(work):
        by_cls.setdefault((L[0].dtype, L[1].dtype), []).append(i)
    checked = 0
    for g in range(groups):
        cls = sorted(by_cls, key=str)[g % len(by_cls)]
        pick = rng.choice(by_cls[cls], min(per_group, len(by_cls[cls])), replace=False).tolist()
        wl = [work[i][:3] for i in pick]
        server = MergeServer(dev, slots=1, batching=True, max_batch_rows=max_batch_rows)
        reqs, _ = asyncio.run(run_poisson(server, wl, np.zeros(len(wl))))
        for i, req in zip(pick, reqs):
            assert req.error is None, req.error
            L, R, P_, m = work[i]
            a = _canonical(mdj.mdj_merge(L, R, P_))
            b = _canonical(req.result)
            for x, y in zip(a, b):
                if not torch.equal(x.view(torch.uint8), y.view(torch.uint8)):
                    raise RuntimeError(f"request {i}: served rows differ from the same request alone")
            req.result = None
            checked += 1
    return {"requests": checked, "how": "batches of up to 4 same-dtype requests, canonical sort, bit for bit"}


def served_section(args, dev):
    """The served workload at its configured scale: a Poisson stream of
    merge requests, each with its own tables generated on the device from the
    request's seed, served by MergeServer with continuous batching versus the
    plain per-request path (one slot, no batching) at 0.5x, 1x and 2x the
    plain path's capacity.  Every served result is checked against the same
    request run alone (fingerprint over all columns' bits, and a full
    canonical compare for a sample), and a seeded sample of requests plus
    every request with both sides at most 1M rows against the CPU oracle."""
    import asyncio
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import torch
    from paper_2101_08878_gb300 import mdj
    from paper_2101_08878_gb300.server import MergeServer, latency_stats, run_poisson

    specs = served_requests(args.serve_requests)
    work = []
    for sp in specs:
        L, R, m = request_tables(sp, dev)
        work.append((L, R, sp["P"], m))
    torch.cuda.synchronize()
    rows_all = sum(sp["nl"] + sp["nr"] for sp in specs)
    # every request alone (the plain path), fingerprinted
    alone_rows, alone = [], []
    for L, R, P_, m in work:
        res = mdj.mdj_merge(L, R, P_)
        assert res.nrows == m
        alone_rows.append(res.nrows)
        alone.append(fingerprint_torch(res))
        del res
    alone = torch.cat(alone).cpu()
    # served and plain runs: every result's fingerprint against the alone one
    fps = {}

    def consume(req):
        if req.result is not None:
            r = req.result
            fps[id(req)] = (r.nrows, fingerprint_torch(r))
            for t in [r.key, r.left_row, r.right_row, *r.left_cols, *r.right_cols]:
                t.record_stream(torch.cuda.current_stream(dev))
            req.result = None

    def run(rate, batching, slots, idx):
        wl = [work[int(i)][:3] for i in idx]
        rows = sum(int(w[0][0].numel() + w[1][0].numel()) for w in wl)
        server = MergeServer(dev, slots=slots, batching=batching, max_batch_rows=args.serve_batch_rows)
        arrivals = np.cumsum(np.random.default_rng(44).exponential(1.0 / rate, len(wl)))
        fps.clear()
        reqs, wall = asyncio.run(asyncio.wait_for(run_poisson(server, wl, arrivals, consume), 600))
        bad = [r.error for r in reqs if r.error is not None]
        if bad:
            raise RuntimeError(f"served requests failed: {bad[0]}")
        got = torch.cat([fps[id(r)][1] for r in reqs]).cpu()
        want = alone[torch.as_tensor(np.asarray(idx, dtype=np.int64))]
        mism = int((got != want).sum()) + sum(1 for r, i in zip(reqs, idx) if fps[id(r)][0] != alone_rows[int(i)])
        if mism:
            raise RuntimeError(f"{mism} served results differ from the same requests run alone")
        st = latency_stats(reqs)
        st["rows_per_s"] = rows / wall
        st["wall_s"] = round(wall, 3)
        st["mean_batch"] = round(float(np.mean(server.group_sizes)), 2)
        st["checked_vs_alone"] = len(reqs)
        return st

    idx_all = np.arange(len(work))
    canonical_checked = served_canonical_check(work, dev, args.serve_batch_rows)
    run(1e9, True, 2, idx_all[:100])  # first launches of each path stay out of the timed runs
    run(1e9, False, 1, idx_all[:100])
    cap = run(1e9, False, 1, idx_all)  # capacity of the plain path: everything queued at once
    cap_rps = len(work) / cap["wall_s"]
    out = {"workload": f"{len(work)} requests, each with its own tables generated on the device from its seed; "
                       f"P in {{1,8,32}}, n_L, n_R log-uniform [1e4, 2e7], int32/int64 keys, float32/float64 "
                       f"payloads, match 0.3; {rows_all} input rows in all",
           "served_config": {"slots": 2, "max_batch_rows": args.serve_batch_rows},
           "plain_config": {"slots": 1, "batching": False},
           "plain_capacity_requests_per_s": round(cap_rps, 2), "rates": []}
    for mult in (0.5, 1.0, 2.0):
        rate = mult * cap_rps
        out["rates"].append({"x_plain_capacity": mult, "requests_per_s": round(rate, 2),
                             "served": run(rate, True, 2, idx_all), "plain": run(rate, False, 1, idx_all)})
    # oracle: a seeded sample plus every request with both sides <= 1M rows
    small = [i for i, sp in enumerate(specs) if sp["nl"] <= 1_000_000 and sp["nr"] <= 1_000_000]
    sample = sorted(set(np.random.default_rng(46).choice(len(specs), min(100, len(specs)), replace=False).tolist())
                    | set(small))
    jobs = [(work[i][0][0].cpu().numpy(), work[i][0][1].cpu().numpy(), work[i][1][0].cpu().numpy(),
             work[i][1][1].cpu().numpy()) for i in sample]
    with ProcessPoolExecutor(max_workers=max(1, min(16, host_cores())), mp_context=mp.get_context("spawn")) as ex:
        want = list(ex.map(_oracle_fp, jobs, chunksize=4))
    got = alone[torch.as_tensor(sample, dtype=torch.int64)].tolist()
    wrong = sum(1 for (n, h), g, i in zip(want, got, sample)
                if n != alone_rows[i] or (h - (1 << 64) if h >= (1 << 63) else h) != g)
    if wrong:
        raise RuntimeError(f"{wrong} of {len(sample)} requests differ from the CPU oracle")
    out["checked_vs_oracle"] = {"requests": len(sample), "with_both_sides_le_1M": len(small), "mismatches": 0}
    out["checked_row_for_row_alone_vs_batched"] = canonical_checked
    del work
    return out


def measured_traffic(step: str):
    """DRAM bytes per merge of one step of the path (dram__bytes_read.sum +
    dram__bytes_write.sum of its kernels) from a committed ncu summary, scaled
    from the captured case by input rows, if the step's source files (comma-
    separated, hashed together) are unchanged since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    src = os.path.join(ROOT, "paper_2101_08878_gb300", "csrc")
    try:
        rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    for r in rows:
        kv = dict(x.split("=", 1) for x in r if "=" in x)
        if kv.get("step") != step:
            continue
        blob = b"".join(open(os.path.join(src, f), "rb").read() for f in kv["files"].split(","))
        h = hashlib.sha256(blob).hexdigest()[:16]
        if h != kv.get("src_sha"):
            return None
        return int(float(kv["bytes_per_input_row"]) * (N_LEFT + N_RIGHT))
    return None


# ---------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return  # the CPU oracle runs once, on rank 0
    import oracle
    oracle.build()
    n = args.ref_sample
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(n, n, FRAC, seed=SEED + 1000)
    for _ in range(args.warmup):
        oracle_step([lk, lp], [rk, rp], P)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m = oracle_step([lk, lp], [rk, rp], P)
    dt = (time.perf_counter() - t0) / args.steps
    assert m == math.floor(FRAC * n)
    value = 2 * n / dt
    sample = (f"{n} x {n} rows per step of the same generator (seed {SEED + 1000}), P={P}: stable partition "
              f"of both sides + sort-merge per partition, single thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get(
            "WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_left": N_LEFT, "n_right": N_RIGHT, "P": P, "match_fraction": FRAC,
                   "sample_rows_per_side": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mdj", choices=["mdj", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--latency-calls", type=int, default=300,
                    help="timed calls of the 1M x 1M, P=1 merge (p50/p99 latency)")
    ap.add_argument("--cpu-sample", type=int, default=10_000_000)
    ap.add_argument("--ref-sample", type=int, default=2_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=256,
                    help="pairs of the batched-vs-plain section (0 skips it)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the served section (0 skips it)")
    ap.add_argument("--serve-batch-rows", type=int, default=80_000_000,
                    help="input rows per continuous-batching group at most (larger requests run alone)")
    ap.add_argument("--serve-pool", type=int, default=32, help="distinct table pairs the requests draw from")
    ap.add_argument("--multikey-steps", type=int, default=3,
                    help="timed calls of the two-key-column section (0 skips it)")
    ap.add_argument("--host-budget-mib", type=int, default=1024,
                    help="device budget of the host-tables section in MiB (0 skips it)")
    ap.add_argument("--transpose-steps", type=int, default=10,
                    help="timed calls per size of the transpose-sum section (0 skips it)")
    ap.add_argument("--stream-windows", type=int, default=6,
                    help="windows of the streamed-output section (0 skips it)")
    ap.add_argument("--stream-left", type=int, default=50_000_000,
                    help="left rows of the streamed-output section (right = 4x); smaller values are for "
                         "profiling captures only")
    ap.add_argument("--rows", type=int, default=None,
                    help="rows per side (default 100M); smaller values are for profiling captures only")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mdj":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.rows:
        global N_LEFT, N_RIGHT, WORKLOAD
        N_LEFT = N_RIGHT = args.rows
        WORKLOAD = WORKLOAD.replace("100M x 100M", f"{args.rows} x {args.rows}")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
