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


def alg_bytes_per_launch(kernel: str, n_side: int, n_left: int, n_right: int, m: int):
    """Bytes the method must move in one launch of `kernel` (8-byte keys and
    payloads, 4-byte row ids); None for kernels outside the model."""
    per_side = {
        "hist": KEY,                                       # read keys
        "shuffle_pass1": (KEY + PAY) + (KEY + PAY + RID),  # read row, write row + row id
        "shuffle_pass2": (KEY + PAY + RID) * 2,            # second level: read + write row and row id
        "scatter_stable": (KEY + PAY) + (KEY + PAY + RID),  # the stable passes (MDJ_STABLE_SHUFFLE=1)
        "scatter_reserve": (KEY + PAY + RID) * 2,
    }
    if kernel in per_side:
        return per_side[kernel] * n_side
    if kernel in ("join_write", "join_write_exact"):
        return (KEY + PAY + RID) * (n_left + n_right) + OUT_ROW * m  # read both sides, write the rows
    return None


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
    mdj.profile_reset()
    mdj.profile_enable(True)
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
    mdj.profile_enable(False)
    prof = mdj.profile_collect()
    ms_total = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_step = ms_total / args.steps
    value = whole_job_rate(N_LEFT + N_RIGHT, world, ms_step / 1e3)

    # ---- roofline: dominant kernel by total device time inside the timed region
    peak, peak_kind = peaks()
    launches = sum(v[0] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launches, dom_ms) = dom
    per_launch_ms = dom_ms / max(dom_launches, 1)
    alg = alg_bytes_per_launch(dom_name, N_LEFT, N_LEFT, N_RIGHT, m_expect)
    achieved = alg / (per_launch_ms / 1e3) / 1e9 if alg else None
    traffic = measured_traffic(dom_name)
    b_alg_step = 64 * (N_LEFT + N_RIGHT) + OUT_ROW * m_expect
    roofline = {
        "bound": "hbm", "kernel": dom_name, "achieved": round(achieved, 1) if achieved else None,
        "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4) if achieved else None,
        "traffic": traffic, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
        else "fallback 6800 GB/s", "launch_ms": round(per_launch_ms, 4),
        "alg_bytes_per_launch": alg,
    }
    step_roof = {"alg_bytes": b_alg_step, "achieved_gbs": round(b_alg_step / (ms_step / 1e3) / 1e9, 1),
                 "frac": round(b_alg_step / (ms_step / 1e3) / 1e9 / peak, 4)}
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

    # ---- end to end: host (pinned) inputs -> device -> merge -> host result
    e2e = None
    if args.e2e_steps > 0:
        hl = [torch.from_numpy(lk).pin_memory(), torch.from_numpy(lp).pin_memory()]
        hr = [torch.from_numpy(rk).pin_memory(), torch.from_numpy(rp).pin_memory()]
        del left[:], right[:]
        torch.cuda.empty_cache()
        out, h2d, d2h = mdj.merge_host(hl, hr, P)  # warm
        del out
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            out, h2d, d2h = mdj.merge_host(hl, hr, P)
            assert out.nrows == m_expect
            del out
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist, dev)
        e2e = {"value": whole_job_rate(N_LEFT + N_RIGHT, world, dt), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": round(dt * 1e3, 3), "steps": args.e2e_steps}

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
        "e2e": e2e, "clocks": clk.summary(),
    }
    if host_tables is not None:
        line["host_tables"] = host_tables
    if multi_key is not None:
        line["multi_key"] = multi_key
    if args.stream_windows > 0:
        torch.cuda.empty_cache()
        line["streamed"] = streamed_section(args, dev)
        line["streamed"]["plain_workload_one_window"] = stream_plain
    if args.transpose_steps > 0:
        torch.cuda.empty_cache()
        line["transpose_sum"] = transpose_section(args, dev)
    if args.batch_pairs > 0:
        line["batched"] = batched_section(args, dev)
    if args.serve_requests > 0:
        torch.cuda.empty_cache()
        line["served"] = served_section(args, dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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
    chunked hash partition into host buckets, then one stream per bucket pair,
    each window handed to a sink that counts rows (nothing is kept).  Wall
    time of one call after one warm-up call on a 1/10 sample."""
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
    seen[0] = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    total, _ = mdj.merge_host_chunked(L, R, P, budget, on_piece=count, device=dev)
    wall = time.perf_counter() - t0
    assert total == seen[0] == m_expect, (total, seen[0])
    in_bytes = sum(c.numel() * c.element_size() for c in L + R)
    return {"workload": "the bench tables in pageable host memory, inner merge, sink counts rows",
            "device_budget_bytes": budget, "input_bytes": in_bytes, "rows": total, "wall_s": round(wall, 3),
            "value": (len(L[0]) + len(R[0])) / wall, "unit": "input rows/s"}


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
            "all_rows_estimate_s": round(m / rate, 1)}


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
    tr, fp = tuner.choose(L, R, lo, ro)
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
        res, po = mdj.mdj_join_batch(L, R, lo, ro, 0, 0, tr, fp)
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
                        "tuning": {"table_rows": tr, "fill_pct": fp}},
            "plain_per_pair": {"value": rows / (ms_p / 1e3), "unit": UNIT, "ms_per_batch": round(ms_p, 3)},
            "speedup": round(ms_p / ms_b, 3)}


def served_section(args, dev):
    """The served workload: Poisson arrivals of merge requests (P in {1, 8, 32}, n_L, n_R
    log-uniform in [1e4, 2e7], int32/int64 keys and float32/float64 payloads
    50/50, match fraction 0.3) over a device-resident pool of tables, served
    by MergeServer with continuous batching versus the plain per-request path
    (one slot, no batching), at 0.5x, 1x and 2x the plain path's capacity."""
    import asyncio
    import torch
    from paper_2101_08878_gb300.server import MergeServer, latency_stats, run_poisson

    rng = np.random.default_rng(4)
    pool, pool_out = [], []
    for i in range(args.serve_pool):
        nl = int(datagen.log_uniform_sizes(rng, 1, 10_000, 20_000_000)[0])
        nr = int(datagen.log_uniform_sizes(rng, 1, 10_000, 20_000_000)[0])
        kd = np.int32 if rng.random() < 0.5 else np.int64
        pd = np.float32 if rng.random() < 0.5 else np.float64
        (lk, lp), (rk, rp) = datagen.match_fraction_tables(nl, nr, FRAC, seed=4000 + i, key_dtype=kd, pay_dtype=pd)
        P = int(rng.choice([1, 8, 32]))
        pool_out.append(int(np.floor(FRAC * nr)))
        pool.append(([torch.from_numpy(lk).to(dev), torch.from_numpy(lp).to(dev)],
                     [torch.from_numpy(rk).to(dev), torch.from_numpy(rp).to(dev)], P))
    picks = rng.integers(0, len(pool), args.serve_requests)
    out_rows = []

    def consume(req):
        # the client reads its result and lets it go, as a caller of a server
        # would; keeping thousands of results would fill the device
        if req.result is not None:
            out_rows.append(req.result.nrows)
            req.result = None

    def run(rate, batching, slots, sel):
        work = [pool[int(i)] for i in sel]
        rows = sum(int(w[0][0].numel() + w[1][0].numel()) for w in work)
        # match fraction 0.3 of the right side: the closed-form output row count
        expect_rows = sum(pool_out[int(i)] for i in sel)
        server = MergeServer(dev, slots=slots, batching=batching, max_batch_rows=args.serve_batch_rows)
        arrivals = np.cumsum(np.random.default_rng(44).exponential(1.0 / rate, len(work)))
        out_rows.clear()
        reqs, wall = asyncio.run(asyncio.wait_for(run_poisson(server, work, arrivals, consume), 300))
        bad = [r.error for r in reqs if r.error is not None]
        if bad:
            raise RuntimeError(f"served requests failed: {bad[0]}")
        if sum(out_rows) != expect_rows:
            raise RuntimeError(f"served output rows {sum(out_rows)} != {expect_rows}")
        st = latency_stats(reqs)
        st["rows_per_s"] = rows / wall
        st["wall_s"] = round(wall, 3)
        st["mean_batch"] = round(float(np.mean(server.group_sizes)), 2)
        return st

    # first launches of each path's kernels (module loads, attribute setup)
    # stay out of the timed runs
    run(1e9, True, 2, picks[:100])
    run(1e9, False, 1, picks[:100])
    # capacity of the plain per-request path: everything queued at once
    cap = run(1e9, False, 1, picks)
    cap_rps = len(picks) / cap["wall_s"]
    out = {"workload": f"{len(picks)} requests drawn from {len(pool)} device-resident table pairs; P in {{1,8,32}}, "
                       f"n_L, n_R log-uniform [1e4, 2e7], int32/int64 keys, float32/float64 payloads, match 0.3",
           "served_config": {"slots": 2, "max_batch_rows": args.serve_batch_rows},
           "plain_config": {"slots": 1, "batching": False},
           "plain_capacity_requests_per_s": round(cap_rps, 2), "rates": []}
    for mult in (0.5, 1.0, 2.0):
        rate = mult * cap_rps
        out["rates"].append({"x_plain_capacity": mult, "requests_per_s": round(rate, 2),
                             "served": run(rate, True, 2, picks), "plain": run(rate, False, 1, picks)})
    return out


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if the
    kernel's source files (comma-separated, hashed together) are unchanged
    since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    src = os.path.join(ROOT, "paper_2101_08878_gb300", "csrc")
    try:
        rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    for r in rows:
        kv = dict(x.split("=", 1) for x in r if "=" in x)
        if kv.get("kernel") != kernel:
            continue
        blob = b"".join(open(os.path.join(src, f), "rb").read() for f in kv["file"].split(","))
        h = hashlib.sha256(blob).hexdigest()[:16]
        if h != kv.get("src_sha"):
            return None
        return int(float(kv["bytes_per_unit"]) * N_LEFT)
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
    ap.add_argument("--e2e-steps", type=int, default=3)
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
