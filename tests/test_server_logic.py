"""Scheduling logic of the merge server on the CPU, with the GPU calls faked:
continuous batching groups compatible requests, admission waits for memory,
oversized requests are rejected, and a failing merge fails only its group."""
import asyncio
import contextlib
import time
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture
def fake_gpu(monkeypatch):
    from paper_2101_08878_gb300 import mdj
    calls = {"merge": 0, "batch": []}
    monkeypatch.setattr(torch.cuda, "Stream", lambda dev=None: types.SimpleNamespace(synchronize=lambda: None))
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "device", lambda d: contextlib.nullcontext())
    calls["free"] = 64 << 30
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda d=None: (calls["free"], 128 << 30))
    calls["cached"] = 2 << 30
    monkeypatch.setattr(torch.cuda, "memory_reserved", lambda d=None: (1 << 30) + calls["cached"])
    monkeypatch.setattr(torch.cuda, "memory_allocated", lambda d=None: 1 << 30)

    def merge(l, r, P):
        time.sleep(0.002)
        calls["merge"] += 1
        if P == 13:
            raise RuntimeError("injected failure")
        n = min(l[0].numel(), r[0].numel())
        return mdj.JoinResult(n, l[0][:n], l[0][:n], l[0][:n], [], [])

    def batch(L, R, lo, ro, P, *a, **k):
        time.sleep(0.004)
        calls["batch"].append(len(P))
        if 13 in P:
            raise RuntimeError("injected failure")
        sizes = [min(lo[i + 1] - lo[i], ro[i + 1] - ro[i]) for i in range(len(P))]
        off = np.concatenate([[0], np.cumsum(sizes)]).tolist()
        key = torch.zeros(off[-1], dtype=L[0].dtype)
        rows = torch.zeros(off[-1], dtype=torch.int32).view(torch.uint32)
        return mdj.JoinResult(off[-1], key, rows, rows, [], []), off

    monkeypatch.setattr(mdj, "mdj_merge", merge)
    monkeypatch.setattr(mdj, "mdj_merge_batch", batch)
    return calls


def _work(n, seed, P=8):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nl, nr = int(rng.integers(1000, 5000)), int(rng.integers(1000, 5000))
        kd = torch.int32 if i % 3 == 0 else torch.int64
        out.append(([torch.zeros(nl, dtype=kd), torch.zeros(nl)], [torch.zeros(nr, dtype=kd), torch.zeros(nr)], P))
    return out


def _serve(server, work, arrivals):
    from paper_2101_08878_gb300.server import run_poisson
    return asyncio.run(asyncio.wait_for(run_poisson(server, work, arrivals), 30))


def test_continuous_batching_groups_by_dtype(fake_gpu):
    from paper_2101_08878_gb300.server import MergeServer
    work = _work(30, 1)
    server = MergeServer(torch.device("cpu"), slots=2)
    reqs, _ = _serve(server, work, np.zeros(len(work)))
    assert all(r.error is None for r in reqs)
    assert sum(server.group_sizes) == len(work) and max(server.group_sizes) > 1
    for r, (l, rt, _) in zip(reqs, work):
        assert r.result.nrows == min(l[0].numel(), rt[0].numel())
        assert r.result.key.dtype == l[0].dtype  # never mixed across dtype classes


def test_admission_waits_for_memory(fake_gpu):
    from paper_2101_08878_gb300.server import MergeServer, Request
    work = _work(8, 2)
    biggest = max(Request(*w).footprint() for w in work)
    budget = int(biggest * 1.2)
    server = MergeServer(torch.device("cpu"), slots=2, memory_budget=budget)
    reqs, _ = _serve(server, work, np.zeros(len(work)))
    assert all(r.error is None for r in reqs)
    assert 0 < server.peak_reserved <= budget  # admitted work never exceeds the budget
    assert len(server.group_sizes) > 1


def test_oversized_request_is_rejected(fake_gpu):
    from paper_2101_08878_gb300.server import MergeServer
    server = MergeServer(torch.device("cpu"), slots=1, memory_budget=1 << 10)
    reqs, _ = _serve(server, _work(2, 3), [0.0, 0.0])
    assert all(isinstance(r.error, MemoryError) for r in reqs) and server.rejected == 2


def test_budget_counts_torch_cached_blocks(fake_gpu):
    from paper_2101_08878_gb300.server import MergeServer
    server = MergeServer(torch.device("cpu"), slots=1, memory_reserve=8 << 30)
    assert server._budget() == (64 << 30) + (2 << 30) - (8 << 30)


def test_no_wait_forever_when_memory_is_held_elsewhere(fake_gpu):
    # free memory drops below every request's footprint while the queue still
    # holds work and nothing runs (results kept by the client): the queued
    # requests fail with MemoryError instead of waiting for memory that no
    # running merge will release
    from paper_2101_08878_gb300 import mdj
    from paper_2101_08878_gb300.server import MergeServer
    real = mdj.mdj_merge

    def hog(l, r, P):
        fake_gpu["free"] = fake_gpu["cached"] = 0
        return real(l, r, P)
    mdj.mdj_merge = hog
    server = MergeServer(torch.device("cpu"), slots=1, batching=False, memory_reserve=0)
    reqs, _ = _serve(server, _work(4, 5), [0.0] * 4)
    assert reqs[0].error is None and reqs[0].result is not None
    assert all(isinstance(r.error, MemoryError) for r in reqs[1:]) and server.rejected == 3


def test_consumer_sees_every_request_once(fake_gpu):
    from paper_2101_08878_gb300.server import MergeServer, run_poisson
    seen = []

    def consume(req):
        seen.append(req.result.nrows)
        req.result = None  # a client that drops its result after reading it
    work = _work(12, 6)
    server = MergeServer(torch.device("cpu"), slots=2)
    reqs, _ = asyncio.run(asyncio.wait_for(run_poisson(server, work, np.zeros(len(work)), consume), 30))
    assert sorted(seen) == sorted(min(l[0].numel(), r[0].numel()) for l, r, _ in work)
    assert all(r.result is None and r.error is None for r in reqs)


def test_failure_is_confined_to_its_group(fake_gpu):
    from paper_2101_08878_gb300.server import MergeServer
    good = _work(6, 4)
    bad = _work(1, 5, P=13)
    work = good[:3] + bad + good[3:]
    server = MergeServer(torch.device("cpu"), slots=1, batching=False)
    reqs, _ = _serve(server, work, np.arange(len(work)) * 0.01)
    assert isinstance(reqs[3].error, RuntimeError)
    assert all(r.error is None for i, r in enumerate(reqs) if i != 3)


def test_latency_stats():
    from paper_2101_08878_gb300.server import Request, latency_stats
    reqs = []
    for i in range(100):
        r = Request([], [], 1, arrival=0.0, done=(i + 1) / 1000)
        reqs.append(r)
    st = latency_stats(reqs)
    assert st["n"] == 100 and st["p50_ms"] == pytest.approx(50.5, abs=1) and st["p99_ms"] == pytest.approx(99, abs=1.5)
