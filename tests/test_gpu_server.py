"""The continuous-batching server: every request's rows are the same alone
and in the mix; admission waits for memory and rejects what never fits."""
import asyncio

import numpy as np
import pytest

from paper_2101_08878_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _canon(res):
    key = res.key.detach().cpu().numpy().astype(np.int64)
    lrow = res.left_row.detach().cpu().numpy().view(np.uint32)
    rrow = res.right_row.detach().cpu().numpy().view(np.uint32)
    order = np.lexsort((rrow, lrow, key))
    cols = [c.detach().cpu().numpy() for c in list(res.left_cols) + list(res.right_cols)]
    return key[order], lrow[order], rrow[order], [c.view(np.uint8).reshape(c.size, -1)[order] for c in cols]


def _workload(n, seed):
    rng = np.random.default_rng(seed)
    work = []
    for i in range(n):
        nl = int(np.exp(rng.uniform(np.log(1e4), np.log(3e5))))
        nr = int(np.exp(rng.uniform(np.log(1e4), np.log(3e5))))
        kd = np.int32 if rng.random() < 0.5 else np.int64
        pd = np.float32 if rng.random() < 0.5 else np.float64
        (lk, lp), (rk, rp) = datagen.match_fraction_tables(nl, nr, 0.3, seed=seed * 1000 + i, key_dtype=kd,
                                                           pay_dtype=pd)
        P = int(rng.choice([1, 8, 32]))
        work.append(([torch.from_numpy(lk).to(DEV), torch.from_numpy(lp).to(DEV)],
                     [torch.from_numpy(rk).to(DEV), torch.from_numpy(rp).to(DEV)], P))
    return work


def _same(a, b):
    assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3]))
    assert len(a[3]) == len(b[3]) and all(np.array_equal(x, y) for x, y in zip(a[3], b[3]))


def test_results_identical_alone_and_in_the_mix():
    from paper_2101_08878_gb300 import mdj
    from paper_2101_08878_gb300.server import MergeServer, latency_stats, run_poisson
    work = _workload(24, seed=4)
    alone = [_canon(mdj.mdj_merge(l, r, P)) for l, r, P in work]
    rng = np.random.default_rng(7)
    arrivals = np.cumsum(rng.exponential(0.0005, len(work)))
    server = MergeServer(DEV, slots=2)
    reqs, wall = asyncio.run(asyncio.wait_for(run_poisson(server, work, arrivals), 120))
    assert all(r.error is None for r in reqs), [r.error for r in reqs if r.error]
    for r, want in zip(reqs, alone):
        _same(_canon(r.result), want)
    assert max(server.group_sizes) > 1  # some requests were batched together
    st = latency_stats(reqs)
    assert st["n"] == len(work) and st["p50_ms"] <= st["p99_ms"]


def test_served_stream_matches_oracle():
    # the served request stream at reduced scale: 120 requests (P, key and payload widths
    # drawn per request) arriving faster than one slot can serve, so groups
    # form; every served result equals the oracle's merge row for row
    import oracle
    from joinhelp import assert_same_result, gpu_result_np
    from paper_2101_08878_gb300.server import MergeServer, run_poisson
    work = _workload(120, seed=11)
    host = [([c.cpu().numpy() for c in l], [c.cpu().numpy() for c in r]) for l, r, _ in work]
    arrivals = np.cumsum(np.random.default_rng(12).exponential(0.0002, len(work)))
    server = MergeServer(DEV, slots=2)
    reqs, _ = asyncio.run(asyncio.wait_for(run_poisson(server, work, arrivals), 300))
    assert all(r.error is None for r in reqs), [r.error for r in reqs if r.error]
    assert sum(server.group_sizes) == len(work) and max(server.group_sizes) > 1
    for req, (hl, hr) in zip(reqs, host):
        assert_same_result(gpu_result_np(req.result), oracle.merge_table(hl, hr))


def test_admission_waits_for_memory_and_rejects_oversized():
    from paper_2101_08878_gb300.server import MergeServer, run_poisson
    work = _workload(6, seed=5)
    one = max(MergeServerFootprint(w) for w in work)
    # room for about one request at a time: all are served, and admitted work
    # never holds more than the budget
    budget = int(one * 1.05)
    server = MergeServer(DEV, slots=2, memory_budget=budget)
    reqs, _ = asyncio.run(asyncio.wait_for(run_poisson(server, work, np.zeros(len(work))), 120))
    assert all(r.error is None for r in reqs)
    assert 0 < server.peak_reserved <= budget
    # a request bigger than the whole budget is rejected, not queued forever
    small = MergeServer(DEV, slots=1, memory_budget=1 << 20)
    reqs, _ = asyncio.run(asyncio.wait_for(run_poisson(small, work[:1], [0.0]), 120))
    assert isinstance(reqs[0].error, MemoryError) and small.rejected == 1


def MergeServerFootprint(w):
    from paper_2101_08878_gb300.server import Request
    return Request(w[0], w[1], w[2]).footprint()
