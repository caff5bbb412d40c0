"""Continuous-batching merge server (asyncio).

Requests (a left and a right table of device-resident columns plus a
partition count P) arrive at any time.  The scheduler keeps them in a FIFO;
whenever one of `slots` workers is free it admits the oldest pending requests
that fit free device memory (a footprint estimate per request, checked
against torch.cuda.mem_get_info minus what admitted work has reserved),
groups compatible ones (same key and payload dtypes) up to a row budget, and
hands the group to the worker: the group's tables are packed into one
segmented table per side on the worker's own CUDA stream and merged with one
mdj_merge_batch call (every request shuffled into its own P partitions, all
partitions of all requests joined by one persistent kernel).  Each request's
future then receives its slice of the output, with row ids relative to its
own tables.  Work of different slots overlaps on the device; requests that
arrive while others run are admitted as soon as a slot and memory free up.

Nothing blocks the event loop: the blocking library calls run in the slot's
worker thread, which completes each request's asyncio future from outside the
loop (call_soon_threadsafe) and wakes the scheduler.  (The paper's send/recv
coroutines reach the same end by polling, Sec. IV-B, Listings 2 and 3; with
thousands of requests outstanding a wake-up costs less than a poll each.)
"""
from __future__ import annotations

import asyncio
import concurrent.futures
import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch

from . import mdj


@dataclass(eq=False)  # identity: requests hold tensors, so no field-wise ==
class Request:
    left: Sequence[torch.Tensor]
    right: Sequence[torch.Tensor]
    P: int
    arrival: float = 0.0
    done: float = 0.0
    result: Optional[mdj.JoinResult] = None
    error: Optional[BaseException] = None
    _future: Optional[asyncio.Future] = field(default=None, repr=False)

    @property
    def rows(self) -> int:
        return int(self.left[0].numel() + self.right[0].numel())

    @property
    def cls(self):
        return tuple(c.dtype for c in self.left) + ("|",) + tuple(c.dtype for c in self.right)

    def footprint(self) -> int:
        """Device bytes the merge may hold: packed inputs, two shuffled copies
        with row ids, and an output buffer of max(n_L, n_R) rows."""
        nl, nr = self.left[0].numel(), self.right[0].numel()
        lw = sum(c.element_size() for c in self.left)
        rw = sum(c.element_size() for c in self.right)
        out_w = self.left[0].element_size() + 8 + (lw - self.left[0].element_size()) + \
            (rw - self.right[0].element_size())
        return int(nl * (lw + 2 * (lw + 4)) + nr * (rw + 2 * (rw + 4)) + max(nl, nr) * out_w + (1 << 20))


class MergeServer:
    """Admits, batches and runs merge requests; see the module docstring."""

    def __init__(self, device: torch.device, slots: int = 2, max_batch_rows: int = 80_000_000,
                 max_batch_requests: int = 64, memory_reserve: int = 8 << 30, memory_budget: Optional[int] = None,
                 batching: bool = True):
        self.device = device
        self.slots = slots
        self.max_batch_rows = max_batch_rows
        self.max_batch_requests = max_batch_requests if batching else 1
        self.memory_reserve = memory_reserve
        self.memory_budget = memory_budget
        self.pending: deque = deque()
        self.reserved = 0
        self.free_slots = slots
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=slots)
        self.streams = [torch.cuda.Stream(device) for _ in range(slots)]
        self._slot_ids = list(range(slots))
        self.completed: List[Request] = []
        self._wake: Optional[asyncio.Event] = None
        self._loop: Optional[asyncio.AbstractEventLoop] = None
        self.rejected = 0
        self.group_sizes: List[int] = []
        self.peak_reserved = 0

    # ----------------------------------------------------------------- API
    async def submit(self, left: Sequence[torch.Tensor], right: Sequence[torch.Tensor], P: int) -> Request:
        """Queue a merge; returns the finished Request (result or error)."""
        req = Request(list(left), list(right), int(P), arrival=time.perf_counter())
        if req.footprint() > self._budget():
            req.error = MemoryError("request does not fit device memory even alone")
            req.done = time.perf_counter()
            self.rejected += 1
            return req
        req._future = asyncio.get_running_loop().create_future()
        self.pending.append(req)
        self._poke()
        return await req._future

    async def serve(self, stop: asyncio.Event):
        """The scheduler coroutine: runs until `stop` is set and all work drained."""
        self._wake = asyncio.Event()
        self._loop = loop = asyncio.get_running_loop()
        inflight = []
        stop_waiter = asyncio.ensure_future(stop.wait())
        while True:
            self._wake.clear()
            try:
                self._dispatch(loop, inflight)
            except Exception as e:  # noqa: BLE001 - fail what is queued, keep serving
                while self.pending:
                    self._complete(self.pending.popleft(), error=e)
            inflight = [f for f in inflight if not f.done()]
            if stop.is_set() and not self.pending and not inflight:
                break
            wake = asyncio.ensure_future(self._wake.wait())
            await asyncio.wait([wake, stop_waiter] + inflight, return_when=asyncio.FIRST_COMPLETED)
            wake.cancel()
        stop_waiter.cancel()

    # -------------------------------------------------------------- internals
    def _poke(self):
        if self._wake is not None:
            self._wake.set()

    def _budget(self) -> int:
        if self.memory_budget is not None:
            return self.memory_budget
        free, _total = torch.cuda.mem_get_info(self.device)
        # blocks torch has cached but not handed out are free to the merge too
        # (its allocations go through torch's allocator)
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return max(free + max(cached, 0) - self.memory_reserve, 0)

    def _dispatch(self, loop, inflight):
        while self.free_slots > 0 and self.pending:
            budget = self._budget() - self.reserved
            group, rows, need = [], 0, 0
            cls = self.pending[0].cls
            # oldest first; stop at the first request that does not fit
            for req in list(self.pending):
                if req.cls != cls:
                    continue
                if group and (len(group) >= self.max_batch_requests or rows + req.rows > self.max_batch_rows):
                    break
                fp = req.footprint()
                if need + fp > budget:
                    break
                group.append(req)
                rows += req.rows
                need += fp
            if not group:
                if self.reserved == 0 and self.free_slots == self.slots:
                    # nothing runs that could free memory: the oldest request
                    # would wait forever, so it fails instead
                    self._complete(self.pending.popleft(),
                                   error=MemoryError("request does not fit the device memory left free"))
                    self.rejected += 1
                    continue
                return  # memory frees up when running work completes
            for req in group:
                self.pending.remove(req)
            self.reserved += need
            self.peak_reserved = max(self.peak_reserved, self.reserved)
            self.group_sizes.append(len(group))
            self.free_slots -= 1
            slot = self._slot_ids.pop()
            fut = loop.run_in_executor(self.pool, self._run_group, group, slot)
            fut.add_done_callback(lambda f, need=need, slot=slot: self._finish(need, slot))
            inflight.append(fut)

    def _complete(self, req: Request, error: Optional[BaseException] = None):
        req.error = error
        req.done = time.perf_counter()
        self.completed.append(req)
        if req._future is not None and not req._future.done():
            req._future.set_result(req)

    def _finish(self, need: int, slot: int):
        self.reserved -= need
        self.free_slots += 1
        self._slot_ids.append(slot)
        self._poke()

    def _run_group(self, group: List[Request], slot: int):
        stream = self.streams[slot]
        try:
            with torch.cuda.device(self.device), torch.cuda.stream(stream):
                outs = self._merge_group(group)
            stream.synchronize()
            for req, res in zip(group, outs):
                req.result = res
        except BaseException as e:  # noqa: BLE001 - reported per request
            for req in group:
                req.error = e
        now = time.perf_counter()
        for req in group:
            req.done = now
            self.completed.append(req)
            self._loop.call_soon_threadsafe(req._future.set_result, req)

    def _merge_group(self, group: List[Request]) -> List[mdj.JoinResult]:
        dev = self.device
        if len(group) == 1:
            r = group[0]
            return [mdj.mdj_merge(r.left, r.right, r.P)]
        lo, ro = [0], [0]
        for r in group:
            lo.append(lo[-1] + r.left[0].numel())
            ro.append(ro[-1] + r.right[0].numel())
        L = [torch.empty(lo[-1], dtype=c.dtype, device=dev) for c in group[0].left]
        R = [torch.empty(ro[-1], dtype=c.dtype, device=dev) for c in group[0].right]
        for i, r in enumerate(group):
            for j, c in enumerate(r.left):
                L[j][lo[i]:lo[i + 1]].copy_(c, non_blocking=True)
            for j, c in enumerate(r.right):
                R[j][ro[i]:ro[i + 1]].copy_(c, non_blocking=True)
        res, off = mdj.mdj_merge_batch(L, R, lo, ro, [r.P for r in group])
        outs = []
        for i, r in enumerate(group):
            a, b = off[i], off[i + 1]
            outs.append(mdj.JoinResult(
                nrows=b - a, key=res.key[a:b],
                left_row=(res.left_row[a:b].view(torch.int32) - lo[i]).view(torch.uint32),
                right_row=(res.right_row[a:b].view(torch.int32) - ro[i]).view(torch.uint32),
                left_cols=[c[a:b] for c in res.left_cols], right_cols=[c[a:b] for c in res.right_cols]))
        return outs


# ------------------------------------------------------------------ drivers

def latency_stats(reqs: List[Request]) -> dict:
    lat = sorted((r.done - r.arrival) * 1e3 for r in reqs if r.error is None)
    if not lat:
        return {"p50_ms": None, "p99_ms": None, "n": 0}

    def pct(q):
        k = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[k]
    return {"p50_ms": round(pct(0.50), 3), "p99_ms": round(pct(0.99), 3), "mean_ms": round(sum(lat) / len(lat), 3),
            "n": len(lat)}


async def run_poisson(server: MergeServer, workload, arrivals, consume=None):
    """Submit workload[i] (left, right, P) at time arrivals[i] (seconds from
    start); returns (requests, wall seconds).  `consume(req)`, if given, is
    called as each request finishes (a client reading its result; it may drop
    req.result so the device memory is released)."""
    stop = asyncio.Event()
    sched = asyncio.ensure_future(server.serve(stop))
    t0 = time.perf_counter()

    async def one(i):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            await asyncio.sleep(delay)
        left, right, P = workload[i]
        req = await server.submit(left, right, P)
        if consume is not None:
            consume(req)
        return req

    reqs = await asyncio.gather(*[one(i) for i in range(len(workload))])
    wall = time.perf_counter() - t0
    stop.set()
    await sched
    return list(reqs), wall
