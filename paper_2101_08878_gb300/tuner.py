"""Autotuner for batched joins: picks the shared-memory table size, the
target bucket fill (which together set every pair's sub-bucket count) and
the join block shape by timing mdj_join_batch on the caller's own batch, and
caches the winner per size class (key dtype, total build rows, pair count,
each rounded to a power of two) in a JSON file.

The search space is small and explicit: table rows in {2048, 4096, 8192}
(shared memory per block and blocks per SM follow from it), fill in
{60, 75, 85, 95} percent, and join blocks of 256 or 512 threads (2048 or
4096 probe rows per work item).  Every candidate gives the same rows; only
the time differs.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Optional, Sequence, Tuple

import torch

from . import mdj

TABLE_ROWS = (2048, 4096, 8192)
FILL_PCT = (60, 75, 85, 95)
JOIN_THREADS = (256, 512)
DEFAULT = (4096, 85, 512)


def _default_cache_path() -> str:
    env = os.environ.get("MDJ_TUNER_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "mdj", "tuner.json")


def size_class(key_dtype: torch.dtype, build_rows: int, npairs: int) -> str:
    r = max(int(build_rows), 1)
    p = max(int(npairs), 1)
    return f"{str(key_dtype).replace('torch.', '')}:rows2^{round(math.log2(r))}:pairs2^{round(math.log2(p))}"


class BatchTuner:
    """Chooses (table_rows, fill_pct, join_threads) for mdj_join_batch per size class."""

    def __init__(self, cache_path: Optional[str] = None):
        self.path = cache_path or _default_cache_path()
        self._lock = threading.Lock()
        self.cache = {}
        try:
            with open(self.path) as f:
                self.cache = json.load(f)
        except (OSError, ValueError):
            self.cache = {}

    def _save(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except OSError:
            pass  # a read-only cache location only costs a re-tune next time

    def lookup(self, key_dtype, build_rows: int, npairs: int) -> Optional[Tuple[int, int, int]]:
        hit = self.cache.get(size_class(key_dtype, build_rows, npairs))
        if not hit or "join_threads" not in hit:  # entries of an older search space are re-tuned
            return None
        return (int(hit["table_rows"]), int(hit["fill_pct"]), int(hit["join_threads"]))

    def tune(self, left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], left_offsets,
             right_offsets, left_key: int = 0, right_key: int = 0, repeats: int = 2) -> Tuple[int, int, int]:
        """Time every candidate on this batch (after one warm-up call each) and
        cache the fastest for the batch's size class."""
        cls = size_class(left_cols[left_key].dtype, int(left_offsets[-1]), len(left_offsets) - 1)
        dev = left_cols[0].device
        stream = torch.cuda.current_stream(dev)
        results = {}
        for tr in TABLE_ROWS:
            for fp in FILL_PCT:
                for jt in JOIN_THREADS:
                    res, _ = mdj.mdj_join_batch(left_cols, right_cols, left_offsets, right_offsets, left_key,
                                                right_key, tr, fp, jt)
                    del res
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(repeats):
                        res, _ = mdj.mdj_join_batch(left_cols, right_cols, left_offsets, right_offsets, left_key,
                                                    right_key, tr, fp, jt)
                        del res
                    e1.record(stream)
                    e1.synchronize()
                    results[(tr, fp, jt)] = e0.elapsed_time(e1) / repeats
        best = min(results, key=results.get)
        with self._lock:
            self.cache[cls] = {"table_rows": best[0], "fill_pct": best[1], "join_threads": best[2],
                               "ms": round(results[best], 4),
                               "candidates": {f"{k[0]}/{k[1]}/{k[2]}": round(v, 4) for k, v in results.items()}}
            self._save()
        return best

    def choose(self, left_cols, right_cols, left_offsets, right_offsets, left_key: int = 0, right_key: int = 0,
               search: bool = True) -> Tuple[int, int, int]:
        """Cached choice for this batch's size class; tunes on a miss when
        `search`, else returns the defaults."""
        hit = self.lookup(left_cols[left_key].dtype, int(left_offsets[-1]), len(left_offsets) - 1)
        if hit:
            return hit
        if not search:
            return DEFAULT
        return self.tune(left_cols, right_cols, left_offsets, right_offsets, left_key, right_key)
