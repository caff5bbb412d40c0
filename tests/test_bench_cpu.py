"""bench.py's CPU legs: the oracle step on a thread pool does the same work
as the single-threaded step, and the CPU baseline reports both."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2101_08878_gb300 import datagen  # noqa: E402


def test_threaded_oracle_step_counts_the_same_rows():
    oracle.build()
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(200_000, 150_000, 0.3, seed=5)
    one = bench.oracle_step([lk, lp], [rk, rp], 8)
    many = bench.oracle_step([lk, lp], [rk, rp], 8, threads=4)
    assert one == many == 45_000


def test_cpu_baseline_reports_single_and_all_cores():
    b = bench.cpu_baseline(100_000)
    assert b["kind"] == "oracle" and b["cores"] == 1 and b["value"] > 0
    assert b["all_cores"]["cores"] >= 1 and b["all_cores"]["value"] > 0


def test_result_fingerprint_numpy_and_torch_agree():
    # the served check compares device fingerprints with the oracle's host
    # ones: both must be the same function of the rows (any row order)
    import numpy as np
    import torch

    import bench
    from paper_2101_08878_gb300.mdj import JoinResult

    rng = np.random.default_rng(3)
    n = 5000
    for kd, pd in ((np.int64, np.float64), (np.int32, np.float32)):
        key = rng.integers(-2**31, 2**31 - 1, n).astype(kd)
        lrow = rng.integers(0, 2**32 - 1, n, dtype=np.uint64).astype(np.uint32)
        rrow = rng.integers(0, 2**32 - 1, n, dtype=np.uint64).astype(np.uint32)
        lpay = rng.random(n).astype(pd)
        rpay = rng.random(n).astype(pd)
        want = bench.fingerprint_np(key, lrow, rrow, lpay, rpay)
        perm = rng.permutation(n)
        res = JoinResult(n, torch.from_numpy(key[perm]), torch.from_numpy(lrow[perm].view(np.int32)).view(torch.uint32),
                         torch.from_numpy(rrow[perm].view(np.int32)).view(torch.uint32),
                         [torch.from_numpy(lpay[perm])], [torch.from_numpy(rpay[perm])])
        got = int(bench.fingerprint_torch(res)[0]) & ((1 << 64) - 1)
        assert want == (n, got)
        # one flipped payload bit changes it
        lpay2 = lpay.copy()
        lpay2.view(np.uint32 if pd == np.float32 else np.uint64)[7] ^= 1
        assert bench.fingerprint_np(key, lrow, rrow, lpay2, rpay) != want
