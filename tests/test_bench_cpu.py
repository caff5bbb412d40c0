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
