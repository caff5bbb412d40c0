"""The N > 1 bench path on the CPU: replicas on world_size 2 over gloo.

On a GPU machine every rank merges its own tables; the job's time is the slowest
rank's (all_reduce MAX) and the job's rate counts every rank's rows.  Here the
same helpers run in two gloo processes with chosen local times, and the
reference arm's non-zero rank exits without doing work.
"""
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
local = [0.75, 2.5][rank]
slowest = bench.max_over_ranks(local, dist, "cpu")
rate = bench.whole_job_rate(200, world, slowest)
print(f"RESULT {{rank}} {{slowest}} {{rate}}", flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_over_ranks_and_job_rate_gloo():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err
    got = sorted(tuple(ln.split()[1:]) for out, _ in outs for ln in out.splitlines() if ln.startswith("RESULT"))
    assert [g[0] for g in got] == ["0", "1"]
    for _, slowest, rate in got:
        assert float(slowest) == 2.5             # both ranks see the slowest replica's time
        assert float(rate) == 200 * 2 / 2.5      # every rank's rows over that time


def test_single_rank_helpers_need_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
