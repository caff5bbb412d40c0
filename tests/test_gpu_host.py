"""Host-resident tables larger than a device budget (mdj_merge_host through
the C ABI) against the oracle.

The smallest budget (64 MiB) makes tables of a few million rows take 16
buckets, several phase-1 chunks and several windows per bucket; every join
type is compared row for row after the canonical sort.
"""
import numpy as np
import pytest

import oracle
from paper_2101_08878_gb300 import datagen
from joinhelp import assert_same_result, gpu_result_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BUDGET = 64 << 20


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _host(cols):
    return [torch.from_numpy(np.ascontiguousarray(c)) for c in cols]


def _check(left, right, P, how, lk=0, rk=0, budget=BUDGET):
    want = oracle.merge_table_how(left, right, how, lk, rk)
    total, got = _mdj().merge_host_chunked(_host(left), _host(right), P, budget, how, lk, rk)
    assert total == want["key"].size == got.nrows
    if total:
        assert_same_result(gpu_result_np(got), want)
    return total


@pytest.mark.parametrize("how", ["inner", "left", "right", "outer"])
def test_host_tables_beyond_the_budget(how):
    left, right = datagen.match_fraction_tables(3_000_000, 3_000_000, 0.3, seed=51)
    total = _check(list(left), list(right), 8, how)
    if how == "inner":
        assert total == 900_000


@pytest.mark.parametrize("memcpy", ["0", "1"])
def test_host_copy_paths_and_unaligned_columns(monkeypatch, memcpy):
    # copy kernels (device access to pageable memory) or cudaMemcpyAsync; the
    # input columns start 4 bytes past a 16-byte boundary, and the 6 and 5
    # phase-1 chunks of the two sides cycle both copy-back buffer sets
    monkeypatch.setenv("MDJ_TEST_HOST_MEMCPY", memcpy)
    (lk, lp), (rk, rp) = datagen.random_tables(3_000_001, 2_500_001, 4_000_000, seed=55, key_dtype=np.int32,
                                               pay_dtype=np.float32)
    left, right = [lk[1:], lp[1:]], [rk[1:], rp[1:]]
    assert all(c.ctypes.data % 16 == 4 for c in left + right)
    _check(left, right, 8, "inner")


@pytest.mark.parametrize("kd", [np.int64, np.int32])
def test_host_tables_that_fit_copy_right_while_left_partitions(kd):
    # a budget that holds both tables: one bucket, the right table copied in
    # on its own stream while the left side is partitioned
    (lk, lp), (rk, rp) = datagen.random_tables(2_000_000, 3_000_000, 2_500_000, seed=56, key_dtype=kd,
                                               pay_dtype=np.float64)
    extra = np.arange(rk.size, dtype=np.int32) * 3
    _check([lk, lp], [rp, rk, extra], 8, "inner", lk=0, rk=1, budget=1 << 30)


@pytest.mark.parametrize("how", ["inner", "outer"])
def test_host_heavy_key_spans_many_windows(how):
    rng = np.random.default_rng(52)
    lk = np.concatenate([np.full(300_000, 9), rng.integers(0, 2_000_000, 1_000_000)]).astype(np.int64)
    rk = np.concatenate([np.full(40, 9), rng.integers(1_000_000, 3_000_000, 1_000_000)]).astype(np.int64)
    lk, rk = lk[rng.permutation(lk.size)], rk[rng.permutation(rk.size)]
    total = _check([lk, rng.random(lk.size)], [rk, rng.random(rk.size)], 8, how)
    assert total > 12_000_000


def test_host_int32_keys_several_columns():
    (lk, lp), (rk, rp) = datagen.random_tables(1_500_000, 2_000_000, 3_000_000, seed=53, key_dtype=np.int32,
                                               pay_dtype=np.float32)
    lx = np.arange(lk.size, dtype=np.int64) * 7
    _check([lk, lp, lx], [rp, rk], 4, "left", lk=0, rk=1)


def test_host_empty_and_sink_abort():
    mdj = _mdj()
    left, right = datagen.match_fraction_tables(1000, 1000, 0.3, seed=54)
    empty = [c[:0] for c in right]
    total, got = mdj.merge_host_chunked(_host(left), _host(empty), 8, BUDGET, "inner")
    assert total == 0 and got.nrows == 0
    total, got = mdj.merge_host_chunked(_host(left), _host(empty), 8, BUDGET, "left")
    assert total == 1000 and bool((got.right_row == torch.tensor(mdj.NO_ROW, dtype=torch.uint32)).all())

    def stop(first_row, piece):
        raise RuntimeError("sink stops")
    with pytest.raises(RuntimeError, match="sink stops"):
        mdj.merge_host_chunked(_host(left), _host(right), 8, BUDGET, "inner", on_piece=stop)
