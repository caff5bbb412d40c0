"""mdj_join / mdj_merge / mdj_count_checksum against the oracle, bit for bit
after the canonical sort by (key, left_row, right_row)."""
import math

import numpy as np
import pytest

import oracle
from joinhelp import assert_same_result, gpu_result_np
from paper_2101_08878_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
I64_MIN, I64_MAX = np.iinfo(np.int64).min, np.iinfo(np.int64).max


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _dev(cols):
    return [torch.from_numpy(np.ascontiguousarray(c)).to(DEV) for c in cols]


def _run(left, right, P=None, lk=0, rk=0):
    mdj = _mdj()
    if P is None:
        res = mdj.mdj_join(_dev(left), _dev(right), lk, rk)
    else:
        res = mdj.mdj_merge(_dev(left), _dev(right), P, lk, rk)
    torch.cuda.synchronize()
    return gpu_result_np(res)


def _check(left, right, P=None, lk=0, rk=0):
    got = _run(left, right, P, lk, rk)
    want = oracle.merge_table(left, right, lk, rk)
    assert_same_result(got, want)
    return got


# ------------------------------------------------------------- small / edge

@pytest.mark.parametrize("P", [None, 1, 8])
@pytest.mark.parametrize("nl,nr", [(0, 0), (0, 100), (100, 0), (1, 1), (7, 5)])
def test_empty_and_tiny(P, nl, nr):
    (lk, lp), (rk, rp) = datagen.random_tables(nl, nr, 4, seed=nl * 31 + nr)
    _check([lk, lp], [rk, rp], P)


@pytest.mark.parametrize("P", [None, 1, 8, 64])
@pytest.mark.parametrize("key_range", [3, 100, 10_000, 10**9])
def test_duplicates(P, key_range):
    (lk, lp), (rk, rp) = datagen.random_tables(3000, 5000, key_range, seed=key_range)
    _check([lk, lp], [rk, rp], P)


@pytest.mark.parametrize("P", [None, 8, 1000, 1024, 2000])
def test_match_fraction_several_buckets(P):
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(200_000, 300_000, 0.3, seed=7)
    got = _check([lk, lp], [rk, rp], P)
    assert got["key"].size == math.floor(0.3 * 300_000)


def test_int32_keys_f32_payloads_multi_column():
    rng = np.random.default_rng(3)
    (lk, lp), (rk, rp) = datagen.random_tables(40_000, 60_000, 20_000, seed=3, key_dtype=np.int32,
                                               pay_dtype=np.float32)
    l_extra = rng.integers(0, 2**63 - 1, lk.size, dtype=np.int64)
    r_extra = rng.integers(-2**31, 2**31 - 1, rk.size).astype(np.int32)
    # key in the middle of the left table, last on the right
    left = [lp, lk, l_extra]
    right = [rp, r_extra, rk]
    _check(left, right, None, 1, 2)
    _check(left, right, 32, 1, 2)


def test_extreme_keys_and_nan_payloads():
    rng = np.random.default_rng(4)
    ext = np.array([I64_MIN, I64_MAX, 0, -1, I64_MIN + 1, I64_MAX - 1], np.int64)
    lk = rng.choice(ext, 3000)
    rk = rng.choice(ext, 2000)
    lp = datagen.uniform_payload(rng, lk.size)
    rp = datagen.uniform_payload(rng, rk.size)
    lp.view(np.uint64)[::3] = np.uint64(0x7FF8000000000001)
    rp.view(np.uint64)[::5] = np.uint64(0xFFF0DEADBEEF0000)
    _check([lk, lp], [rk, rp], None)
    _check([lk, lp], [rk, rp], 8)


def test_heavy_key_exceeding_one_table():
    # one key repeated more times than one shared-memory table holds: the
    # bucket is split into several build chunks
    rng = np.random.default_rng(5)
    lk = np.concatenate([np.full(20_000, 42, np.int64), rng.integers(0, 10**6, 5000)])
    rk = np.concatenate([np.full(300, 42, np.int64), rng.integers(0, 10**6, 5000)])
    rng.shuffle(lk)
    rng.shuffle(rk)
    got = _check([lk, datagen.uniform_payload(rng, lk.size)], [rk, datagen.uniform_payload(rng, rk.size)], 4)
    assert got["key"].size >= 20_000 * 300


def test_P_invariance():
    (lk, lp), (rk, rp) = datagen.zipf_tables(12_000, 20_000, 20_000, 1.1, seed=6)
    base = _run([lk, lp], [rk, rp], None)
    for P in (1, 3, 8, 64, 1025):
        got = _run([lk, lp], [rk, rp], P)
        assert_same_result(got, base)


def test_two_level_plan():
    # enough build rows that the plan needs a second partition pass
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(4_000_000, 2_000_000, 0.3, seed=8)
    got = _check([lk, lp], [rk, rp], 8)
    assert got["key"].size == math.floor(0.3 * 2_000_000)


def test_two_level_plan_stable_passes(monkeypatch):
    # the stable partition passes (MDJ_STABLE_SHUFFLE=1) give the same result
    monkeypatch.setenv("MDJ_STABLE_SHUFFLE", "1")
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(4_000_000, 2_000_000, 0.3, seed=8)
    got = _check([lk, lp], [rk, rp], 8)
    assert got["key"].size == math.floor(0.3 * 2_000_000)


@pytest.mark.parametrize("kd,pd", [(np.int32, np.float32), (np.int64, np.float32), (np.int32, np.float64)])
def test_two_level_plan_dtypes_and_duplicates(kd, pd):
    # 5M build rows: more sub-buckets than one pass can make, so two passes
    rng = np.random.default_rng(17)
    n = 5_000_000
    lk = rng.integers(0, 2_000_000, n).astype(kd)
    rk = rng.integers(0, 4_000_000, n // 2).astype(kd)
    lp = datagen.uniform_payload(rng, n, pd)
    rp = datagen.uniform_payload(rng, n // 2, pd)
    _check([lk, lp], [rk, rp], 8)


def test_plain_merge_1M_P1():
    # plain inner merge, P = 1: 1M x 1M, unique left keys, match fraction 0.3
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(1_000_000, 1_000_000, 0.3, seed=0)
    got = _check([lk, lp], [rk, rp], 1)
    assert got["key"].size == 300_000


def test_deterministic_for_unique_left(monkeypatch):
    # ordered output mode: item ranges follow item order (decoupled look-back)
    monkeypatch.setenv("MDJ_ORDERED_OUTPUT", "1")
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(100_000, 100_000, 0.5, seed=9)
    mdj = _mdj()
    a = mdj.mdj_merge(_dev([lk, lp]), _dev([rk, rp]), 8)
    b = mdj.mdj_merge(_dev([lk, lp]), _dev([rk, rp]), 8)
    assert torch.equal(a.key, b.key) and torch.equal(a.left_row, b.left_row)
    assert torch.equal(a.right_row, b.right_row)


# ---------------------------------------------------------- count/checksum

@pytest.mark.parametrize("P", [1, 8, 64])
@pytest.mark.parametrize("pay", [np.float64, np.float32])
def test_count_checksum(P, pay):
    (lk, lp), (rk, rp) = datagen.zipf_tables(40_000, 80_000, 3_000, 1.1, seed=P, pay_dtype=pay)
    mdj = _mdj()
    got = mdj.mdj_count_checksum(_dev([lk, lp]), _dev([rk, rp]), P)
    assert got == oracle.count_checksum(lk, lp, rk, rp)


def test_count_checksum_key_only_tables():
    (lk, _), (rk, _) = datagen.random_tables(5000, 7000, 300, seed=12)
    mdj = _mdj()
    got = mdj.mdj_count_checksum(_dev([lk]), _dev([rk]), 8)
    # no payload column: payload bits are 0 on both sides
    want = oracle.count_checksum(lk, np.zeros(lk.size, np.uint64), rk, np.zeros(rk.size, np.uint64))
    assert got == want


# ------------------------------------------------------------------ errors

def test_invalid_arguments():
    mdj = _mdj()
    k64 = torch.arange(10, device=DEV)
    k32 = k64.int()
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_merge([k64], [k32], 8)  # key dtype mismatch
    assert e.value.status == -1
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_merge([k64], [k64], 0)
    assert e.value.status == -1
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_merge([k64], [k64], 8, 1, 0)  # key column out of range
    assert e.value.status == -1
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_join([k64.float()], [k64.float()])
    assert e.value.status == -2


@pytest.mark.parametrize("ordered", ["0", "1"])
def test_output_buffer_overflow_takes_exact_pass(monkeypatch, ordered):
    # an optimistic buffer smaller than the join forces the exact second pass
    # at the item offsets the first pass recorded (atomic or looked-back)
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(50_000, 70_000, 0.5, seed=21)
    monkeypatch.setenv("MDJ_OUTPUT_ROWS", "1000")
    monkeypatch.setenv("MDJ_ORDERED_OUTPUT", ordered)
    got = _check([lk, lp], [rk, rp], 8)
    assert got["key"].size == 35_000


@pytest.mark.parametrize("ordered", ["0", "1"])
def test_item_count_above_bound_reruns_exactly(monkeypatch, ordered):
    # the join's descriptor arrays are sized without reading its item count;
    # a bound of one item forces the rerun with exact arrays
    monkeypatch.setenv("MDJ_TEST_ITEM_BOUND", "1")
    monkeypatch.setenv("MDJ_ORDERED_OUTPUT", ordered)
    (lk, lp), (rk, rp) = datagen.zipf_tables(30_000, 50_000, 40_000, 1.1, seed=24)
    _check([lk, lp], [rk, rp], 8)


def test_bounded_wait_reports_timeout_and_context_survives(monkeypatch):
    # item 0 withholds its count (test hook): every look-back wait must give up
    # after its bound, the call must say so, and the next call must work
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(100_000, 100_000, 0.3, seed=22)
    mdj = _mdj()
    monkeypatch.setenv("MDJ_ORDERED_OUTPUT", "1")
    monkeypatch.setenv("MDJ_TEST_WITHHOLD_FIRST_ITEM", "1")
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_merge(_dev([lk, lp]), _dev([rk, rp]), 8)
    assert e.value.status == -6
    monkeypatch.delenv("MDJ_TEST_WITHHOLD_FIRST_ITEM")
    _check([lk, lp], [rk, rp], 8)


@pytest.mark.parametrize("ordered", ["0", "1"])
def test_both_output_modes_match_oracle(monkeypatch, ordered):
    monkeypatch.setenv("MDJ_ORDERED_OUTPUT", ordered)
    (lk, lp), (rk, rp) = datagen.zipf_tables(20_000, 30_000, 50_000, 1.1, seed=23)
    _check([lk, lp], [rk, rp], 8)


def test_merge_host_end_to_end():
    # host (pinned) tables in, host result out: same rows as the device merge
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(700_000, 900_000, 0.4, seed=21)
    mdj = _mdj()
    hl = [torch.from_numpy(lk).pin_memory(), torch.from_numpy(lp).pin_memory()]
    hr = [torch.from_numpy(rk).pin_memory(), torch.from_numpy(rp).pin_memory()]
    out, h2d, d2h = mdj.merge_host(hl, hr, 8)
    assert h2d == 16 * (700_000 + 900_000)
    assert out.nrows == math.floor(0.4 * 900_000) and not out.key.is_cuda
    assert d2h == out.nrows * (8 + 4 + 4 + 8 + 8)
    dev = mdj.mdj_merge(_dev([lk, lp]), _dev([rk, rp]), 8)
    a = torch.sort((out.key << 32) | out.right_row.view(torch.int32).to(torch.int64)).values
    b = torch.sort(((dev.key << 32) | dev.right_row.view(torch.int32).to(torch.int64)).cpu()).values
    assert torch.equal(a, b)
