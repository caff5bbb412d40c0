"""mdj_join_batch: many independent partition-pair joins in one call.

Each pair's slice of the output is compared with the oracle's merge of that
pair's two slices (row ids shifted by the slice starts); the config-3 shape
(256 pairs, sizes log-uniform in [1K, 4M] per side, match fraction U[0.1,0.9])
is checked at full size by the per-pair closed-form row count plus the oracle
on a sample of pairs.
"""
import math

import numpy as np
import pytest

import oracle
from joinhelp import bits
from paper_2101_08878_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _concat(pairs):
    lk = np.concatenate([p[0][0] for p in pairs])
    lp = np.concatenate([p[0][1] for p in pairs])
    rk = np.concatenate([p[1][0] for p in pairs])
    rp = np.concatenate([p[1][1] for p in pairs])
    lo = np.concatenate([[0], np.cumsum([p[0][0].size for p in pairs])]).astype(np.uint64)
    ro = np.concatenate([[0], np.cumsum([p[1][0].size for p in pairs])]).astype(np.uint64)
    return (lk, lp), (rk, rp), lo, ro


def _np(t):
    return t.detach().cpu().numpy()


def _check_pair(res_np, po, i, pair, lo, ro):
    (lk, lp), (rk, rp) = pair
    a, b = po[i], po[i + 1]
    key = res_np["key"][a:b]
    lrow = res_np["left_row"][a:b].astype(np.int64) - int(lo[i])
    rrow = res_np["right_row"][a:b].astype(np.int64) - int(ro[i])
    assert np.all((lrow >= 0) & (lrow < lk.size)) and np.all((rrow >= 0) & (rrow < rk.size))
    order = np.lexsort((rrow, lrow, key))
    want = oracle.merge_table([lk, lp], [rk, rp])
    assert np.array_equal(key[order], want["key"])
    assert np.array_equal(lrow[order].astype(np.uint32), want["left_row"])
    assert np.array_equal(rrow[order].astype(np.uint32), want["right_row"])
    assert np.array_equal(bits(res_np["lpay"][a:b][order]), bits(want["left_cols"][0]))
    assert np.array_equal(bits(res_np["rpay"][a:b][order]), bits(want["right_cols"][0]))


def _run_batch(pairs, **kw):
    (lk, lp), (rk, rp), lo, ro = _concat(pairs)
    mdj = _mdj()
    res, po = mdj.mdj_join_batch([torch.from_numpy(lk).to(DEV), torch.from_numpy(lp).to(DEV)],
                                 [torch.from_numpy(rk).to(DEV), torch.from_numpy(rp).to(DEV)], lo, ro, **kw)
    torch.cuda.synchronize()
    res_np = {"key": _np(res.key), "left_row": _np(res.left_row).view(np.uint32),
              "right_row": _np(res.right_row).view(np.uint32), "lpay": _np(res.left_cols[0]),
              "rpay": _np(res.right_cols[0])}
    return res, res_np, po, lo, ro


def _ragged_pairs(seed):
    rng = np.random.default_rng(seed)
    pairs = []
    for i in range(40):
        nl, nr = int(rng.integers(0, 30_000)), int(rng.integers(0, 30_000))
        if i % 7 == 0:
            nl = 0
        if i % 11 == 0:
            nr = 0
        kr = int(rng.choice([50, 5_000, 10**9]))
        pairs.append(datagen.random_tables(nl, nr, kr, seed=seed * 100 + i))
    return pairs


@pytest.mark.parametrize("seed", [1, 2])
def test_batch_ragged_pairs_match_oracle(seed):
    pairs = _ragged_pairs(seed)
    res, res_np, po, lo, ro = _run_batch(pairs)
    assert po[0] == 0 and po[-1] == res.nrows and all(po[i] <= po[i + 1] for i in range(len(pairs)))
    for i, pair in enumerate(pairs):
        _check_pair(res_np, po, i, pair, lo, ro)


def test_batch_pair_ranges_are_fixed_and_survive_a_small_item_bound(monkeypatch):
    # two-pass ordered output: item offsets from a scan of counted items, so
    # every pair's range is the same in every run (rows within a pair follow
    # the unstable segmented scatter); a bound of one item forces the rerun
    # with exact arrays and must give the same ranges and rows
    pairs = _ragged_pairs(3)
    _, a_np, po_a, lo, ro = _run_batch(pairs)
    _, b_np, po_b, _, _ = _run_batch(pairs)
    monkeypatch.setenv("MDJ_TEST_ITEM_BOUND", "1")
    _, c_np, po_c, _, _ = _run_batch(pairs)
    assert list(po_a) == list(po_b) == list(po_c)
    for res_np, po in ((a_np, po_a), (b_np, po_b), (c_np, po_c)):
        for i, pair in enumerate(pairs):
            _check_pair(res_np, po, i, pair, lo, ro)


def test_batch_int32_keys_and_float32_payloads():
    # the 4-byte key and payload instantiations of the count and exact passes
    rng = np.random.default_rng(12)
    pairs = []
    for i in range(24):
        nl, nr = int(rng.integers(1, 40_000)), int(rng.integers(1, 40_000))
        pairs.append(datagen.random_tables(nl, nr, int(rng.choice([40, 20_000, 10**9])), seed=700 + i,
                                           key_dtype=np.int32, pay_dtype=np.float32))
    res, res_np, po, lo, ro = _run_batch(pairs)
    assert res.key.dtype == torch.int32 and res.left_cols[0].dtype == torch.float32
    for i, pair in enumerate(pairs):
        _check_pair(res_np, po, i, pair, lo, ro)


@pytest.mark.parametrize("table_rows,fill_pct", [(1024, 50), (2048, 85), (8192, 95), (8192, 30)])
def test_batch_tuning_does_not_change_rows(table_rows, fill_pct):
    pairs = [datagen.match_fraction_tables(n, 2 * n, 0.5, seed=n) for n in (100, 5_000, 60_000, 150_000)]
    res, res_np, po, lo, ro = _run_batch(pairs, table_rows=table_rows, fill_pct=fill_pct)
    for i, pair in enumerate(pairs):
        assert po[i + 1] - po[i] == math.floor(0.5 * 2 * pair[0][0].size)
        _check_pair(res_np, po, i, pair, lo, ro)


def test_batch_invalid_arguments():
    mdj = _mdj()
    k = torch.arange(10, device=DEV)
    with pytest.raises(mdj.MdjError):
        mdj.mdj_join_batch([k], [k], [0, 5, 9], [0, 5, 10])      # last offset != rows
    with pytest.raises(mdj.MdjError):
        mdj.mdj_join_batch([k], [k], [0, 6, 5, 10], [0, 5, 5, 10])  # decreasing
    with pytest.raises(mdj.MdjError):
        mdj.mdj_join_batch([k], [k], [0, 10], [0, 10], table_rows=100)
    with pytest.raises(mdj.MdjError):
        mdj.mdj_join_batch([k], [k], [0, 10], [0, 10], table_rows=16384)


@pytest.mark.slow
def test_batch_256_pairs_full_size():
    # 256 pairs, n_L, n_R log-uniform in [1K, 4M], match fraction U[0.1, 0.9]
    pairs = datagen.batch_pairs(256, 1_000, 4_000_000, seed=3)
    res, res_np, po, lo, ro = _run_batch(pairs)
    rng = np.random.default_rng(0)
    for i, ((lk, _), (rk, _)) in enumerate(pairs):
        # unique left keys: each right row meets at most one left row, and the
        # generator makes exactly floor(f * n_R) of them match
        n_match = int(np.count_nonzero(rk < lk.size))
        assert po[i + 1] - po[i] == n_match
    for i in rng.choice(len(pairs), 6, replace=False):
        _check_pair(res_np, po, int(i), pairs[int(i)], lo, ro)


def _run_merge_batch(pairs, P, **kw):
    (lk, lp), (rk, rp), lo, ro = _concat(pairs)
    mdj = _mdj()
    res, po = mdj.mdj_merge_batch([torch.from_numpy(lk).to(DEV), torch.from_numpy(lp).to(DEV)],
                                  [torch.from_numpy(rk).to(DEV), torch.from_numpy(rp).to(DEV)], lo, ro, P, **kw)
    torch.cuda.synchronize()
    res_np = {"key": _np(res.key), "left_row": _np(res.left_row).view(np.uint32),
              "right_row": _np(res.right_row).view(np.uint32), "lpay": _np(res.left_cols[0]),
              "rpay": _np(res.right_cols[0])}
    return res, res_np, po, lo, ro


def test_merge_batch_mixed_partition_counts_match_oracle():
    pairs = _ragged_pairs(3)
    P = [(1, 8, 32, 3, 1024)[i % 5] for i in range(len(pairs))]
    res, res_np, po, lo, ro = _run_merge_batch(pairs, P)
    for i, pair in enumerate(pairs):
        _check_pair(res_np, po, i, pair, lo, ro)


def test_merge_batch_larger_requests():
    pairs = [datagen.match_fraction_tables(n, n, 0.3, seed=n) for n in (300_000, 1_500_000, 40_000)]
    res, res_np, po, lo, ro = _run_merge_batch(pairs, [8, 32, 1])
    for i, pair in enumerate(pairs):
        assert po[i + 1] - po[i] == math.floor(0.3 * pair[1][0].size)
        _check_pair(res_np, po, i, pair, lo, ro)


def test_merge_batch_rejects_bad_P():
    mdj = _mdj()
    k = torch.arange(10, device=DEV)
    for bad in ([0], [1025]):
        with pytest.raises(mdj.MdjError):
            mdj.mdj_merge_batch([k], [k], [0, 10], [0, 10], bad)


@pytest.mark.parametrize("jt", [256, 512])
def test_join_block_shapes_give_the_same_rows(jt):
    # the tuner's block-shape knob: 256- and 512-thread join blocks (2048 and
    # 4096 probe rows per item) give the same rows per pair as one join per pair
    pairs = [datagen.match_fraction_tables(n, m, 0.4, seed=n) for n, m in ((3_000, 9_000), (50_000, 20_000),
                                                                           (7_000, 70_000))]
    (lk, lp), (rk, rp), lo, ro = _concat(pairs)
    mdj = _mdj()
    L = [torch.from_numpy(lk).to(DEV), torch.from_numpy(lp).to(DEV)]
    R = [torch.from_numpy(rk).to(DEV), torch.from_numpy(rp).to(DEV)]
    res, po = mdj.mdj_join_batch(L, R, lo, ro, 0, 0, 2048, 60, jt)
    for i, ((a, b), (c, d)) in enumerate(pairs):
        want = oracle.merge_table([a, b], [c, d])
        assert po[i + 1] - po[i] == want["key"].size
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_join_batch(L, R, lo, ro, 0, 0, 0, 0, 384)
    assert e.value.status == -1


def test_tuner_picks_and_caches(tmp_path):
    from paper_2101_08878_gb300.tuner import BatchTuner
    pairs = [datagen.match_fraction_tables(n, n, 0.5, seed=n) for n in (20_000, 80_000)]
    (lk, lp), (rk, rp), lo, ro = _concat(pairs)
    L = [torch.from_numpy(lk).to(DEV), torch.from_numpy(lp).to(DEV)]
    R = [torch.from_numpy(rk).to(DEV), torch.from_numpy(rp).to(DEV)]
    path = str(tmp_path / "tuner.json")
    t = BatchTuner(path)
    assert t.lookup(L[0].dtype, int(lo[-1]), 2) is None
    best = t.choose(L, R, lo, ro)
    assert best[0] in (2048, 4096, 8192) and best[1] in (60, 75, 85, 95) and best[2] in (256, 512)
    again = BatchTuner(path)  # reloaded from the cache file
    assert again.lookup(L[0].dtype, int(lo[-1]), 2) == best
    assert again.choose(L, R, lo, ro, search=False) == best
