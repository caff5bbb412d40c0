"""The merge on several key columns (mdj_merge_multi through the C ABI)
against the oracle: the same (left_row, right_row) pairs, and every output
column equal to its source row's bits.  With MDJ_TEST_WEAK_TUPLE_HASH=1 the
surrogate is the first key column alone, so distinct tuples collide and the
verification must remove the false pairs."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _run_and_check(left, right, lkeys, rkeys, P):
    mdj = _mdj()
    res = mdj.mdj_merge_multi([torch.from_numpy(c).to(DEV) for c in left],
                              [torch.from_numpy(c).to(DEV) for c in right], lkeys, rkeys, P)
    torch.cuda.synchronize()
    want_l, want_r = oracle.merge_multi(left, right, lkeys, rkeys)
    lrow = res.left_row.cpu().numpy().view(np.uint32).astype(np.int64)
    rrow = res.right_row.cpu().numpy().view(np.uint32).astype(np.int64)
    order = np.lexsort((rrow, lrow))
    assert res.nrows == want_l.size
    assert np.array_equal(lrow[order], want_l) and np.array_equal(rrow[order], want_r)
    bits = (lambda a: a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64))
    lorder = list(lkeys) + [j for j in range(len(left)) if j not in lkeys]
    rorder = [j for j in range(len(right)) if j not in rkeys]
    assert len(res.left_cols) == len(lorder) and len(res.right_cols) == len(rorder)
    for got, j in zip(res.left_cols, lorder):
        assert np.array_equal(bits(got.cpu().numpy()), bits(left[j][lrow]))
    for got, j in zip(res.right_cols, rorder):
        assert np.array_equal(bits(got.cpu().numpy()), bits(right[j][rrow]))
    return res.nrows


def _tables(seed, n_l, n_r):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 300, n_l).astype(np.int32)
    b = rng.integers(0, 50, n_l).astype(np.int64)
    c = rng.integers(0, 2**32, n_l, dtype=np.uint64).astype(np.uint32) % 7
    ra = rng.integers(0, 300, n_r).astype(np.int32)
    rb = rng.integers(0, 50, n_r).astype(np.int64)
    rc = rng.integers(0, 2**32, n_r, dtype=np.uint64).astype(np.uint32) % 7
    return rng, (a, b, c), (ra, rb, rc)


@pytest.mark.parametrize("P", [1, 8])
def test_two_keys(P):
    rng, (a, b, _), (ra, rb, _) = _tables(71, 60_000, 80_000)
    left = [a, b, rng.random(a.size)]
    right = [rng.random(ra.size), rb, ra]
    assert _run_and_check(left, right, [0, 1], [2, 1], P) > 0


def test_three_keys_mixed_types():
    rng, (a, b, c), (ra, rb, rc) = _tables(72, 50_000, 50_000)
    left = [rng.random(a.size).astype(np.float32), c, a, b]
    right = [rb, ra, rc, rng.integers(0, 9, ra.size).astype(np.int64)]
    _run_and_check(left, right, [2, 3, 1], [1, 0, 2], 8)


def test_colliding_surrogates_are_removed(monkeypatch):
    monkeypatch.setenv("MDJ_TEST_WEAK_TUPLE_HASH", "1")
    rng, (a, b, _), (ra, rb, _) = _tables(73, 40_000, 40_000)
    # every left row shares its first key column with ~130 right rows but
    # matches few of them on the pair
    n = _run_and_check([a, b, rng.random(a.size)], [ra, rb, rng.random(ra.size)], [0, 1], [0, 1], 8)
    assert 0 < n < 40_000 * 40_000 // 300


def test_no_match_and_empty():
    a = np.arange(1000, dtype=np.int64)
    b = np.zeros(1000, np.int64)
    assert _run_and_check([a, b], [a, b + 1], [0, 1], [0, 1], 4) == 0
    assert _run_and_check([a[:0], b[:0]], [a, b], [0, 1], [0, 1], 4) == 0


# ------------------------------------------------------ outer joins on tuples

def _run_how(left, right, lkeys, rkeys, P, how):
    mdj = _mdj()
    res = mdj.mdj_merge_multi([torch.from_numpy(c).to(DEV) for c in left],
                              [torch.from_numpy(c).to(DEV) for c in right], lkeys, rkeys, P, how=how)
    torch.cuda.synchronize()
    want = oracle.merge_multi_how(left, right, lkeys, rkeys, how)
    assert res.nrows == want["left_row"].size
    lrow = res.left_row.cpu().numpy().view(np.uint32)
    rrow = res.right_row.cpu().numpy().view(np.uint32)
    order = np.lexsort((rrow, lrow))
    assert np.array_equal(lrow[order], want["left_row"]) and np.array_equal(rrow[order], want["right_row"])
    bits = (lambda a: a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64))
    assert len(res.left_cols) == len(want["left_cols"]) and len(res.right_cols) == len(want["right_cols"])
    for got, w in zip(res.left_cols, want["left_cols"]):
        assert np.array_equal(bits(got.cpu().numpy())[order], bits(w))
    for got, w in zip(res.right_cols, want["right_cols"]):
        assert np.array_equal(bits(got.cpu().numpy())[order], bits(w))
    return res.nrows


@pytest.mark.parametrize("how", ["left", "right", "outer"])
@pytest.mark.parametrize("P", [1, 8])
def test_outer_joins_on_two_keys(how, P):
    rng, (a, b, _), (ra, rb, _) = _tables(74, 60_000, 80_000)
    left = [a, b, rng.random(a.size)]
    right = [rng.random(ra.size), rb, ra]
    inner = _run_and_check(left, right, [0, 1], [2, 1], P)
    assert _run_how(left, right, [0, 1], [2, 1], P, how) > inner


@pytest.mark.parametrize("how", ["left", "right", "outer"])
def test_outer_joins_on_three_keys_mixed_types(how):
    rng, (a, b, c), (ra, rb, rc) = _tables(75, 30_000, 50_000)
    left = [rng.random(a.size).astype(np.float32), c, a, b]
    right = [rb, ra, rc, rng.integers(0, 9, ra.size).astype(np.int64)]
    _run_how(left, right, [2, 3, 1], [1, 0, 2], 8, how)


@pytest.mark.parametrize("how", ["left", "outer"])
def test_outer_rows_whose_only_candidates_collide(monkeypatch, how):
    # with the weak surrogate a left row can have candidates but no true
    # partner: it must come out unmatched, once
    monkeypatch.setenv("MDJ_TEST_WEAK_TUPLE_HASH", "1")
    rng, (a, b, _), (ra, rb, _) = _tables(76, 20_000, 20_000)
    _run_how([a, b, rng.random(a.size)], [ra, rb + 40, rng.random(ra.size)], [0, 1], [0, 1], 8, how)


@pytest.mark.parametrize("how", ["left", "right", "outer"])
def test_outer_on_tuples_with_empty_or_unmatched_sides(how):
    a = np.arange(1000, dtype=np.int64)
    b = np.zeros(1000, np.int64)
    assert _run_how([a, b], [a, b + 1], [0, 1], [0, 1], 4, how) == (2000 if how == "outer" else 1000)
    n = _run_how([a[:0], b[:0]], [a, b], [0, 1], [0, 1], 4, how)
    assert n == (0 if how == "left" else 1000)
