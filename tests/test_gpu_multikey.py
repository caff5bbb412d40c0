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
