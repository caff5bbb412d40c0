"""Streamed merge output (mdj_stream_* through the C ABI) against the oracle.

The stream writes the join of mdj_merge window by window into fixed buffers.
Every test joins the windows back together and compares them row for row with
the oracle's merge after the canonical sort by (key, left_row, right_row), so
a row that is lost, duplicated or written with the wrong partner fails.  The
cases cover heavy keys on the build side (grouped in global memory), heavy keys
on the probe side (probe chunks over several blocks), ragged windows, windows
out of order, re-emission, the resumable cursor, and empty sides.
"""
import numpy as np
import pytest

import oracle
from paper_2101_08878_gb300 import datagen
from joinhelp import assert_same_result, gpu_result_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _dev(cols):
    return [torch.from_numpy(np.ascontiguousarray(c)).to(DEV) for c in cols]


def _concat(parts, mdj):
    """Host JoinResult of windows (each already copied to the host)."""
    cat = (lambda xs: torch.cat(xs) if xs else None)
    return mdj.JoinResult(
        sum(p.nrows for p in parts), cat([p.key for p in parts]), cat([p.left_row for p in parts]),
        cat([p.right_row for p in parts]),
        [cat([p.left_cols[j] for p in parts]) for j in range(len(parts[0].left_cols))],
        [cat([p.right_cols[j] for p in parts]) for j in range(len(parts[0].right_cols))])


def _host(v, mdj):
    cp = (lambda t: t.cpu())
    return mdj.JoinResult(v.nrows, cp(v.key), cp(v.left_row), cp(v.right_row), [cp(t) for t in v.left_cols],
                          [cp(t) for t in v.right_cols])


def _stream_all(left, right, P, window, lk=0, rk=0, how="inner"):
    mdj = _mdj()
    with mdj.MergeStream(_dev(left), _dev(right), P, lk, rk, how) as st:
        parts = [_host(v, mdj) for _, v in st.windows(window)]
        total = st.total_rows
    torch.cuda.synchronize()
    if not parts:
        return total, None
    return total, _concat(parts, mdj)


def _check(left, right, P, window, lk=0, rk=0, how="inner"):
    want = oracle.merge_table_how(left, right, how, lk, rk)
    total, got = _stream_all(left, right, P, window, lk, rk, how)
    assert total == want["key"].size
    if total:
        assert_same_result(gpu_result_np(got), want)
    return total


@pytest.mark.parametrize("P", [1, 8, 64])
def test_stream_matches_oracle_unique_build_keys(P):
    left, right = datagen.match_fraction_tables(200_000, 300_000, 0.3, seed=31)
    assert _check(list(left), list(right), P, window=7_777) == 90_000


@pytest.mark.parametrize("P", [1, 8])
def test_stream_matches_oracle_duplicate_keys(P):
    # keys over a small range: groups of ~5 build rows, many-to-many
    left, right = datagen.random_tables(150_000, 120_000, 30_000, seed=32)
    _check(list(left), list(right), P, window=100_003)


def test_stream_small_build_side_unpartitioned():
    # P = 1 and a build side below one table: no shuffle, the inputs are read in place
    left, right = datagen.random_tables(3_000, 5_000, 2_000, seed=40)
    _check(list(left), list(right), 1, window=999)


def _skewed_tables(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    # build side: key 7 has 6000 rows (its sub-bucket outgrows a shared-memory
    # table), key 11 has 3; probe side: key 7 has 2000 rows, key 11 has
    # 150,000 (its sub-bucket's probe side spans three chunks)
    lk = np.concatenate([np.full(6000, 7), np.full(3, 11), rng.integers(1000, 30_000, 40_000)]).astype(np.int64)
    rk = np.concatenate([np.full(2000, 7), np.full(150_000, 11), rng.integers(1000, 40_000, 60_000)]).astype(np.int64)
    lk = lk[rng.permutation(lk.size)]
    rk = rk[rng.permutation(rk.size)]
    lp = datagen.uniform_payload(rng, lk.size)
    rp = datagen.uniform_payload(rng, rk.size)
    return [lk, lp], [rk, rp]


@pytest.mark.parametrize("P", [1, 8])
def test_stream_heavy_keys_both_sides(P):
    left, right = _skewed_tables(33)
    total = _check(left, right, P, window=1_000_003)
    assert total > 12_000_000 + 450_000


def test_stream_int32_keys_several_columns():
    (lk, lp), (rk, rp) = datagen.random_tables(60_000, 90_000, 50_000, seed=34, key_dtype=np.int32,
                                               pay_dtype=np.float32)
    rng = np.random.Generator(np.random.PCG64(35))
    lx = rng.integers(0, 2**62, lk.size, dtype=np.int64)
    ry = rng.integers(-2**31, 2**31 - 1, rk.size, dtype=np.int64).astype(np.int32)
    # key column not first on the right
    _check([lk, lp, lx], [rp, rk, ry], 8, window=4096, lk=0, rk=1)


def test_stream_windows_are_resumable_and_repeatable():
    mdj = _mdj()
    left, right = _skewed_tables(36)
    with mdj.MergeStream(_dev(left), _dev(right), 8) as st:
        n = st.total_rows
        a, b, c = 1234, n // 3 + 17, n - 5
        buf1 = st.buffers(c - a)
        whole = _host(st.emit(a, c - a, buf1), mdj)
        buf2 = st.buffers(c - a)
        part2 = _host(st.emit(b, c - b, buf2), mdj)   # later window first
        part1 = _host(st.emit(a, b - a, buf2), mdj)
        again = _host(st.emit(a, c - a, buf2), mdj)
        for name in ("key", "left_row", "right_row"):
            w = getattr(whole, name)
            assert torch.equal(torch.cat([getattr(part1, name), getattr(part2, name)]), w)
            assert torch.equal(getattr(again, name), w)
        assert torch.equal(again.left_cols[0].view(torch.int64), whole.left_cols[0].view(torch.int64))
        # the cursor: ragged last window, then nothing
        seen = 0
        cur = st.buffers(999_999)
        while True:
            first, v = st.next(cur)
            if v.nrows == 0:
                break
            assert first == seen
            seen += v.nrows
        assert seen == n
        # a zero-row window is a no-op; a window past the end is refused
        st.emit(n, 0, cur)
        with pytest.raises(mdj.MdjError) as e:
            st.emit(n - 1, 2, cur)
        assert e.value.status == -1


def test_stream_skips_null_columns():
    mdj = _mdj()
    left, right = datagen.match_fraction_tables(50_000, 50_000, 0.5, seed=37)
    with mdj.MergeStream(_dev(left), _dev(right), 4) as st:
        buf = st.buffers(st.total_rows)
        sentinel = torch.full_like(buf.left_cols[0].view(torch.int64), -7)
        buf.left_cols[0].view(torch.int64).copy_(sentinel)
        buf.key.fill_(-9)
        proj = mdj.JoinResult(buf.nrows, None, buf.left_row, buf.right_row, [None], buf.right_cols)
        st.emit(0, st.total_rows, proj)
        torch.cuda.synchronize()
        assert torch.equal(buf.left_cols[0].view(torch.int64), sentinel)
        assert bool((buf.key == -9).all())
        li = buf.left_row.view(torch.int32).to(torch.int64)
        ri = buf.right_row.view(torch.int32).to(torch.int64)
        L0, R0 = torch.from_numpy(left[0]).to(DEV), torch.from_numpy(right[0]).to(DEV)
        assert torch.equal(L0[li], R0[ri])


@pytest.mark.parametrize("nl,nr", [(0, 1000), (1000, 0), (0, 0)])
def test_stream_empty_side(nl, nr):
    left, right = datagen.match_fraction_tables(max(nl, 1), max(nr, 1), 0.3, seed=38)
    left = [c[:nl] for c in left]
    right = [c[:nr] for c in right]
    total, got = _stream_all(left, right, 8, 1000)
    assert total == 0 and got is None


def test_stream_no_matching_key():
    rng = np.random.Generator(np.random.PCG64(39))
    lk = rng.integers(0, 1000, 20_000).astype(np.int64)
    rk = rng.integers(5000, 6000, 30_000).astype(np.int64)
    total, _ = _stream_all([lk, lk.astype(np.float64)], [rk, rk.astype(np.float64)], 8, 100)
    assert total == 0


def test_stream_skewed_materialised_variant():
    # the Zipf(1.1) merge at 50K x 200K (about 2.0e8 rows) through a 16M-row buffer
    mdj = _mdj()
    (lk, lp), (rk, rp) = datagen.zipf_tables(50_000, 200_000, 10_000_000, 1.1, seed=2)
    L, R = _dev([lk, lp]), _dev([rk, rp])
    lrow, rrow = oracle.merge_pairs(lk, rk)
    want = (lk[lrow].astype(np.int64) << 34) | (lrow.astype(np.int64) << 18) | rrow.astype(np.int64)
    del lrow, rrow
    with mdj.MergeStream(L, R, 64) as st:
        assert st.total_rows == want.size
        packed = torch.empty(st.total_rows, dtype=torch.int64, device=DEV)
        for q0, v in st.windows(1 << 24):
            li = v.left_row.view(torch.int32).to(torch.int64)
            ri = v.right_row.view(torch.int32).to(torch.int64)
            assert torch.equal(v.key, L[0][li]) and torch.equal(v.key, R[0][ri])
            assert torch.equal(v.left_cols[0].view(torch.int64), L[1].view(torch.int64)[li])
            assert torch.equal(v.right_cols[0].view(torch.int64), R[1].view(torch.int64)[ri])
            packed[q0:q0 + v.nrows] = (v.key << 34) | (li << 18) | ri
    packed, _ = torch.sort(packed)
    assert torch.equal(packed, torch.from_numpy(want).to(DEV))


@pytest.mark.slow
def test_stream_skewed_full_size_windows():
    # the Zipf(1.1) merge at full size (50M x 200M, P = 64): about 2.0e14 rows,
    # so the count must equal the oracle's exactly and sampled windows (the
    # start, deep inside the heaviest groups, the end) must hold valid, distinct
    # pairs with their source rows' payload bits
    mdj = _mdj()
    (lk, lp), (rk, rp) = datagen.zipf_tables(50_000_000, 200_000_000, 10_000_000, 1.1, seed=2)
    want_count, _ = oracle.count_checksum_dense(lk, lp, rk, rp, 10_000_000)
    L, R = _dev([lk, lp]), _dev([rk, rp])
    del lk, lp, rk, rp
    rows = 1 << 24
    with mdj.MergeStream(L, R, 64) as st:
        n = st.total_rows
        assert n == want_count
        buf = st.buffers(rows)
        for q0 in (0, n // 3, n // 2 + 12_345, (2 * n) // 3, n - rows):
            v = st.emit(q0, rows, buf)
            li = v.left_row.view(torch.int32).to(torch.int64)
            ri = v.right_row.view(torch.int32).to(torch.int64)
            assert torch.equal(v.key, L[0][li]) and torch.equal(v.key, R[0][ri])
            assert torch.equal(v.left_cols[0].view(torch.int64), L[1].view(torch.int64)[li])
            assert torch.equal(v.right_cols[0].view(torch.int64), R[1].view(torch.int64)[ri])
            pair = torch.sort(li * 200_000_000 + ri).values
            assert torch.unique_consecutive(pair).numel() == rows


# ------------------------------------------------ merge variants (outer joins)

OUTER = ["left", "right", "outer"]


@pytest.mark.parametrize("how", OUTER)
@pytest.mark.parametrize("P", [1, 8])
def test_outer_unique_build_keys(how, P):
    left, right = datagen.match_fraction_tables(150_000, 200_000, 0.3, seed=41)
    _check(list(left), list(right), P, window=50_001, how=how)


@pytest.mark.parametrize("how", OUTER)
def test_outer_duplicate_keys(how):
    # overlapping but different key ranges: unmatched rows on both sides
    rng = np.random.default_rng(42)
    lk = rng.integers(0, 40_000, 120_000).astype(np.int64)
    rk = rng.integers(20_000, 70_000, 90_000).astype(np.int64)
    _check([lk, rng.random(lk.size)], [rk, rng.random(rk.size)], 8, window=77_777, how=how)


@pytest.mark.parametrize("how", OUTER)
def test_outer_heavy_keys(how):
    left, right = _skewed_tables(43)
    rng = np.random.default_rng(44)
    # plus left-only and right-only keys, one of them heavy on each side
    left[0] = np.concatenate([left[0], np.full(5000, -3), rng.integers(10**9, 2 * 10**9, 3000)])
    left[1] = np.concatenate([left[1], rng.random(8000)])
    right[0] = np.concatenate([right[0], np.full(7000, -5), rng.integers(3 * 10**9, 4 * 10**9, 3000)])
    right[1] = np.concatenate([right[1], rng.random(10_000)])
    _check(left, right, 8, window=2_000_003, how=how)


@pytest.mark.parametrize("how", OUTER)
def test_outer_int32_several_columns(how):
    (lk, lp), (rk, rp) = datagen.random_tables(40_000, 60_000, 100_000, seed=45, key_dtype=np.int32,
                                               pay_dtype=np.float32)
    rng = np.random.default_rng(46)
    lx = rng.integers(0, 2**62, lk.size, dtype=np.int64)
    _check([lk, lp, lx], [rp, rk], 4, window=9_999, lk=0, rk=1, how=how)


@pytest.mark.parametrize("how", ["inner"] + OUTER)
@pytest.mark.parametrize("nl,nr", [(0, 3000), (3000, 0), (0, 0)])
def test_outer_empty_side(how, nl, nr):
    left, right = datagen.match_fraction_tables(max(nl, 1), max(nr, 1), 0.3, seed=47)
    left = [c[:nl] for c in left]
    right = [c[:nr] for c in right]
    want = oracle.merge_table_how(left, right, how)
    total, got = _stream_all(left, right, 8, 1000, how=how)
    assert total == want["key"].size
    if total:
        assert_same_result(gpu_result_np(got), want)


@pytest.mark.parametrize("how", OUTER)
def test_outer_small_unpartitioned(how):
    left, right = datagen.random_tables(2_000, 3_000, 4_000, seed=48)
    _check(list(left), list(right), 1, window=333, how=how)


def test_merge_how_one_call():
    mdj = _mdj()
    rng = np.random.default_rng(49)
    lk = rng.integers(0, 5000, 20_000).astype(np.int64)
    rk = rng.integers(2500, 7500, 20_000).astype(np.int64)
    left, right = [lk, rng.random(lk.size)], [rk, rng.random(rk.size)]
    res = mdj.merge(_dev(left), _dev(right), 8, how="outer")
    torch.cuda.synchronize()
    want = oracle.merge_table_how(left, right, "outer")
    assert_same_result(gpu_result_np(res), want)


# ------------------------------------------------ edge cases of the stream

@pytest.mark.parametrize("how", ["inner", "outer"])
def test_stream_all_keys_equal(how):
    # one key on both sides: one group of 5000 build rows (the global-memory
    # path) against 3000 probe rows, 15M rows in windows
    rng = np.random.default_rng(81)
    lk = np.full(5000, 42, np.int64)
    rk = np.full(3000, 42, np.int64)
    assert _check([lk, rng.random(5000)], [rk, rng.random(3000)], 8, window=4_000_000, how=how) == 15_000_000


def test_stream_extreme_keys_and_nan_payloads():
    rng = np.random.default_rng(82)
    ext = np.array([np.iinfo(np.int64).min, np.iinfo(np.int64).max, -1, 0], np.int64)
    lk = np.concatenate([ext, rng.integers(-5, 5, 2000)]).astype(np.int64)
    rk = np.concatenate([ext[::-1], ext, rng.integers(-5, 5, 3000)]).astype(np.int64)
    nan_bits = np.array([0x7FF8000000000001, 0xFFF0000000000001, 0x7FF4000000000000], np.uint64)
    lp = rng.random(lk.size)
    rp = rng.random(rk.size)
    lp.view(np.uint64)[:3] = nan_bits
    rp.view(np.uint64)[-3:] = nan_bits
    for how in ("inner", "left", "right", "outer"):
        _check([lk, lp], [rk, rp], 8, window=50_000, how=how)


@pytest.mark.parametrize("nl,nr,P", [(1, 1, 1), (1, 1, 64), (3, 2, 1024), (2, 5, 2048)])
def test_stream_tiny_tables_and_more_partitions_than_rows(nl, nr, P):
    lk = np.arange(nl, dtype=np.int64) % 2
    rk = np.arange(nr, dtype=np.int64) % 2
    left = [lk, np.arange(nl, dtype=np.float64)]
    right = [rk, np.arange(nr, dtype=np.float64)]
    for how in ("inner", "outer"):
        _check(left, right, P, window=1, how=how)
