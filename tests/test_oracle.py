"""Pins for the CPU oracle, against facts that do not come from the oracle itself.

The paper prints no output values for the merge (all its plots are figures,
Sec. V-B/V-C), so the oracle is pinned by: a hand-worked example, an
independent nested-loop join on tiny inputs, the closed form of the
match-fraction generator, the count identity m = sum_k lc(k) rc(k), explicit
pair enumeration for the checksum, partition invariants, and the data volumes
the paper states per worker.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2101_08878_gb300 import datagen

I64_MIN = np.iinfo(np.int64).min
I64_MAX = np.iinfo(np.int64).max


# ------------------------------------------------------------------ hashing

def test_fmix64_fixes_zero():
    # Every step of the finalizer (xor-shift, odd multiply) maps 0 to 0; a
    # stray added constant or a wrong seed would not.
    assert int(oracle.fmix64(np.zeros(1, np.uint64))[0]) == 0


def test_fmix64_is_a_bijection_on_a_sample():
    # fmix64 is a composition of invertible maps, so distinct inputs never collide.
    rng = np.random.default_rng(1)
    x = np.unique(np.concatenate([np.arange(1 << 20, dtype=np.uint64),
                                  rng.integers(0, 2**64 - 1, 1 << 20, dtype=np.uint64, endpoint=True)]))
    y = oracle.fmix64(x)
    assert np.unique(y).size == x.size


def test_fmix64_avalanche():
    # Strict avalanche: flipping any input bit flips each output bit with
    # probability ~1/2.  A dropped xor-shift or multiply breaks this badly.
    rng = np.random.default_rng(2)
    x = rng.integers(0, 2**64 - 1, 4000, dtype=np.uint64, endpoint=True)
    hx = oracle.fmix64(x)
    worst = 0.0
    for bit in range(64):
        d = hx ^ oracle.fmix64(x ^ np.uint64(1 << bit))
        bits = np.unpackbits(d.view(np.uint8).reshape(-1, 8), axis=1)
        p = bits.mean(axis=0)
        worst = max(worst, float(np.abs(p - 0.5).max()))
    assert worst < 0.06, worst


_M64 = (1 << 64) - 1


def _rotl64(x, r):
    return ((x << r) | (x >> (64 - r))) & _M64


def _murmur3_x64_128(data: bytes, seed: int, fin) -> bytes:
    """MurmurHash3_x64_128 (Appleby's published algorithm, restated here):
    16-byte blocks mixed into two 64-bit lanes, the tail, the length, and
    `fin` (the 64-bit finalizer) applied to both lanes."""
    c1, c2 = 0x87C37B91114253D5, 0x4CF5AD432745937F
    h1 = h2 = seed & 0xFFFFFFFF
    n = len(data)
    nblocks = n // 16
    for i in range(nblocks):
        k1 = int.from_bytes(data[16 * i:16 * i + 8], "little")
        k2 = int.from_bytes(data[16 * i + 8:16 * i + 16], "little")
        k1 = _rotl64((k1 * c1) & _M64, 31) * c2 & _M64
        h1 ^= k1
        h1 = (_rotl64(h1, 27) + h2) & _M64
        h1 = (h1 * 5 + 0x52DCE729) & _M64
        k2 = _rotl64((k2 * c2) & _M64, 33) * c1 & _M64
        h2 ^= k2
        h2 = (_rotl64(h2, 31) + h1) & _M64
        h2 = (h2 * 5 + 0x38495AB5) & _M64
    tail = data[16 * nblocks:]
    if len(tail) > 8:
        k2 = int.from_bytes(tail[8:], "little")
        h2 ^= _rotl64((k2 * c2) & _M64, 33) * c1 & _M64
    if tail:
        k1 = int.from_bytes(tail[:8], "little")
        h1 ^= _rotl64((k1 * c1) & _M64, 31) * c2 & _M64
    h1 ^= n
    h2 ^= n
    h1 = (h1 + h2) & _M64
    h2 = (h2 + h1) & _M64
    h1, h2 = fin(h1), fin(h2)
    h1 = (h1 + h2) & _M64
    h2 = (h2 + h1) & _M64
    return h1.to_bytes(8, "little") + h2.to_bytes(8, "little")


def _smhasher_verification(fin) -> int:
    # SMHasher's verification value: hash the keys {}, {0}, {0,1}, ...,
    # {0..254} with seed 256 - length, hash the 256 concatenated results with
    # seed 0, and read the first four bytes as a little-endian integer.
    key = bytes(range(256))
    hashes = b"".join(_murmur3_x64_128(key[:i], 256 - i, fin) for i in range(256))
    return int.from_bytes(_murmur3_x64_128(hashes, 0, fin)[:4], "little")


def _oracle_fin(h: int) -> int:
    return int(oracle.fmix64(np.array([h], dtype=np.uint64))[0])


def test_fmix64_is_murmur3_finalizer_known_answer():
    # SMHasher publishes 0x6384BA69 as the verification value of
    # MurmurHash3_x64_128, whose finalizer is fmix64.  With the oracle's
    # fmix64 as the finalizer the whole hash must reproduce it; this pins the
    # exact multipliers and shifts, which the partition rule rests on.
    assert _smhasher_verification(_oracle_fin) == 0x6384BA69


def _fmix_variant(m1, m2, s1, s2, s3):
    def fin(h):
        h ^= h >> s1
        h = (h * m1) & _M64
        h ^= h >> s2
        h = (h * m2) & _M64
        h ^= h >> s3
        return h
    return fin


@pytest.mark.parametrize("variant", [
    (0xC4CEB9FE1A85EC53, 0xFF51AFD7ED558CCD, 33, 33, 33),   # multipliers swapped
    (0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53, 31, 33, 33),   # first shift 31
    (0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC53, 33, 33, 32),   # last shift 32
    (0xFF51AFD7ED558CCD, 0xC4CEB9FE1A85EC55, 33, 33, 33),   # one multiplier bit off
])
def test_known_answer_rejects_plausible_finalizer_mistakes(variant):
    # The same known answer fails for finalizers with one plausible mistake
    # (these pass the zero, bijection and avalanche tests above).
    assert _smhasher_verification(_fmix_variant(*variant)) != 0x6384BA69
    x = np.random.default_rng(5).integers(0, 2**64 - 1, 300, dtype=np.uint64, endpoint=True)
    mutated = np.array([_fmix_variant(*variant)(int(v)) for v in x], dtype=np.uint64)
    assert not np.array_equal(oracle.fmix64(x), mutated)


def test_partition_ids_sign_extend_int32():
    # int32 and int64 columns holding equal values must hash to equal partitions.
    v = np.array([-5, -1, 0, 1, 7, 2**31 - 1, -(2**31)], dtype=np.int64)
    for P in (1, 2, 8, 37, 65536):
        assert np.array_equal(oracle.partition_ids(v, P), oracle.partition_ids(v.astype(np.int32), P))


def test_partition_ids_uniform():
    n, P = 1_000_000, 8
    c = np.bincount(oracle.partition_ids(np.arange(n, dtype=np.int64), P), minlength=P)
    sigma = math.sqrt(n * (1 / P) * (1 - 1 / P))
    assert np.all(np.abs(c - n / P) < 5 * sigma), c


def test_partition_power_of_two_uses_low_bits():
    # For P = 2^k, h mod P is the low k bits of h.
    keys = np.arange(-1000, 1000, dtype=np.int64)
    h = oracle.fmix64(keys.view(np.uint64))
    for k in (1, 3, 10, 16):
        assert np.array_equal(oracle.partition_ids(keys, 1 << k), (h & np.uint64((1 << k) - 1)).astype(np.uint32))


# ---------------------------------------------------------------- partition

@pytest.mark.parametrize("P", [1, 2, 3, 8, 64, 1000, 65536])
@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_partition_invariants(P, dtype):
    rng = np.random.default_rng(P)
    n = 20_000
    keys = rng.integers(-50_000, 50_000, n).astype(dtype)
    offsets, perm = oracle.partition(keys, P)
    pid = oracle.partition_ids(keys, P)
    # a permutation of 0..n-1
    assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.uint32))
    # offsets are the exclusive prefix sum of the partition sizes
    assert offsets[0] == 0 and offsets[-1] == n
    assert np.array_equal(np.diff(offsets), np.bincount(pid, minlength=P))
    for p in range(min(P, 70)):
        seg = perm[offsets[p]:offsets[p + 1]]
        assert np.all(pid[seg] == p)
        assert np.all(np.diff(seg.astype(np.int64)) > 0)  # stable: input order kept


def test_partition_empty_and_single():
    off, perm = oracle.partition(np.zeros(0, np.int64), 4)
    assert list(off) == [0, 0, 0, 0, 0] and perm.size == 0
    off, perm = oracle.partition(np.array([42], np.int64), 1)
    assert list(off) == [0, 1] and list(perm) == [0]


def test_partition_table_gathers_columns():
    keys = np.array([5, 9, 5, 1, 9, 9], np.int64)
    pay = np.arange(6, dtype=np.float64) / 10
    off, rid, (pk, pp) = oracle.partition_table([keys, pay], 0, 3)
    assert np.array_equal(pk, keys[rid]) and np.array_equal(pp.view(np.uint64), pay[rid].view(np.uint64))


# -------------------------------------------------------------------- merge

def test_merge_hand_worked_example():
    # left  rows: 0:k3 1:k1 2:k3 3:k7      right rows: 0:k3 1:k3 2:k9 3:k1
    # pairs by key: k1 -> (1,3); k3 -> (0,0) (0,1) (2,0) (2,1); k7, k9 unmatched.
    l = np.array([3, 1, 3, 7], np.int64)
    r = np.array([3, 3, 9, 1], np.int64)
    lrow, rrow = oracle.merge_pairs(l, r)
    assert list(zip(lrow.tolist(), rrow.tolist())) == [(1, 3), (0, 0), (0, 1), (2, 0), (2, 1)]


CASES = [
    # (n_l, n_r, key_range, dtype, seed)
    (0, 0, 10, np.int64, 0),
    (0, 50, 10, np.int64, 1),
    (50, 0, 10, np.int64, 2),
    (1, 1, 1, np.int64, 3),
    (300, 400, 50, np.int64, 4),      # heavy duplicates
    (1000, 1000, 5, np.int32, 5),     # very heavy duplicates
    (2000, 1500, 100_000, np.int64, 6),
    (2000, 2000, 3000, np.int32, 7),
]


@pytest.mark.parametrize("n_l,n_r,key_range,dtype,seed", CASES)
def test_merge_matches_brute_force(n_l, n_r, key_range, dtype, seed):
    (lk, _), (rk, _) = datagen.random_tables(n_l, n_r, key_range, seed, key_dtype=dtype)
    got = oracle.merge_pairs(lk, rk)
    want = oracle.brute_force(lk, rk)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_merge_extreme_keys():
    ext = np.array([I64_MIN, I64_MAX, 0, -1, I64_MIN, I64_MAX, I64_MIN + 1], np.int64)
    r = np.array([I64_MAX, I64_MIN, I64_MIN, 5, -1, I64_MAX - 1], np.int64)
    got = oracle.merge_pairs(ext, r)
    want = oracle.brute_force(ext, r)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert got[0].size == 2 * 2 + 2 * 1 + 1  # INT64_MIN: 2x2, INT64_MAX: 2x1, -1: 1x1


def test_merge_count_identity():
    # m = sum over keys of lc(k) * rc(k), counted with np.unique (no join).
    (lk, _), (rk, _) = datagen.zipf_tables(20_000, 30_000, 2_000, 1.1, seed=9)
    lu, lc = np.unique(lk, return_counts=True)
    ru, rc = np.unique(rk, return_counts=True)
    common, li, ri = np.intersect1d(lu, ru, return_indices=True)
    m = int(np.sum(lc[li].astype(np.int64) * rc[ri].astype(np.int64)))
    lrow, rrow = oracle.merge_pairs(lk, rk)
    assert lrow.size == m
    assert np.array_equal(lk[lrow], rk[rrow])


@pytest.mark.parametrize("n_l,n_r,frac", [(1000, 1000, 0.3), (10_000, 25_000, 0.3), (5000, 3000, 0.9), (100, 100, 0.0)])
def test_merge_closed_form_match_fraction(n_l, n_r, frac):
    (lk, _), (rk, _) = datagen.match_fraction_tables(n_l, n_r, frac, seed=n_l + n_r)
    lrow, rrow = oracle.merge_pairs(lk, rk)
    assert lrow.size == math.floor(frac * n_r)
    assert np.array_equal(lk[lrow], rk[rrow])
    assert np.unique(rrow).size == rrow.size  # each right row meets one left row


def test_merge_table_schema_and_bits():
    (lk, lp), (rk, rp) = datagen.match_fraction_tables(500, 700, 0.5, seed=3)
    # NaN payload bit patterns must survive untouched
    lp = lp.copy()
    lp.view(np.uint64)[::7] = np.uint64(0x7FF8DEADBEEF0001)
    res = oracle.merge_table([lk, lp], [rk, rp])
    assert np.array_equal(res["key"], lk[res["left_row"]])
    assert np.array_equal(res["left_cols"][0].view(np.uint64), lp.view(np.uint64)[res["left_row"]])
    assert np.array_equal(res["right_cols"][0].view(np.uint64), rp.view(np.uint64)[res["right_row"]])


def test_merge_key_dtype_mismatch_rejected():
    with pytest.raises(TypeError):
        oracle.merge_pairs(np.zeros(3, np.int32), np.zeros(3, np.int64))


# ----------------------------------------------------------- count/checksum

@pytest.mark.parametrize("seed,dup", [(0, 50), (1, 5), (2, 100_000)])
@pytest.mark.parametrize("pay", [np.float64, np.float32])
def test_count_checksum_equals_pair_enumeration(seed, dup, pay):
    (lk, lp), (rk, rp) = datagen.random_tables(700, 900, dup, seed, pay_dtype=pay)
    cnt, chk = oracle.count_checksum(lk, lp, rk, rp)
    li, rj = oracle.brute_force(lk, rk)
    f, g = oracle.checksum_terms(lk, lp, rp)
    mask = (1 << 64) - 1
    want = 0
    for a, b in zip(li.tolist(), rj.tolist()):
        want = (want + int(f[a]) * int(g[b])) & mask
    assert cnt == li.size
    assert chk == want


def test_checksum_terms_depend_on_every_field():
    # f must change with the key, the left row and the payload bits; g with the
    # right row and its payload bits (a dropped term would leave one fixed).
    lk = np.array([1, 2, 1], np.int64)
    lp = np.array([0.5, 0.5, 0.25])
    rp = np.array([0.5, 0.25, 0.5])
    f, g = oracle.checksum_terms(lk, lp, rp)
    assert len(set(f.tolist())) == 3 and len(set(g.tolist())) == 3
    f2, _ = oracle.checksum_terms(lk, lp + 1.0, rp)
    assert not np.any(f2 == f)


# --------------------------------------------------------- paper arithmetic

def test_data_volume_matches_paper():
    # Sec. V-B: 3.2 GB per worker at chunk size 1E8; Sec. V-C: 1.6 GB per GPU
    # at 5E7 and 51.2 GB on 32 GPUs.  Reading: rows per table per worker, one
    # 8-byte key + one 8-byte payload, two tables.
    per_row = np.dtype(np.int64).itemsize + np.dtype(np.float64).itemsize
    assert 1e8 * per_row * 2 == 3.2e9
    assert 5e7 * per_row * 2 == 1.6e9
    assert 32 * 5e7 * per_row * 2 == 51.2e9
    assert [k * 3.2 for k in range(1, 7)] == pytest.approx([3.2, 6.4, 9.6, 12.8, 16.0, 19.2])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dense_count_checksum_equals_sort_merge(seed):
    # the per-key-array form used for the full-size skewed config agrees with
    # the sort-merge form on the same Zipf tables
    (lk, lp), (rk, rp) = datagen.zipf_tables(30_000, 60_000, 2_000, 1.1, seed=seed)
    assert oracle.count_checksum_dense(lk, lp, rk, rp, 2_000) == oracle.count_checksum(lk, lp, rk, rp)


def test_dense_count_checksum_rejects_out_of_range_keys():
    with pytest.raises(ValueError):
        oracle.count_checksum_dense(np.array([5], np.int64), np.zeros(1), np.array([1], np.int64),
                                    np.zeros(1), 3)


def test_zipf_skew_matches_closed_form():
    # the Zipf(1.1) generator over 1e7 values: P(key = 0) = 1 / H(1e7, 1.1);
    # expected pair count of the skewed config, n_L n_R sum_k p_k^2, ~2.0e14
    k = np.arange(1, 10_000_001, dtype=np.float64)
    w = k ** -1.1
    p = w / w.sum()
    assert abs(1 / w.sum() - 0.1164) < 5e-4
    assert 1.9e14 < 5e7 * 2e8 * float(np.sum(p * p)) < 2.1e14
    rng = np.random.default_rng(5)
    keys = datagen.zipf_keys(rng, 2_000_000, 10_000_000, 1.1)
    assert abs(np.mean(keys == 0) - p[0]) < 5 * np.sqrt(p[0] * (1 - p[0]) / 2_000_000)


# ------------------------------------------------ transpose-sum (Fig. 7, 9(a))

def _loop_transpose_add(x):
    n = x.shape[0]
    y = np.empty_like(x)
    for i in range(n):
        for j in range(n):
            y[i, j] = x[i, j] + x[j, i]
    return y


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.int64, np.int32])
def test_transpose_add_equals_element_loop(dtype):
    rng = np.random.default_rng(11)
    x = (rng.standard_normal((9, 9)) * 1000).astype(dtype)
    assert np.array_equal(oracle.transpose_add(x), _loop_transpose_add(x))


def test_transpose_add_symmetric_and_antisymmetric_inputs():
    # y = x + x^T is symmetric bit for bit (IEEE addition commutes); a
    # symmetric x gives exactly 2x, an antisymmetric x (u - u^T) exactly 0
    rng = np.random.default_rng(12)
    u = rng.random((37, 37))
    y = oracle.transpose_add(u)
    assert np.array_equal(y.view(np.uint64), y.T.view(np.uint64))
    s = u + u.T
    assert np.array_equal(oracle.transpose_add(s), 2 * s)
    a = u - u.T
    assert np.array_equal(oracle.transpose_add(a), np.zeros_like(a))
    assert np.array_equal(np.diag(oracle.transpose_add(u)), 2 * np.diag(u))


def test_transpose_add_integer_wraparound():
    x = np.array([[2**63 - 1, 5], [-7, 0]], dtype=np.int64)
    y = oracle.transpose_add(x)
    assert y[0, 0] == -2 and y[0, 1] == -2 and y[1, 0] == -2 and y[1, 1] == 0
    x32 = np.array([[2**31 - 1, 1], [1, -2**31]], dtype=np.int32)
    assert oracle.transpose_add(x32)[0, 0] == -2 and oracle.transpose_add(x32)[1, 1] == 0


def test_transpose_sum_sizes_of_the_paper():
    # 16K x 16K (Fig. 7) and 20E3 x 20E3 (Fig. 9(a)) float64 arrays
    assert 16384 * 16384 * 8 == 2 * 2**30
    assert 20_000 * 20_000 * 8 == 3_200_000_000
    with pytest.raises(ValueError):
        oracle.transpose_add(np.zeros((2, 3)))


# ------------------------------------------------ merge variants (outer joins)

def _loop_outer(lk, lp, rk, rp, how):
    """Nested loops, written from the definition: every matching pair; then
    each left row without a match (left, outer) and each right row without a
    match (right, outer), once, with the other side missing."""
    rows = []
    for i in range(lk.size):
        found = False
        for j in range(rk.size):
            if lk[i] == rk[j]:
                rows.append((int(lk[i]), i, j, lp[i], rp[j]))
                found = True
        if not found and how in ("left", "outer"):
            rows.append((int(lk[i]), i, oracle.NO_ROW, lp[i], 0.0))
    if how in ("right", "outer"):
        for j in range(rk.size):
            if not any(lk[i] == rk[j] for i in range(lk.size)):
                rows.append((int(rk[j]), oracle.NO_ROW, j, 0.0, rp[j]))
    rows.sort(key=lambda t: (t[0], t[1], t[2]))
    return rows


@pytest.mark.parametrize("how", ["inner", "left", "right", "outer"])
def test_merge_variants_equal_nested_loops(how):
    rng = np.random.default_rng(21)
    lk = rng.integers(0, 40, 120).astype(np.int64)
    rk = rng.integers(20, 70, 90).astype(np.int64)
    lp, rp = rng.random(lk.size), rng.random(rk.size)
    got = oracle.merge_table_how([lk, lp], [rk, rp], how)
    want = _loop_outer(lk, lp, rk, rp, how)
    assert got["key"].size == len(want)
    assert [int(x) for x in got["key"]] == [t[0] for t in want]
    assert [int(x) for x in got["left_row"]] == [t[1] for t in want]
    assert [int(x) for x in got["right_row"]] == [t[2] for t in want]
    assert np.array_equal(got["left_cols"][0], np.array([t[3] for t in want]))
    assert np.array_equal(got["right_cols"][0], np.array([t[4] for t in want]))


def test_merge_variant_row_counts():
    # left join: each left row max(1, matches); right join likewise; outer =
    # inner + unmatched on both sides; missing sides carry zero bits
    rng = np.random.default_rng(22)
    lk = rng.integers(0, 500, 3000).astype(np.int32)
    rk = rng.integers(250, 900, 2000).astype(np.int32)
    lp, rp = rng.random(lk.size).astype(np.float32), rng.random(rk.size).astype(np.float32)
    lc = np.bincount(lk, minlength=900)
    rc = np.bincount(rk, minlength=900)
    inner = int(np.sum(lc * rc))
    left = oracle.merge_table_how([lk, lp], [rk, rp], "left")
    right = oracle.merge_table_how([lk, lp], [rk, rp], "right")
    outer = oracle.merge_table_how([lk, lp], [rk, rp], "outer")
    assert left["key"].size == int(np.sum(np.maximum(1, rc[lk])))
    assert right["key"].size == int(np.sum(np.maximum(1, lc[rk])))
    assert outer["key"].size == inner + int(np.sum(rc[lk] == 0)) + int(np.sum(lc[rk] == 0))
    miss = outer["right_row"] == oracle.NO_ROW
    assert np.all(outer["right_cols"][0][miss].view(np.uint32) == 0)
    assert np.all(lk[outer["left_row"][miss]] == outer["key"][miss])
    assert np.array_equal(oracle.merge_table_how([lk, lp], [rk, rp], "inner")["key"],
                          oracle.merge_table([lk, lp], [rk, rp])["key"])


# ------------------------------------------------ several key columns

def test_merge_multi_equals_nested_loops():
    rng = np.random.default_rng(61)
    a = rng.integers(0, 6, 200).astype(np.int64)
    b = rng.integers(0, 5, 200).astype(np.int32)
    c = rng.integers(0, 6, 150).astype(np.int64)
    d = rng.integers(0, 5, 150).astype(np.int32)
    lrow, rrow = oracle.merge_multi([a, b], [d, c], [0, 1], [1, 0])
    want = sorted((i, j) for i in range(a.size) for j in range(c.size) if a[i] == c[j] and b[i] == d[j])
    assert list(zip(lrow.tolist(), rrow.tolist())) == want
    # one key column: the plain merge's pairs
    l1, r1 = oracle.merge_multi([a], [c], [0], [0])
    pl, pr = oracle.merge_pairs(a, c)
    assert sorted(zip(l1.tolist(), r1.tolist())) == sorted(zip(pl.tolist(), pr.tolist()))


def test_merge_multi_is_not_a_merge_on_the_first_column():
    # tuples equal on the first column only must not join
    # (the first column alone would join (0,0) (0,1) (1,0) (1,1) (2,2))
    a = np.array([1, 1, 2], np.int64)
    b = np.array([5, 6, 5], np.int64)
    rb = np.array([6, 5, 9], np.int64)
    lrow, rrow = oracle.merge_multi([a, b], [a, rb], [0, 1], [0, 1])
    assert list(zip(lrow.tolist(), rrow.tolist())) == [(0, 1), (1, 0)]


# ------------------------------------------------------ outer joins on tuples

@pytest.mark.parametrize("how", ["inner", "left", "right", "outer"])
def test_merge_multi_how_on_one_key_is_the_single_key_merge(how):
    # with one key column the tuple merge is the plain merge: same row pairs,
    # the same unmatched rows and the same zeroed or coalesced columns
    rng = np.random.default_rng(81)
    left = [rng.integers(0, 60, 400).astype(np.int64), rng.random(400)]
    right = [rng.random(300), rng.integers(30, 90, 300).astype(np.int64)]
    a = oracle.merge_multi_how(left, right, [0], [1], how)
    b = oracle.merge_table_how(left, right, how, 0, 1)
    ka = np.lexsort((a["right_row"], a["left_row"]))
    kb = np.lexsort((b["right_row"], b["left_row"]))
    assert np.array_equal(a["left_row"][ka], b["left_row"][kb])
    assert np.array_equal(a["right_row"][ka], b["right_row"][kb])
    assert np.array_equal(a["left_cols"][0][ka], b["key"][kb])
    assert np.array_equal(a["left_cols"][1][ka].view(np.uint64), b["left_cols"][0][kb].view(np.uint64))
    assert np.array_equal(a["right_cols"][0][ka].view(np.uint64), b["right_cols"][0][kb].view(np.uint64))


@pytest.mark.parametrize("how", ["inner", "left", "right", "outer"])
def test_merge_multi_how_matches_nested_loops_on_pairs(how):
    # the definition written out on tiny tables: (i, j) joins when both key
    # columns agree; a row with no partner on the kept side appears once
    rng = np.random.default_rng(82)
    la, lb = rng.integers(0, 4, 40).astype(np.int32), rng.integers(0, 3, 40).astype(np.int64)
    ra, rb = rng.integers(1, 5, 30).astype(np.int32), rng.integers(0, 3, 30).astype(np.int64)
    left, right = [la, lb, np.arange(40, dtype=np.int64) * 10], [rb, ra, np.arange(30, dtype=np.int64) + 7]
    got = oracle.merge_multi_how(left, right, [0, 1], [1, 0], how)
    pairs = [(i, j) for i in range(40) for j in range(30) if la[i] == ra[j] and lb[i] == rb[j]]
    rows = list(pairs)
    if how in ("left", "outer"):
        rows += [(i, oracle.NO_ROW) for i in range(40) if not any(p[0] == i for p in pairs)]
    if how in ("right", "outer"):
        rows += [(oracle.NO_ROW, j) for j in range(30) if not any(p[1] == j for p in pairs)]
    rows.sort()
    assert list(zip(got["left_row"].tolist(), got["right_row"].tolist())) == rows
    for k, (i, j) in enumerate(rows):
        # key columns: the present side's tuple; other columns: zero when missing
        want_a = la[i] if i != oracle.NO_ROW else ra[j]
        want_b = lb[i] if i != oracle.NO_ROW else rb[j]
        assert got["left_cols"][0][k] == want_a and got["left_cols"][1][k] == want_b
        assert got["left_cols"][2][k] == (i * 10 if i != oracle.NO_ROW else 0)
        assert got["right_cols"][0][k] == (j + 7 if j != oracle.NO_ROW else 0)
