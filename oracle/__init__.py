"""CPU oracle for the shuffle + inner hash join (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (``libmdj.so`` and its
Python binding) never does, and it shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, compiled with gcc into
``liboracle.so`` next to it); this module only marshals numpy arrays, plus one
independent nested-loop join (``brute_force``) used to pin the C sort-merge on
tiny inputs.  What each function computes is the plain definition of the
operation named in Sec. V-B ("cuDF Merge", Fig. 8 and Fig. 9(b,c)) of the
paper: a hash-partitioned shuffle followed by an inner equi-join.  The
paper's other application benchmark, the sum of an array and its transpose
(Sec. V-B, Fig. 7; Sec. V-C, Fig. 9(a)), is ``transpose_add``: its plain
numpy definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        lib.oracle_fmix64.restype = u64
        lib.oracle_fmix64.argtypes = [u64]
        lib.oracle_partition_of.restype = u32
        lib.oracle_partition_of.argtypes = [ctypes.c_int64, u32]
        lib.oracle_partition.restype = i32
        lib.oracle_partition.argtypes = [vp, i32, u64, u32, vp, vp]
        lib.oracle_merge.restype = i32
        lib.oracle_merge.argtypes = [vp, u64, vp, u64, i32, vp, vp, u64, ctypes.POINTER(u64)]
        lib.oracle_count_checksum.restype = i32
        lib.oracle_count_checksum.argtypes = [vp, vp, i32, u64, vp, vp, i32, u64, i32,
                                              ctypes.POINTER(u64), ctypes.POINTER(u64)]
        lib.oracle_count_checksum_dense.restype = i32
        lib.oracle_count_checksum_dense.argtypes = [vp, vp, i32, u64, vp, vp, i32, u64, i32, u64,
                                                    ctypes.POINTER(u64), ctypes.POINTER(u64)]
        lib.oracle_fmix64_array.restype = None
        lib.oracle_fmix64_array.argtypes = [vp, u64, vp]
        lib.oracle_partition_ids.restype = None
        lib.oracle_partition_ids.argtypes = [vp, i32, u64, u32, vp]
        lib.oracle_checksum_terms.restype = None
        lib.oracle_checksum_terms.argtypes = [vp, i32, vp, i32, u64, vp, i32, u64, vp, vp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _key_array(keys) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    if keys.dtype not in (np.int32, np.int64):
        raise TypeError(f"oracle keys must be int32 or int64, got {keys.dtype}")
    return keys


def _bits(pay) -> np.ndarray:
    pay = np.ascontiguousarray(pay)
    if pay.dtype.itemsize == 4:
        return pay.view(np.uint32)
    if pay.dtype.itemsize == 8:
        return pay.view(np.uint64)
    raise TypeError(f"payload width must be 4 or 8 bytes, got {pay.dtype}")


# ----------------------------------------------------------------- hashing

def fmix64(x: np.ndarray) -> np.ndarray:
    """MurmurHash3 64-bit finalizer applied elementwise (uint64 in, uint64 out)."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.empty_like(x)
    _load().oracle_fmix64_array(_ptr(x), x.size, _ptr(out))
    return out


def partition_ids(keys, P: int) -> np.ndarray:
    """p = fmix64(sext64(key)) mod P for every key (uint32)."""
    keys = _key_array(keys)
    out = np.empty(keys.size, dtype=np.uint32)
    _load().oracle_partition_ids(_ptr(keys), keys.dtype.itemsize, keys.size, P, _ptr(out))
    return out


# --------------------------------------------------------------- partition

def partition(keys, P: int):
    """Stable hash partition: returns (offsets int64[P+1], perm uint32[n])."""
    keys = _key_array(keys)
    offsets = np.empty(P + 1, dtype=np.int64)
    perm = np.empty(keys.size, dtype=np.uint32)
    rc = _load().oracle_partition(_ptr(keys), keys.dtype.itemsize, keys.size, P,
                                  _ptr(offsets), _ptr(perm))
    if rc != 0:
        raise ValueError("oracle_partition failed")
    return offsets, perm


def partition_table(cols, key_col: int, P: int):
    """Stable partition of a whole table (list of 1-D arrays).

    Returns (offsets, row_ids, partitioned columns): column j of the output is
    the input column gathered by row_ids.
    """
    offsets, perm = partition(cols[key_col], P)
    return offsets, perm, [np.ascontiguousarray(np.asarray(c)[perm]) for c in cols]


# ------------------------------------------------------------------- merge

def merge_pairs(lkeys, rkeys):
    """Inner equi-join row pairs (lrow, rrow), canonical order (key, lrow, rrow)."""
    lkeys, rkeys = _key_array(lkeys), _key_array(rkeys)
    if lkeys.dtype != rkeys.dtype:
        raise TypeError("left and right key columns must have the same dtype")
    lib = _load()
    m = ctypes.c_uint64(0)
    dummy = np.empty(1, dtype=np.uint32)
    rc = lib.oracle_merge(_ptr(lkeys), lkeys.size, _ptr(rkeys), rkeys.size,
                          lkeys.dtype.itemsize, _ptr(dummy), _ptr(dummy), 0, ctypes.byref(m))
    if rc != 0:
        raise ValueError("oracle_merge failed")
    lrow = np.empty(m.value, dtype=np.uint32)
    rrow = np.empty(m.value, dtype=np.uint32)
    rc = lib.oracle_merge(_ptr(lkeys), lkeys.size, _ptr(rkeys), rkeys.size,
                          lkeys.dtype.itemsize, _ptr(lrow), _ptr(rrow), m.value, ctypes.byref(m))
    if rc != 0:
        raise ValueError("oracle_merge failed")
    return lrow, rrow


def merge_table(left_cols, right_cols, key_col_l: int = 0, key_col_r: int = 0):
    """The full merge result in canonical order.

    Output schema: key, left_row, right_row, then the left non-key columns in
    order, then the right non-key columns in order (values gathered, bits
    preserved).
    """
    lrow, rrow = merge_pairs(left_cols[key_col_l], right_cols[key_col_r])
    lk = np.asarray(left_cols[key_col_l])
    return {
        "key": lk[lrow],
        "left_row": lrow,
        "right_row": rrow,
        "left_cols": [np.asarray(c)[lrow] for j, c in enumerate(left_cols) if j != key_col_l],
        "right_cols": [np.asarray(c)[rrow] for j, c in enumerate(right_cols) if j != key_col_r],
    }


NO_ROW = 0xFFFFFFFF  # row id of the missing side of an outer-join row


def merge_table_how(left_cols, right_cols, how: str, key_col_l: int = 0, key_col_r: int = 0):
    """The merge variants, canonical order (key, left_row, right_row; NO_ROW last).

    "inner" is merge_table.  "left" adds every left row whose key no right row
    has, once, with no right row; "right" adds every right row whose key no
    left row has, once, with no left row; "outer" adds both.  A missing side
    has row id NO_ROW and all-zero bits in its columns; the key is the present
    side's.
    """
    if how not in ("inner", "left", "right", "outer"):
        raise ValueError(f"unknown join type {how!r}")
    inner = merge_table(left_cols, right_cols, key_col_l, key_col_r)
    lk = np.asarray(left_cols[key_col_l])
    rk = np.asarray(right_cols[key_col_r])
    lcols = [np.asarray(c) for j, c in enumerate(left_cols) if j != key_col_l]
    rcols = [np.asarray(c) for j, c in enumerate(right_cols) if j != key_col_r]
    ul = np.nonzero(~np.isin(lk, rk))[0] if how in ("left", "outer") else np.empty(0, np.int64)
    ur = np.nonzero(~np.isin(rk, lk))[0] if how in ("right", "outer") else np.empty(0, np.int64)
    none_l = np.full(ul.size, NO_ROW, np.uint32)
    none_r = np.full(ur.size, NO_ROW, np.uint32)
    key = np.concatenate([inner["key"], lk[ul], rk[ur]])
    lrow = np.concatenate([inner["left_row"], ul.astype(np.uint32), none_r])
    rrow = np.concatenate([inner["right_row"], none_l, ur.astype(np.uint32)])
    left_out = [np.concatenate([a, c[ul], np.zeros(ur.size, c.dtype)]) for a, c in zip(inner["left_cols"], lcols)]
    right_out = [np.concatenate([a, np.zeros(ul.size, c.dtype), c[ur]]) for a, c in zip(inner["right_cols"], rcols)]
    order = np.lexsort((rrow, lrow, key))
    return {"key": key[order], "left_row": lrow[order], "right_row": rrow[order],
            "left_cols": [c[order] for c in left_out], "right_cols": [c[order] for c in right_out]}


def merge_multi(left_cols, right_cols, left_keys, right_keys):
    """Inner merge on key tuples (left_keys[a] = right_keys[a] for every a):
    row pairs (lrow, rrow) in (lrow, rrow) order.  The tuples of both tables
    are numbered by np.unique over their rows (equal tuples, equal number),
    then the numbers are merged by merge_pairs."""
    lt = np.stack([np.asarray(left_cols[k]).astype(np.int64) for k in left_keys], axis=1)
    rt = np.stack([np.asarray(right_cols[k]).astype(np.int64) for k in right_keys], axis=1)
    both = np.concatenate([lt, rt], axis=0) if lt.size + rt.size else np.zeros((0, len(left_keys)), np.int64)
    _, ids = np.unique(both, axis=0, return_inverse=True)
    ids = ids.reshape(-1).astype(np.int64)
    lrow, rrow = merge_pairs(ids[:lt.shape[0]], ids[lt.shape[0]:])
    order = np.lexsort((rrow, lrow))
    return lrow[order], rrow[order]


def merge_multi_how(left_cols, right_cols, left_keys, right_keys, how: str):
    """The merge variants on key tuples (a merge variant, as merge_table_how on
    a single key).  "inner" is merge_multi; "left" adds every left row that no
    right row matches on the whole tuple, once, with no right row; "right"
    adds every unmatched right row, with no left row; "outer" adds both.
    Returns a dict: left_row, right_row (NO_ROW for a missing side) and the
    output columns in the order of mdj_merge_multi: left_cols = the key
    columns in left_keys order, then the left table's other columns; right_cols
    = the right table's other columns.  A missing side's columns are all-zero
    bits, except that the key columns of a right-only row hold the right
    row's tuple (the key is the present side's).  Canonical order: (left_row,
    right_row) with NO_ROW last."""
    if how not in ("inner", "left", "right", "outer"):
        raise ValueError(f"unknown join type {how!r}")
    lrow, rrow = merge_multi(left_cols, right_cols, left_keys, right_keys)
    nl = len(left_cols[0]) if len(left_cols) else 0
    nr = len(right_cols[0]) if len(right_cols) else 0
    ul = np.setdiff1d(np.arange(nl), lrow) if how in ("left", "outer") else np.empty(0, np.int64)
    ur = np.setdiff1d(np.arange(nr), rrow) if how in ("right", "outer") else np.empty(0, np.int64)
    lrow_all = np.concatenate([lrow.astype(np.int64), ul, np.full(ur.size, NO_ROW, np.int64)])
    rrow_all = np.concatenate([rrow.astype(np.int64), np.full(ul.size, NO_ROW, np.int64), ur])
    lorder = list(left_keys) + [j for j in range(len(left_cols)) if j not in left_keys]
    rorder = [j for j in range(len(right_cols)) if j not in right_keys]
    left_out = []
    for pos, j in enumerate(lorder):
        c = np.asarray(left_cols[j])
        right_part = (np.asarray(right_cols[right_keys[pos]])[ur] if pos < len(left_keys)
                      else np.zeros(ur.size, c.dtype))
        left_out.append(np.concatenate([c[lrow.astype(np.int64)], c[ul], right_part.astype(c.dtype)]))
    right_out = []
    for j in rorder:
        c = np.asarray(right_cols[j])
        right_out.append(np.concatenate([c[rrow.astype(np.int64)], np.zeros(ul.size, c.dtype), c[ur]]))
    order = np.lexsort((rrow_all, lrow_all))
    return {"left_row": lrow_all[order].astype(np.uint32), "right_row": rrow_all[order].astype(np.uint32),
            "left_cols": [c[order] for c in left_out], "right_cols": [c[order] for c in right_out]}


def brute_force(lkeys, rkeys):
    """Nested-loop inner join (independent of the C code) for tiny inputs.

    Every (i, j) with lkeys[i] == rkeys[j], sorted by (key, i, j).
    """
    lk = np.asarray(lkeys).astype(np.int64)
    rk = np.asarray(rkeys).astype(np.int64)
    if lk.size * rk.size > 50_000_000:
        raise ValueError("brute_force is for tiny inputs only")
    li, rj = np.nonzero(lk[:, None] == rk[None, :])
    order = np.lexsort((rj, li, lk[li]))
    return li[order].astype(np.uint32), rj[order].astype(np.uint32)


# ------------------------------------------------------- count + checksum

def checksum_terms(lkeys, lpay, rpay):
    """Per-row checksum terms f(l) (left) and g(r) (right), uint64."""
    lkeys = _key_array(lkeys)
    lb, rb = _bits(lpay), _bits(rpay)
    f = np.empty(lkeys.size, dtype=np.uint64)
    g = np.empty(rb.size, dtype=np.uint64)
    _load().oracle_checksum_terms(_ptr(lkeys), lkeys.dtype.itemsize, _ptr(lb), lb.dtype.itemsize,
                                  lkeys.size, _ptr(rb), rb.dtype.itemsize, rb.size, _ptr(f), _ptr(g))
    return f, g


def count_checksum(lkeys, lpay, rkeys, rpay):
    """(pair count, sum over pairs of f(l)*g(r) mod 2^64), by key groups."""
    lkeys, rkeys = _key_array(lkeys), _key_array(rkeys)
    if lkeys.dtype != rkeys.dtype:
        raise TypeError("left and right key columns must have the same dtype")
    lb, rb = _bits(lpay), _bits(rpay)
    cnt, chk = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = _load().oracle_count_checksum(_ptr(lkeys), _ptr(lb), lb.dtype.itemsize, lkeys.size,
                                       _ptr(rkeys), _ptr(rb), rb.dtype.itemsize, rkeys.size,
                                       lkeys.dtype.itemsize, ctypes.byref(cnt), ctypes.byref(chk))
    if rc != 0:
        raise ValueError("oracle_count_checksum failed")
    return cnt.value, chk.value


def count_checksum_dense(lkeys, lpay, rkeys, rpay, key_range: int):
    """count_checksum for keys in [0, key_range), by per-key arrays (no sort)."""
    lkeys, rkeys = _key_array(lkeys), _key_array(rkeys)
    if lkeys.dtype != rkeys.dtype:
        raise TypeError("left and right key columns must have the same dtype")
    lb, rb = _bits(lpay), _bits(rpay)
    cnt, chk = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = _load().oracle_count_checksum_dense(_ptr(lkeys), _ptr(lb), lb.dtype.itemsize, lkeys.size,
                                             _ptr(rkeys), _ptr(rb), rb.dtype.itemsize, rkeys.size,
                                             lkeys.dtype.itemsize, key_range, ctypes.byref(cnt),
                                             ctypes.byref(chk))
    if rc != 0:
        raise ValueError("oracle_count_checksum_dense failed (key outside [0, key_range)?)")
    return cnt.value, chk.value


# ------------------------------------------------------- transpose-sum

def transpose_add(x):
    """y = x + x.T (Sec. V-B "Sum of cuPy Array and its Transpose"): one
    addition per element in the array's own dtype (IEEE for floats, modulo
    2^bits for integers, as numpy adds arrays)."""
    x = np.asarray(x)
    if x.ndim != 2 or x.shape[0] != x.shape[1]:
        raise ValueError("x must be a square matrix")
    return x + x.T
