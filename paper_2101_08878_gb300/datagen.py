"""Seeded synthetic tables shaped like the paper's cuDF merge benchmark.

This module only draws random inputs; it holds none of the join's arithmetic
(no hashing, partitioning or matching), so both the CUDA path and the CPU
oracle can consume its arrays.

The paper gives the benchmark parameters but not the generator (Sec. V-B,
Fig. 8: "Chunk Size: 1E8, Shuffle: True, Fraction Match: 0.3"; Fig. 9(b):
"Chunk Size: 5E7").  Readings used here:

* chunk size = rows per table per worker, one 8-byte key and one 8-byte
  payload column: 1e8 rows x 16 B x 2 tables = 3.2 GB per worker, which is the
  paper's stated data volume per worker (Sec. V-B), and 5e7 rows give 1.6 GB
  (Sec. V-C).
* fraction match f: left keys are a seeded permutation of [0, n_L) (unique);
  exactly floor(f * n_R) right rows draw keys uniformly with replacement from
  the left keys, the others draw uniformly from the disjoint range
  [n_L, 2 n_L); right row positions are then shuffled.  Every matching right
  row meets exactly one left row, so the join has exactly floor(f * n_R) rows.
* payloads are U[0, 1) doubles (53 random bits) or floats (24 random bits).
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_payload(rng: np.random.Generator, n: int, dtype=np.float64) -> np.ndarray:
    """U[0,1) payload column: (u64 >> 11) * 2^-53 for f64, (u32 >> 8) * 2^-24 for f32."""
    if np.dtype(dtype) == np.float64:
        u = rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64, endpoint=True)
        return (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    if np.dtype(dtype) == np.float32:
        u = rng.integers(0, 2**32 - 1, size=n, dtype=np.uint32, endpoint=True)
        return ((u >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    raise TypeError(f"unsupported payload dtype {dtype}")


def match_fraction_tables(n_l: int, n_r: int, frac: float, seed: int,
                          key_dtype=np.int64, pay_dtype=np.float64):
    """Left/right (key, payload) tables with unique left keys and match fraction `frac`.

    Returns ((lkey, lpay), (rkey, rpay)); the join of the two has exactly
    floor(frac * n_r) rows.
    """
    if 2 * n_l > np.iinfo(key_dtype).max + 1:
        raise ValueError("key range [0, 2 n_l) does not fit the key dtype")
    rng = _rng(seed)
    lkey = rng.permutation(n_l).astype(key_dtype)
    n_match = int(math.floor(frac * n_r))
    rkey = np.empty(n_r, dtype=key_dtype)
    if n_l > 0:
        rkey[:n_match] = rng.integers(0, n_l, size=n_match, dtype=np.int64).astype(key_dtype)
        rkey[n_match:] = rng.integers(n_l, 2 * n_l, size=n_r - n_match, dtype=np.int64).astype(key_dtype)
    else:
        rkey[:] = rng.integers(0, 2**31 - 1, size=n_r, dtype=np.int64).astype(key_dtype)
    rkey = rkey[rng.permutation(n_r)]
    lpay = uniform_payload(rng, n_l, pay_dtype)
    rpay = uniform_payload(rng, n_r, pay_dtype)
    return (lkey, lpay), (rkey, rpay)


def zipf_keys(rng: np.random.Generator, n: int, n_values: int, s: float, key_dtype=np.int64) -> np.ndarray:
    """n keys in [0, n_values) with P(key = k-1) proportional to k^-s (exact inverse CDF)."""
    k = np.arange(1, n_values + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-s))
    cdf /= cdf[-1]
    u = rng.random(n)
    return np.minimum(np.searchsorted(cdf, u, side="right"), n_values - 1).astype(key_dtype)


def zipf_tables(n_l: int, n_r: int, n_values: int, s: float, seed: int,
                key_dtype=np.int64, pay_dtype=np.float64):
    """Skewed many-to-many tables: both sides draw keys Zipf(s) over n_values values."""
    rng = _rng(seed)
    lkey = zipf_keys(rng, n_l, n_values, s, key_dtype)
    rkey = zipf_keys(rng, n_r, n_values, s, key_dtype)
    return (lkey, uniform_payload(rng, n_l, pay_dtype)), (rkey, uniform_payload(rng, n_r, pay_dtype))


def random_tables(n_l: int, n_r: int, key_range: int, seed: int, key_dtype=np.int64,
                  pay_dtype=np.float64, key_low: int | None = None):
    """Keys uniform in [key_low, key_low + key_range) on both sides (duplicates likely)."""
    rng = _rng(seed)
    lo = -(key_range // 2) if key_low is None else key_low
    lkey = rng.integers(lo, lo + key_range, size=n_l, dtype=np.int64).astype(key_dtype)
    rkey = rng.integers(lo, lo + key_range, size=n_r, dtype=np.int64).astype(key_dtype)
    return (lkey, uniform_payload(rng, n_l, pay_dtype)), (rkey, uniform_payload(rng, n_r, pay_dtype))


def log_uniform_sizes(rng: np.random.Generator, count: int, lo: int, hi: int) -> np.ndarray:
    """Integer sizes log-uniform in [lo, hi]."""
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=count))).astype(np.int64).clip(lo, hi)


def batch_pairs(npairs: int, lo: int, hi: int, seed: int, frac_lo: float = 0.1, frac_hi: float = 0.9):
    """Independent partition-pair tables for the batched form.

    Per pair: n_L, n_R log-uniform in [lo, hi], match fraction U[frac_lo, frac_hi],
    int64 keys, float64 payloads.  Returns a list of ((lkey, lpay), (rkey, rpay)).
    """
    rng = _rng(seed)
    nl = log_uniform_sizes(rng, npairs, lo, hi)
    nr = log_uniform_sizes(rng, npairs, lo, hi)
    fr = rng.uniform(frac_lo, frac_hi, size=npairs)
    sub = rng.integers(0, 2**62, size=npairs)
    return [match_fraction_tables(int(a), int(b), float(f), int(s)) for a, b, f, s in zip(nl, nr, fr, sub)]
