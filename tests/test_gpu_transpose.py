"""y = x + x^T (mdj_transpose_add through the C ABI) against the oracle.

Bit for bit in every dtype: one IEEE addition per float element, addition
modulo 2^bits for integers.  Sizes cover one element, ragged tiles on both
sides of the 64-element tile edge, many tiles, and the paper's 16K x 16K
array (Fig. 7); the 20E3 x 20E3 array (Fig. 9(a)) runs as a slow case.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _random(n, dtype, seed):
    rng = np.random.default_rng(seed)
    if np.dtype(dtype).kind == "f":
        return (rng.standard_normal((n, n)) * 1e3).astype(dtype)
    info = np.iinfo(dtype)
    return rng.integers(info.min, info.max, size=(n, n), dtype=dtype, endpoint=True)


def _bits(a):
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 200, 1000, 4099])
@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.int64, np.int32])
def test_transpose_add_matches_oracle(n, dtype):
    x = _random(n, dtype, seed=n)
    y = _mdj().transpose_add(torch.from_numpy(x).to(DEV))
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(oracle.transpose_add(x)))


def test_transpose_add_in_place():
    x = _random(777, np.float64, seed=3)
    t = torch.from_numpy(x).to(DEV)
    out = _mdj().transpose_add(t, out=t)
    assert out.data_ptr() == t.data_ptr()
    assert np.array_equal(_bits(t.cpu().numpy()), _bits(oracle.transpose_add(x)))


def test_transpose_add_rejects_partial_overlap():
    mdj = _mdj()
    lib = mdj.load()
    buf = torch.zeros(2 * 64 * 64, dtype=torch.float64, device=DEV)
    rc = lib.mdj_transpose_add(buf.data_ptr(), buf.data_ptr() + 8 * 64, 64, mdj.MDJ_F64, None)
    assert rc == -1


def test_transpose_add_paper_size_16k():
    x = _random(16384, np.float64, seed=16)
    y = _mdj().transpose_add(torch.from_numpy(x).to(DEV))
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(oracle.transpose_add(x)))


@pytest.mark.slow
def test_transpose_add_paper_size_20e3():
    x = _random(20_000, np.float64, seed=20)
    y = _mdj().transpose_add(torch.from_numpy(x).to(DEV))
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(oracle.transpose_add(x)))
