"""mdj_partition (the shuffle) against the oracle's stable partition, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2101_08878_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mdj():
    from paper_2101_08878_gb300 import mdj
    return mdj


def _table(n, key_dtype, seed, key_range=None):
    rng = np.random.default_rng(seed)
    kr = key_range or max(4 * n, 16)
    key = rng.integers(-kr, kr, n).astype(key_dtype)
    f64 = datagen.uniform_payload(rng, n, np.float64)
    f32 = datagen.uniform_payload(rng, n, np.float32)
    i32 = rng.integers(-2**31, 2**31 - 1, n).astype(np.int32)
    return [key, f64, f32, i32]


def _check(cols_np, key_col, P):
    mdj = _mdj()
    dev = torch.device("cuda", 0)
    cols = [torch.from_numpy(c).to(dev) for c in cols_np]
    off, rid, outs = mdj.mdj_partition(cols, key_col, P)
    torch.cuda.synchronize()
    w_off, w_rid, w_cols = oracle.partition_table(cols_np, key_col, P)
    assert np.array_equal(off.cpu().numpy(), w_off)
    assert np.array_equal(rid.cpu().numpy().view(np.uint32), w_rid)
    for g, w in zip(outs, w_cols):
        g = g.cpu().numpy()
        assert g.dtype == w.dtype
        assert np.array_equal(g.view(np.uint8), w.view(np.uint8))


@pytest.mark.parametrize("n", [0, 1, 37, 8191, 8192, 8193, 100_003])
@pytest.mark.parametrize("P", [1, 8, 1024])
def test_partition_sizes(n, P):
    _check(_table(n, np.int64, seed=n + P), 0, P)


@pytest.mark.parametrize("P", [2, 3, 7, 64, 1000, 1023])
@pytest.mark.parametrize("key_dtype", [np.int32, np.int64])
def test_partition_fanouts(P, key_dtype):
    _check(_table(50_000, key_dtype, seed=P), 0, P)


@pytest.mark.parametrize("P", [1025, 4096, 65536])
def test_partition_lsd_large_P(P):
    # P above one pass's fan-out: two stable digit passes
    _check(_table(200_000, np.int64, seed=P), 0, P)


def test_partition_key_not_first_and_duplicates():
    cols = _table(60_000, np.int32, seed=5, key_range=40)  # heavy duplicates
    cols = [cols[1], cols[2], cols[0], cols[3]]
    _check(cols, 2, 16)


def test_partition_extreme_keys():
    rng = np.random.default_rng(11)
    ext = np.array([np.iinfo(np.int64).min, np.iinfo(np.int64).max, 0, -1], np.int64)
    key = rng.choice(ext, 20_000)
    _check([key, datagen.uniform_payload(rng, key.size)], 0, 8)


def test_partition_invalid_args():
    mdj = _mdj()
    dev = torch.device("cuda", 0)
    k = torch.arange(10, device=dev)
    for P in (0, 65537):
        with pytest.raises(mdj.MdjError) as e:
            mdj.mdj_partition([k], 0, P)
        assert e.value.status == -1
    with pytest.raises(mdj.MdjError) as e:
        mdj.mdj_partition([k.double()], 0, 4)  # float key
    assert e.value.status == -2
