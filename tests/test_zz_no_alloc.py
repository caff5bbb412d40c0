"""mdj_partition_noalloc: the partition entry point for callers that may not
allocate device memory (it works in a fixed scratch array inside the library).

Called through the C ABI and checked, bit for bit, against mdj_partition (the
allocating entry point) on two calls in a row with different shapes, so that
anything a previous call left in the shared scratch array would show up.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2101_08878_gb300 import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _noalloc(cols, key_col, P):
    from paper_2101_08878_gb300 import mdj
    lib = mdj.load()
    tab, keep = mdj._table(cols)
    n = cols[0].numel()
    outs = [torch.empty_like(c) for c in cols]
    ptrs = (ctypes.c_void_p * len(cols))(*[o.data_ptr() if n else None for o in outs])
    rid = torch.empty(n, dtype=torch.uint32, device=DEV)
    off = torch.empty(P + 1, dtype=torch.int64, device=DEV)
    rc = lib.mdj_partition_noalloc(ctypes.byref(tab), key_col, P, ptrs, rid.data_ptr() if n else None,
                                   off.data_ptr(), torch.cuda.current_stream(DEV).cuda_stream)
    torch.cuda.synchronize()
    return rc, off, rid, outs


def _table(n, seed):
    rng = np.random.default_rng(seed)
    key = rng.integers(-3 * n, 3 * n, n).astype(np.int64)
    pay = datagen.uniform_payload(rng, n)
    tag = rng.integers(0, 2**31 - 1, n).astype(np.int32)
    return [torch.from_numpy(c).to(DEV) for c in (key, pay, tag)]


def test_noalloc_partition_matches_partition_on_two_calls():
    from paper_2101_08878_gb300 import mdj
    for n, P, seed in [(300_000, 64, 1), (123_457, 8, 2)]:
        cols = _table(n, seed)
        rc, off, rid, outs = _noalloc(cols, 0, P)
        assert rc == 0, mdj.mdj_status_string(rc)
        w_off, w_rid, w_outs = mdj.mdj_partition(cols, 0, P)
        torch.cuda.synchronize()
        assert torch.equal(off, w_off)
        assert torch.equal(rid.view(torch.int32), w_rid.view(torch.int32))
        for g, w in zip(outs, w_outs):
            assert torch.equal(g.view(torch.uint8), w.view(torch.uint8))


def test_noalloc_rejects_what_does_not_fit():
    from paper_2101_08878_gb300 import mdj
    # 1024 partitions of 20M rows need more scratch words than the array holds
    cols = [torch.zeros(20_000_000, dtype=torch.int64, device=DEV)]
    rc, _, _, _ = _noalloc(cols, 0, 1024)
    assert rc == -3, mdj.mdj_status_string(rc)
    # more partitions than one pass handles
    rc, _, _, _ = _noalloc(cols[:1], 0, 2000)
    assert rc == -1
