"""Helpers shared by the parity tests: move a GPU join result to numpy, sort it
canonically by (key, left_row, right_row) and compare it bit for bit with the
oracle's merge of the same inputs."""
import numpy as np

import oracle


def to_np(t):
    return t.detach().cpu().numpy()


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype.itemsize == 4 else a.view(np.uint64)


def gpu_result_np(res):
    out = {
        "key": to_np(res.key),
        "left_row": to_np(res.left_row).view(np.uint32),
        "right_row": to_np(res.right_row).view(np.uint32),
        "left_cols": [to_np(c) for c in res.left_cols],
        "right_cols": [to_np(c) for c in res.right_cols],
    }
    order = np.lexsort((out["right_row"], out["left_row"], out["key"].astype(np.int64)))
    for k in ("key", "left_row", "right_row"):
        out[k] = out[k][order]
    out["left_cols"] = [c[order] for c in out["left_cols"]]
    out["right_cols"] = [c[order] for c in out["right_cols"]]
    return out


def assert_same_result(got, want):
    """got: canonical GPU result; want: oracle.merge_table output (canonical)."""
    assert got["key"].size == want["key"].size, (got["key"].size, want["key"].size)
    assert got["key"].dtype == want["key"].dtype
    assert np.array_equal(got["key"], want["key"])
    assert np.array_equal(got["left_row"], want["left_row"])
    assert np.array_equal(got["right_row"], want["right_row"])
    assert len(got["left_cols"]) == len(want["left_cols"])
    assert len(got["right_cols"]) == len(want["right_cols"])
    for g, w in zip(got["left_cols"], want["left_cols"]):
        assert np.array_equal(bits(g), bits(w))
    for g, w in zip(got["right_cols"], want["right_cols"]):
        assert np.array_equal(bits(g), bits(w))


def oracle_result(left_np, right_np, lk=0, rk=0):
    return oracle.merge_table(left_np, right_np, lk, rk)
