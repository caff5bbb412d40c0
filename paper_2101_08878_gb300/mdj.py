"""ctypes binding of libmdj.so (declared in include/mdj.h).

Argument marshalling only: every step of the shuffle and join runs in the
library's CUDA kernels.  Device memory for workspace and outputs comes from
PyTorch's caching allocator through an mdj_allocator callback, and every call
runs on the current torch CUDA stream.  There is no CPU fallback: if the
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdj.so")

MDJ_MAX_COLS = 16
MDJ_OK = 0
STATUS = {
    0: "MDJ_OK", -1: "MDJ_ERR_INVALID_ARG", -2: "MDJ_ERR_UNSUPPORTED_DTYPE", -3: "MDJ_ERR_TOO_LARGE",
    -4: "MDJ_ERR_OOM", -5: "MDJ_ERR_CUDA", -6: "MDJ_ERR_DEVICE_TIMEOUT", -7: "MDJ_ERR_INTERNAL",
    -8: "MDJ_ERR_ABORTED",
}
MDJ_I32, MDJ_I64, MDJ_F32, MDJ_F64, MDJ_U32, MDJ_U64 = 1, 2, 3, 4, 5, 6
HOW = {"inner": 0, "left": 1, "right": 2, "outer": 3}   # mdj_how
NO_ROW = 0xFFFFFFFF  # row id of the missing side of an outer-join row

_TORCH_TO_MDJ = {
    torch.int32: MDJ_I32, torch.int64: MDJ_I64, torch.float32: MDJ_F32, torch.float64: MDJ_F64,
    torch.uint32: MDJ_U32, torch.uint64: MDJ_U64,
}
_MDJ_TO_TORCH = {v: k for k, v in _TORCH_TO_MDJ.items()}

EXPORTED = [
    "mdj_partition", "mdj_partition_noalloc", "mdj_join", "mdj_merge", "mdj_count_checksum", "mdj_join_batch",
    "mdj_merge_batch", "mdj_stream_open", "mdj_stream_emit", "mdj_stream_next", "mdj_stream_rows",
    "mdj_stream_close", "mdj_transpose_add", "mdj_merge_host", "mdj_merge_multi", "mdj_merge_multi_how",
    "mdj_result_release",
    "mdj_status_string", "mdj_last_error", "mdj_version", "mdj_profile_enable", "mdj_profile_reset",
    "mdj_profile_collect", "mdj_profile_count", "mdj_profile_get",
]


class MdjError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


# ---------------------------------------------------------------- C structs

class MdjCol(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class MdjTable(ctypes.Structure):
    _fields_ = [("cols", ctypes.POINTER(MdjCol)), ("ncols", ctypes.c_int32), ("nrows", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class MdjAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


class MdjResult(ctypes.Structure):
    _fields_ = [
        ("nrows", ctypes.c_uint64), ("key_dtype", ctypes.c_int32), ("n_left_cols", ctypes.c_int32),
        ("n_right_cols", ctypes.c_int32), ("left_dtypes", ctypes.c_int32 * MDJ_MAX_COLS),
        ("right_dtypes", ctypes.c_int32 * MDJ_MAX_COLS), ("key", ctypes.c_void_p),
        ("left_row", ctypes.c_void_p), ("right_row", ctypes.c_void_p),
        ("left_cols", ctypes.c_void_p * MDJ_MAX_COLS), ("right_cols", ctypes.c_void_p * MDJ_MAX_COLS),
    ]


class MdjWindow(ctypes.Structure):
    _fields_ = [
        ("key", ctypes.c_void_p), ("left_row", ctypes.c_void_p), ("right_row", ctypes.c_void_p),
        ("left_cols", ctypes.c_void_p * MDJ_MAX_COLS), ("right_cols", ctypes.c_void_p * MDJ_MAX_COLS),
    ]


SINK_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(MdjResult), ctypes.c_uint64, ctypes.c_void_p)


class MdjTuning(ctypes.Structure):
    _fields_ = [("table_rows", ctypes.c_uint32), ("fill_pct", ctypes.c_uint32), ("join_threads", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 5)]


_lib = None
_lib_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libmdj.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libmdj.so not found at {path}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
        P = ctypes.POINTER
        lib.mdj_partition.restype = ctypes.c_int
        lib.mdj_partition.argtypes = [P(MdjTable), i32, u32, P(vp), vp, vp, P(MdjAllocator), vp]
        lib.mdj_partition_noalloc.restype = ctypes.c_int
        lib.mdj_partition_noalloc.argtypes = [P(MdjTable), i32, u32, P(vp), vp, vp, vp]
        for name in ("mdj_join",):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [P(MdjTable), i32, P(MdjTable), i32, P(MdjAllocator), vp, P(MdjResult)]
        lib.mdj_merge.restype = ctypes.c_int
        lib.mdj_merge.argtypes = [P(MdjTable), i32, P(MdjTable), i32, u32, P(MdjAllocator), vp, P(MdjResult)]
        lib.mdj_count_checksum.restype = ctypes.c_int
        lib.mdj_count_checksum.argtypes = [P(MdjTable), i32, P(MdjTable), i32, u32, P(MdjAllocator), vp,
                                           P(u64), P(u64)]
        lib.mdj_join_batch.restype = ctypes.c_int
        lib.mdj_join_batch.argtypes = [P(MdjTable), i32, P(u64), P(MdjTable), i32, P(u64), i32, P(MdjTuning),
                                       P(MdjAllocator), vp, P(MdjResult), P(u64)]
        lib.mdj_merge_batch.restype = ctypes.c_int
        lib.mdj_merge_batch.argtypes = [P(MdjTable), i32, P(u64), P(MdjTable), i32, P(u64), i32, P(u32),
                                        P(MdjTuning), P(MdjAllocator), vp, P(MdjResult), P(u64)]
        lib.mdj_stream_open.restype = ctypes.c_int
        lib.mdj_stream_open.argtypes = [P(MdjTable), i32, P(MdjTable), i32, u32, i32, P(MdjAllocator), vp, P(vp),
                                        P(u64)]
        lib.mdj_stream_emit.restype = ctypes.c_int
        lib.mdj_stream_emit.argtypes = [vp, u64, u64, P(MdjWindow)]
        lib.mdj_stream_next.restype = ctypes.c_int
        lib.mdj_stream_next.argtypes = [vp, u64, P(MdjWindow), P(u64), P(u64)]
        lib.mdj_stream_rows.restype = u64
        lib.mdj_stream_rows.argtypes = [vp]
        lib.mdj_stream_close.restype = None
        lib.mdj_stream_close.argtypes = [vp]
        lib.mdj_merge_multi.restype = ctypes.c_int
        lib.mdj_merge_multi.argtypes = [P(MdjTable), P(i32), P(MdjTable), P(i32), i32, u32, P(MdjAllocator), vp,
                                        P(MdjResult)]
        lib.mdj_merge_multi_how.restype = ctypes.c_int
        lib.mdj_merge_multi_how.argtypes = [P(MdjTable), P(i32), P(MdjTable), P(i32), i32, u32, i32,
                                            P(MdjAllocator), vp, P(MdjResult)]
        lib.mdj_merge_host.restype = ctypes.c_int
        lib.mdj_merge_host.argtypes = [P(MdjTable), i32, P(MdjTable), i32, u32, i32, u64, SINK_FN, vp,
                                       P(MdjAllocator), vp, P(u64)]
        lib.mdj_transpose_add.restype = ctypes.c_int
        lib.mdj_transpose_add.argtypes = [vp, vp, u64, i32, vp]
        lib.mdj_result_release.restype = None
        lib.mdj_result_release.argtypes = [P(MdjResult), P(MdjAllocator), vp]
        lib.mdj_status_string.restype = ctypes.c_char_p
        lib.mdj_status_string.argtypes = [ctypes.c_int]
        lib.mdj_version.restype = ctypes.c_int
        lib.mdj_last_error.restype = ctypes.c_char_p
        lib.mdj_profile_enable.argtypes = [ctypes.c_int]
        lib.mdj_profile_enable.restype = None
        lib.mdj_profile_reset.restype = None
        lib.mdj_profile_collect.restype = ctypes.c_int
        lib.mdj_profile_count.restype = ctypes.c_int
        lib.mdj_profile_get.restype = ctypes.c_int
        lib.mdj_profile_get.argtypes = [ctypes.c_int, P(ctypes.c_char_p), P(u64), P(ctypes.c_double)]
        _lib = lib
        return lib


# ------------------------------------------------------------ torch memory

class TorchAllocator:
    """mdj_allocator backed by torch's caching allocator on one device.

    Buffers stay referenced in `live` until the library releases them or the
    caller adopts them (join outputs)."""

    def __init__(self, device: torch.device):
        self.device = device
        self.live = {}
        self.failed = False
        self._alloc = ALLOC_FN(self._on_alloc)
        self._release = RELEASE_FN(self._on_release)
        self.struct = MdjAllocator(self._alloc, self._release, None)

    def _on_alloc(self, nbytes, ctx, stream):
        try:
            t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=self.device)
        except Exception:  # noqa: BLE001 - an allocation failure becomes MDJ_ERR_OOM
            self.failed = True
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _on_release(self, ptr, ctx, stream):
        if ptr:
            self.live.pop(int(ptr), None)

    def adopt(self, ptr, n: int, dtype: torch.dtype) -> torch.Tensor:
        if not ptr or n == 0:
            return torch.empty(0, dtype=dtype, device=self.device)
        t = self.live.pop(int(ptr))
        return t[: n * torch.empty((), dtype=dtype).element_size()].view(dtype)


# ----------------------------------------------------------------- helpers

def _table(cols: Sequence[torch.Tensor]):
    if not 1 <= len(cols) <= MDJ_MAX_COLS:
        raise ValueError(f"a table needs 1..{MDJ_MAX_COLS} columns")
    n = cols[0].numel()
    arr = (MdjCol * len(cols))()
    for j, c in enumerate(cols):
        if not c.is_cuda:
            raise ValueError("columns must be CUDA tensors")
        if c.dim() != 1 or c.numel() != n or not c.is_contiguous():
            raise ValueError("columns must be contiguous 1-D tensors of equal length")
        if c.dtype not in _TORCH_TO_MDJ:
            raise TypeError(f"unsupported column dtype {c.dtype}")
        arr[j].data = c.data_ptr() if n else None
        arr[j].dtype = _TORCH_TO_MDJ[c.dtype]
    return MdjTable(arr, len(cols), n), arr


def _stream_handle(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _check(rc: int, what: str):
    if rc != MDJ_OK:
        detail = ""
        if rc == -5 and _lib is not None:
            detail = _lib.mdj_last_error().decode(errors="replace")
        raise MdjError(rc, what + (f" [{detail}]" if detail else ""))


@dataclass
class JoinResult:
    """Columns of an inner join result (device tensors, nrows each)."""
    nrows: int
    key: torch.Tensor
    left_row: torch.Tensor
    right_row: torch.Tensor
    left_cols: List[torch.Tensor]
    right_cols: List[torch.Tensor]


def _adopt_result(res: MdjResult, alloc: TorchAllocator) -> JoinResult:
    m = int(res.nrows)
    kd = _MDJ_TO_TORCH.get(res.key_dtype, torch.int64)
    return JoinResult(
        nrows=m,
        key=alloc.adopt(res.key, m, kd),
        left_row=alloc.adopt(res.left_row, m, torch.uint32),
        right_row=alloc.adopt(res.right_row, m, torch.uint32),
        left_cols=[alloc.adopt(res.left_cols[j], m, _MDJ_TO_TORCH[res.left_dtypes[j]])
                   for j in range(res.n_left_cols)],
        right_cols=[alloc.adopt(res.right_cols[j], m, _MDJ_TO_TORCH[res.right_dtypes[j]])
                    for j in range(res.n_right_cols)],
    )


# --------------------------------------------------------------- public API

def mdj_partition(cols: Sequence[torch.Tensor], key_col: int, P: int, row_ids: bool = True):
    """Stable hash partition (see mdj.h).  Returns (offsets int64[P+1], row_ids uint32[n] or None, columns)."""
    lib = load()
    dev = cols[0].device
    tab, keep = _table(cols)
    n = tab.nrows
    outs = [torch.empty(n, dtype=c.dtype, device=dev) for c in cols]
    out_ptrs = (ctypes.c_void_p * len(cols))(*[o.data_ptr() if n else None for o in outs])
    rid = torch.empty(n, dtype=torch.uint32, device=dev) if row_ids else None
    offsets = torch.empty(P + 1, dtype=torch.int64, device=dev)
    alloc = TorchAllocator(dev)
    rc = lib.mdj_partition(ctypes.byref(tab), key_col, P, out_ptrs,
                           rid.data_ptr() if (rid is not None and n) else None, offsets.data_ptr(),
                           ctypes.byref(alloc.struct), _stream_handle(dev))
    _check(rc, "mdj_partition")
    return offsets, rid, outs


def mdj_join(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor],
             left_key: int = 0, right_key: int = 0) -> JoinResult:
    """Inner equi-join without shuffle (see mdj.h)."""
    lib = load()
    dev = left_cols[0].device
    lt, lk = _table(left_cols)
    rt, rk = _table(right_cols)
    alloc = TorchAllocator(dev)
    res = MdjResult()
    rc = lib.mdj_join(ctypes.byref(lt), left_key, ctypes.byref(rt), right_key, ctypes.byref(alloc.struct),
                      _stream_handle(dev), ctypes.byref(res))
    _check(rc, "mdj_join")
    return _adopt_result(res, alloc)


def mdj_merge(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], P: int,
              left_key: int = 0, right_key: int = 0) -> JoinResult:
    """Hash shuffle into P partitions + per-partition inner join (see mdj.h)."""
    lib = load()
    dev = left_cols[0].device
    lt, lk = _table(left_cols)
    rt, rk = _table(right_cols)
    alloc = TorchAllocator(dev)
    res = MdjResult()
    rc = lib.mdj_merge(ctypes.byref(lt), left_key, ctypes.byref(rt), right_key, P, ctypes.byref(alloc.struct),
                       _stream_handle(dev), ctypes.byref(res))
    _check(rc, "mdj_merge")
    return _adopt_result(res, alloc)


def mdj_merge_multi(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], left_keys: Sequence[int],
                    right_keys: Sequence[int], P: int, how: str = "inner") -> JoinResult:
    """Merge on several key columns (mdj_merge_multi / mdj_merge_multi_how in
    mdj.h), `how` one of inner, left, right, outer.  The result's key is
    empty; left_cols = the left key columns (in left_keys order), then the
    left table's other columns; right_cols = the right table's other columns.
    A missing side has row id NO_ROW and zeroed columns; a right-only row's
    key columns hold its own tuple."""
    if how not in HOW:
        raise ValueError(f"how must be one of {sorted(HOW)}")
    lib = load()
    dev = left_cols[0].device
    lt, lkeep = _table(left_cols)
    rt, rkeep = _table(right_cols)
    if len(left_keys) != len(right_keys):
        raise ValueError("left_keys and right_keys need the same length")
    nk = len(left_keys)
    lk = (ctypes.c_int32 * max(nk, 1))(*left_keys)
    rk = (ctypes.c_int32 * max(nk, 1))(*right_keys)
    alloc = TorchAllocator(dev)
    res = MdjResult()
    if how == "inner":
        rc = lib.mdj_merge_multi(ctypes.byref(lt), lk, ctypes.byref(rt), rk, nk, P, ctypes.byref(alloc.struct),
                                 _stream_handle(dev), ctypes.byref(res))
    else:
        rc = lib.mdj_merge_multi_how(ctypes.byref(lt), lk, ctypes.byref(rt), rk, nk, P, HOW[how],
                                     ctypes.byref(alloc.struct), _stream_handle(dev), ctypes.byref(res))
    _check(rc, "mdj_merge_multi")
    return _adopt_result(res, alloc)


def mdj_count_checksum(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], P: int,
                       left_key: int = 0, right_key: int = 0):
    """(pair count, pair checksum) of the merge without materialising it (see mdj.h)."""
    lib = load()
    dev = left_cols[0].device
    lt, lk = _table(left_cols)
    rt, rk = _table(right_cols)
    alloc = TorchAllocator(dev)
    cnt, chk = ctypes.c_uint64(0), ctypes.c_uint64(0)
    rc = lib.mdj_count_checksum(ctypes.byref(lt), left_key, ctypes.byref(rt), right_key, P,
                                ctypes.byref(alloc.struct), _stream_handle(dev), ctypes.byref(cnt),
                                ctypes.byref(chk))
    _check(rc, "mdj_count_checksum")
    return cnt.value, chk.value


def mdj_join_batch(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], left_offsets,
                   right_offsets, left_key: int = 0, right_key: int = 0, table_rows: int = 0,
                   fill_pct: int = 0, join_threads: int = 0):
    """Independent joins of pair i = left rows [left_offsets[i], left_offsets[i+1])
    with right rows [right_offsets[i], right_offsets[i+1]) (see mdj.h).

    Returns (JoinResult of all pairs, pair_offsets) where pair i's output rows
    are [pair_offsets[i], pair_offsets[i+1]); row ids index the whole tables."""
    lib = load()
    dev = left_cols[0].device
    lt, lk = _table(left_cols)
    rt, rk = _table(right_cols)
    lo = [int(x) for x in left_offsets]
    ro = [int(x) for x in right_offsets]
    if len(lo) != len(ro) or len(lo) < 2:
        raise ValueError("left_offsets and right_offsets need npairs + 1 entries each")
    npairs = len(lo) - 1
    lo_c = (ctypes.c_uint64 * len(lo))(*lo)
    ro_c = (ctypes.c_uint64 * len(ro))(*ro)
    po_c = (ctypes.c_uint64 * len(lo))()
    tun = MdjTuning(table_rows, fill_pct, join_threads)
    alloc = TorchAllocator(dev)
    res = MdjResult()
    rc = lib.mdj_join_batch(ctypes.byref(lt), left_key, lo_c, ctypes.byref(rt), right_key, ro_c, npairs,
                            ctypes.byref(tun), ctypes.byref(alloc.struct), _stream_handle(dev), ctypes.byref(res),
                            po_c)
    _check(rc, "mdj_join_batch")
    return _adopt_result(res, alloc), [int(x) for x in po_c]


def mdj_merge_batch(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], left_offsets,
                    right_offsets, P, left_key: int = 0, right_key: int = 0, table_rows: int = 0,
                    fill_pct: int = 0, join_threads: int = 0):
    """Independent merges: request i = left rows [left_offsets[i], left_offsets[i+1])
    and right rows [right_offsets[i], right_offsets[i+1]), shuffled into P[i]
    partitions and joined (see mdj.h).  Returns (JoinResult, req_offsets)."""
    lib = load()
    dev = left_cols[0].device
    lt, lk = _table(left_cols)
    rt, rk = _table(right_cols)
    lo = [int(x) for x in left_offsets]
    ro = [int(x) for x in right_offsets]
    pp = [int(x) for x in P]
    if len(lo) != len(ro) or len(lo) < 2 or len(pp) != len(lo) - 1:
        raise ValueError("offsets need nreq + 1 entries and P nreq entries")
    nreq = len(lo) - 1
    lo_c = (ctypes.c_uint64 * len(lo))(*lo)
    ro_c = (ctypes.c_uint64 * len(ro))(*ro)
    p_c = (ctypes.c_uint32 * nreq)(*pp)
    out_c = (ctypes.c_uint64 * len(lo))()
    tun = MdjTuning(table_rows, fill_pct, join_threads)
    alloc = TorchAllocator(dev)
    res = MdjResult()
    rc = lib.mdj_merge_batch(ctypes.byref(lt), left_key, lo_c, ctypes.byref(rt), right_key, ro_c, nreq, p_c,
                             ctypes.byref(tun), ctypes.byref(alloc.struct), _stream_handle(dev), ctypes.byref(res),
                             out_c)
    _check(rc, "mdj_merge_batch")
    return _adopt_result(res, alloc), [int(x) for x in out_c]


class MergeStream:
    """The merge of mdj_merge, written window by window (mdj_stream_* in mdj.h).

    Opening runs the shuffle and groups the left rows by key; `total_rows`
    is then exact, and rows [q0, q0 + n) of the fixed output order can be
    written at any time into a window buffer.  `how` is "inner", "left",
    "right" or "outer"; a row's missing side has row id NO_ROW and zero bits
    in its columns.  The handle's device memory comes from torch's caching
    allocator and is held until close().  The input tensors must stay alive
    and unchanged until close()."""

    def __init__(self, left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], P: int,
                 left_key: int = 0, right_key: int = 0, how: str = "inner"):
        if how not in HOW:
            raise ValueError(f"how must be one of {sorted(HOW)}")
        lib = load()
        self._lib = lib
        self.device = left_cols[0].device
        self._inputs = (list(left_cols), list(right_cols))
        lt, lk = _table(left_cols)
        rt, rk = _table(right_cols)
        self._alloc = TorchAllocator(self.device)
        self._h = ctypes.c_void_p()
        total = ctypes.c_uint64(0)
        rc = lib.mdj_stream_open(ctypes.byref(lt), left_key, ctypes.byref(rt), right_key, P, HOW[how],
                                 ctypes.byref(self._alloc.struct), _stream_handle(self.device),
                                 ctypes.byref(self._h), ctypes.byref(total))
        _check(rc, "mdj_stream_open")
        self.total_rows = int(total.value)
        self.key_dtype = left_cols[left_key].dtype
        self.left_dtypes = [c.dtype for j, c in enumerate(left_cols) if j != left_key]
        self.right_dtypes = [c.dtype for j, c in enumerate(right_cols) if j != right_key]

    def buffers(self, rows: int) -> JoinResult:
        """A window buffer of `rows` rows (every column) on the handle's device."""
        dev = self.device
        return JoinResult(rows, torch.empty(rows, dtype=self.key_dtype, device=dev),
                          torch.empty(rows, dtype=torch.uint32, device=dev),
                          torch.empty(rows, dtype=torch.uint32, device=dev),
                          [torch.empty(rows, dtype=d, device=dev) for d in self.left_dtypes],
                          [torch.empty(rows, dtype=d, device=dev) for d in self.right_dtypes])

    @staticmethod
    def _window(buf: JoinResult, nrows: int) -> MdjWindow:
        w = MdjWindow()
        for name in ("key", "left_row", "right_row"):
            t = getattr(buf, name)
            if t is not None:
                if t.numel() < nrows:
                    raise ValueError(f"window buffer {name} holds {t.numel()} rows, {nrows} needed")
                setattr(w, name, t.data_ptr() if nrows else None)
        for side, arr in (("left_cols", w.left_cols), ("right_cols", w.right_cols)):
            for j, t in enumerate(getattr(buf, side)):
                if t is not None:
                    if t.numel() < nrows:
                        raise ValueError(f"window buffer {side}[{j}] holds {t.numel()} rows, {nrows} needed")
                    arr[j] = t.data_ptr() if nrows else None
        return w

    def emit(self, first_row: int, nrows: int, buf: JoinResult) -> JoinResult:
        """Rows [first_row, first_row + nrows) into `buf` (None entries are skipped);
        returns views of the written rows."""
        if self._h is None:
            raise RuntimeError("stream is closed")
        w = self._window(buf, nrows)
        _check(self._lib.mdj_stream_emit(self._h, first_row, nrows, ctypes.byref(w)), "mdj_stream_emit")
        return _view(buf, nrows)

    def next(self, buf: JoinResult, max_rows: Optional[int] = None):
        """The next window after the cursor (at most max_rows, default the buffer's
        rows): (first_row, views); views.nrows == 0 at the end."""
        if self._h is None:
            raise RuntimeError("stream is closed")
        cap = buf.nrows if max_rows is None else int(max_rows)
        w = self._window(buf, min(cap, self.total_rows))
        first, n = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(self._lib.mdj_stream_next(self._h, cap, ctypes.byref(w), ctypes.byref(first), ctypes.byref(n)),
               "mdj_stream_next")
        return int(first.value), _view(buf, int(n.value))

    def windows(self, rows: int):
        """Iterates (first_row, views) over the whole result through one buffer of
        `rows` rows; each window is valid until the next iteration."""
        buf = self.buffers(rows)
        for q0 in range(0, self.total_rows, rows):
            yield q0, self.emit(q0, min(rows, self.total_rows - q0), buf)

    def close(self):
        if self._h is not None:
            self._lib.mdj_stream_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def merge(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], P: int, how: str = "inner",
          left_key: int = 0, right_key: int = 0) -> JoinResult:
    """The merge with a join type: "inner" is mdj_merge; "left", "right" and
    "outer" run the streamed path and write every row in one window."""
    if how == "inner":
        return mdj_merge(left_cols, right_cols, P, left_key, right_key)
    with MergeStream(left_cols, right_cols, P, left_key, right_key, how) as st:
        buf = st.buffers(st.total_rows)
        if st.total_rows:
            st.emit(0, st.total_rows, buf)
        return buf


def _view(buf: JoinResult, n: int) -> JoinResult:
    cut = (lambda t: None if t is None else t[:n])
    return JoinResult(n, cut(buf.key), cut(buf.left_row), cut(buf.right_row), [cut(t) for t in buf.left_cols],
                      [cut(t) for t in buf.right_cols])


class _DeviceArray:
    """A borrowed device array, seen by torch through __cuda_array_interface__."""

    _TYPESTR = {torch.int32: "<i4", torch.int64: "<i8", torch.float32: "<f4", torch.float64: "<f8",
                torch.uint32: "<u4", torch.uint64: "<u8"}

    def __init__(self, ptr: int, n: int, dtype: torch.dtype):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": self._TYPESTR[dtype], "data": (ptr, False),
                                         "version": 3, "strides": None}


def _host_table(cols: Sequence[torch.Tensor]):
    if not 1 <= len(cols) <= MDJ_MAX_COLS:
        raise ValueError(f"a table needs 1..{MDJ_MAX_COLS} columns")
    n = cols[0].numel()
    arr = (MdjCol * len(cols))()
    for j, c in enumerate(cols):
        if c.is_cuda or c.dim() != 1 or c.numel() != n or not c.is_contiguous():
            raise ValueError("columns must be contiguous 1-D host tensors of equal length")
        if c.dtype not in _TORCH_TO_MDJ:
            raise TypeError(f"unsupported column dtype {c.dtype}")
        arr[j].data = c.data_ptr() if n else None
        arr[j].dtype = _TORCH_TO_MDJ[c.dtype]
    return MdjTable(arr, len(cols), n), arr


def merge_host_chunked(left_cols: Sequence[torch.Tensor], right_cols: Sequence[torch.Tensor], P: int,
                       device_budget: int, how: str = "inner", left_key: int = 0, right_key: int = 0,
                       on_piece=None, device: Optional[torch.device] = None):
    """The merge of host (CPU) tables that need not fit device memory
    (mdj_merge_host in mdj.h).  on_piece(first_row, JoinResult) receives each
    window as device tensors valid only during the call; by default the
    windows are copied to the host and returned as one JoinResult of CPU
    tensors.  Returns (total rows, that JoinResult or None)."""
    if how not in HOW:
        raise ValueError(f"how must be one of {sorted(HOW)}")
    lib = load()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    lt, lk_keep = _host_table(left_cols)
    rt, rk_keep = _host_table(right_cols)
    parts = []
    failure = []

    def collect(first_row, res):
        parts.append(JoinResult(res.nrows, res.key.cpu(), res.left_row.cpu(), res.right_row.cpu(),
                                [c.cpu() for c in res.left_cols], [c.cpu() for c in res.right_cols]))

    consume = on_piece or collect

    def sink(piece_p, first_row, ctx):
        try:
            pc = piece_p.contents
            n = int(pc.nrows)
            view = (lambda ptr, dt: torch.as_tensor(_DeviceArray(ptr, n, dt), device=dev))
            res = JoinResult(n, view(pc.key, _MDJ_TO_TORCH[pc.key_dtype]), view(pc.left_row, torch.uint32),
                             view(pc.right_row, torch.uint32),
                             [view(pc.left_cols[j], _MDJ_TO_TORCH[pc.left_dtypes[j]]) for j in range(pc.n_left_cols)],
                             [view(pc.right_cols[j], _MDJ_TO_TORCH[pc.right_dtypes[j]])
                              for j in range(pc.n_right_cols)])
            consume(int(first_row), res)
            return 0
        except Exception as e:  # noqa: BLE001 - reported after the call returns
            failure.append(e)
            return 1

    cb = SINK_FN(sink)
    alloc = TorchAllocator(dev)
    total = ctypes.c_uint64(0)
    rc = lib.mdj_merge_host(ctypes.byref(lt), left_key, ctypes.byref(rt), right_key, P, HOW[how], int(device_budget),
                            cb, None, ctypes.byref(alloc.struct), _stream_handle(dev), ctypes.byref(total))
    if failure:
        raise failure[0]
    _check(rc, "mdj_merge_host")
    if on_piece is not None:
        return int(total.value), None
    if not parts:
        kd = left_cols[left_key].dtype
        empty = (lambda dt: torch.empty(0, dtype=dt))
        return 0, JoinResult(0, empty(kd), empty(torch.uint32), empty(torch.uint32),
                             [empty(c.dtype) for j, c in enumerate(left_cols) if j != left_key],
                             [empty(c.dtype) for j, c in enumerate(right_cols) if j != right_key])
    cat = torch.cat
    out = JoinResult(int(total.value), cat([p.key for p in parts]), cat([p.left_row for p in parts]),
                     cat([p.right_row for p in parts]),
                     [cat([p.left_cols[j] for p in parts]) for j in range(len(parts[0].left_cols))],
                     [cat([p.right_cols[j] for p in parts]) for j in range(len(parts[0].right_cols))])
    return int(total.value), out


def transpose_add(x: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """y = x + x.T for a square, contiguous CUDA matrix (mdj_transpose_add in mdj.h).
    `out` may be x itself (in place) or None (a new tensor)."""
    lib = load()
    if not x.is_cuda or x.dim() != 2 or x.shape[0] != x.shape[1] or not x.is_contiguous():
        raise ValueError("x must be a square, contiguous CUDA matrix")
    if x.dtype not in _TORCH_TO_MDJ:
        raise TypeError(f"unsupported dtype {x.dtype}")
    y = torch.empty_like(x) if out is None else out
    if y.shape != x.shape or y.dtype != x.dtype or not y.is_contiguous() or y.device != x.device:
        raise ValueError("out must match x in shape, dtype and device and be contiguous")
    n = x.shape[0]
    _check(lib.mdj_transpose_add(x.data_ptr() if n else None, y.data_ptr() if n else None, n,
                                 _TORCH_TO_MDJ[x.dtype], _stream_handle(x.device)), "mdj_transpose_add")
    return y


def mdj_status_string(status: int) -> str:
    return load().mdj_status_string(status).decode()


def mdj_version() -> int:
    return load().mdj_version()


# ------------------------------------------------------------------ tracing

def profile_enable(on: bool = True):
    load().mdj_profile_enable(1 if on else 0)


def profile_reset():
    load().mdj_profile_reset()


def profile_collect() -> dict:
    """{kernel name: (launches, total device ms)} accumulated since the last reset."""
    lib = load()
    _check(lib.mdj_profile_collect(), "mdj_profile_collect")
    out = {}
    for i in range(lib.mdj_profile_count()):
        name = ctypes.c_char_p()
        launches = ctypes.c_uint64()
        ms = ctypes.c_double()
        _check(lib.mdj_profile_get(i, ctypes.byref(name), ctypes.byref(launches), ctypes.byref(ms)),
               "mdj_profile_get")
        out[name.value.decode()] = (launches.value, ms.value)
    return out


# --------------------------------------------------------------- host → host

def merge_host(left_cols, right_cols, P: int, left_key: int = 0, right_key: int = 0,
               device: Optional[torch.device] = None):
    """End-to-end merge of host (pinned) tensors: copy in, mdj_merge, copy the
    result out.  Returns (JoinResult with CPU tensors, h2d bytes, d2h bytes)."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    s = torch.cuda.current_stream(dev)
    dl = [c.to(dev, non_blocking=True) for c in left_cols]
    dr = [c.to(dev, non_blocking=True) for c in right_cols]
    h2d = sum(c.numel() * c.element_size() for c in list(left_cols) + list(right_cols))
    res = mdj_merge(dl, dr, P, left_key, right_key)

    def host(t):
        h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
        h.copy_(t, non_blocking=True)
        return h
    out = JoinResult(res.nrows, host(res.key), host(res.left_row), host(res.right_row),
                     [host(c) for c in res.left_cols], [host(c) for c in res.right_cols])
    s.synchronize()
    d2h = sum(t.numel() * t.element_size() for t in [out.key, out.left_row, out.right_row, *out.left_cols,
                                                      *out.right_cols])
    return out, h2d, d2h
