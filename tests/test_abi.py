"""The C ABI library loads and exports every entry point include/mdj.h
declares, and its host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdj.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"MDJ_API\s+[\w\s\*]*?\b(mdj_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_08878_gb300 import _build, mdj
    try:
        _build.build()
    except (OSError, RuntimeError) as e:  # no nvcc on this machine
        pytest.skip(f"cannot build libmdj.so here: {e}")
    return mdj.load()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mdj_partition", "mdj_join", "mdj_merge", "mdj_count_checksum", "mdj_result_release",
              "mdj_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2101_08878_gb300 import mdj
    names = declared()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(mdj.EXPORTED) | set(names)
    assert set(mdj.EXPORTED) == set(names)


def test_version_and_status_strings(lib):
    assert lib.mdj_version() == 1
    assert lib.mdj_status_string(0) == b"ok"
    assert b"invalid" in lib.mdj_status_string(-1)
    assert lib.mdj_status_string(12345) == b"unknown status"


def test_argument_checks_need_no_gpu(lib):
    from paper_2101_08878_gb300.mdj import MdjCol, MdjResult, MdjTable
    # null tables / bad key index / bad dtypes / P out of range are rejected
    # before any CUDA call
    res = MdjResult()
    assert lib.mdj_merge(None, 0, None, 0, 8, None, None, ctypes.byref(res)) == -1
    cols = (MdjCol * 1)()
    cols[0].data = None
    cols[0].dtype = 2  # I64, zero rows: null data allowed
    t = MdjTable(cols, 1, 0)
    assert lib.mdj_merge(ctypes.byref(t), 1, ctypes.byref(t), 0, 8, None, None, ctypes.byref(res)) == -1
    assert lib.mdj_merge(ctypes.byref(t), 0, ctypes.byref(t), 0, 0, None, None, ctypes.byref(res)) == -1
    assert lib.mdj_merge(ctypes.byref(t), 0, ctypes.byref(t), 0, 65537, None, None, ctypes.byref(res)) == -1
    fcols = (MdjCol * 1)()
    fcols[0].dtype = 4  # F64 key
    ft = MdjTable(fcols, 1, 0)
    assert lib.mdj_merge(ctypes.byref(ft), 0, ctypes.byref(ft), 0, 8, None, None, ctypes.byref(res)) == -2
    icols = (MdjCol * 1)()
    icols[0].dtype = 1  # I32 key vs I64 key
    it = MdjTable(icols, 1, 0)
    assert lib.mdj_merge(ctypes.byref(t), 0, ctypes.byref(it), 0, 8, None, None, ctypes.byref(res)) == -1
    big = MdjTable(cols, 1, 1 << 32)
    assert lib.mdj_merge(ctypes.byref(big), 0, ctypes.byref(t), 0, 8, None, None, ctypes.byref(res)) == -3
    bad = (MdjCol * 1)()
    bad[0].dtype = 99
    bt = MdjTable(bad, 1, 0)
    assert lib.mdj_partition(ctypes.byref(bt), 0, 4, None, None, None, None, None) == -2
    many = MdjTable(cols, 17, 0)
    assert lib.mdj_join(ctypes.byref(many), 0, ctypes.byref(t), 0, None, None, ctypes.byref(res)) == -1


def test_stream_argument_checks_need_no_gpu(lib):
    from paper_2101_08878_gb300.mdj import MdjCol, MdjTable, MdjWindow
    h = ctypes.c_void_p()
    total = ctypes.c_uint64(7)
    cols = (MdjCol * 1)()
    cols[0].dtype = 2
    t = MdjTable(cols, 1, 0)
    # null tables, bad key index, P out of range, float key, key dtype mismatch
    assert lib.mdj_stream_open(None, 0, ctypes.byref(t), 0, 8, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -1
    assert h.value is None and total.value == 0
    assert lib.mdj_stream_open(ctypes.byref(t), 1, ctypes.byref(t), 0, 8, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -1
    assert lib.mdj_stream_open(ctypes.byref(t), 0, ctypes.byref(t), 0, 0, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -1
    assert lib.mdj_stream_open(ctypes.byref(t), 0, ctypes.byref(t), 0, 65537, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -1
    fcols = (MdjCol * 1)()
    fcols[0].dtype = 4
    ft = MdjTable(fcols, 1, 0)
    assert lib.mdj_stream_open(ctypes.byref(ft), 0, ctypes.byref(ft), 0, 8, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -2
    icols = (MdjCol * 1)()
    icols[0].dtype = 1
    it = MdjTable(icols, 1, 0)
    assert lib.mdj_stream_open(ctypes.byref(t), 0, ctypes.byref(it), 0, 8, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -1
    big = MdjTable(cols, 1, 1 << 32)
    assert lib.mdj_stream_open(ctypes.byref(big), 0, ctypes.byref(t), 0, 8, 0, None, None, ctypes.byref(h),
                               ctypes.byref(total)) == -3
    assert lib.mdj_stream_open(ctypes.byref(t), 0, ctypes.byref(t), 0, 8, 0, None, None, None,
                               ctypes.byref(total)) == -1
    # join type outside mdj_how
    for how in (-1, 4):
        assert lib.mdj_stream_open(ctypes.byref(t), 0, ctypes.byref(t), 0, 8, how, None, None, ctypes.byref(h),
                                   ctypes.byref(total)) == -1
    # calls on a missing handle
    w = MdjWindow()
    first, n = ctypes.c_uint64(0), ctypes.c_uint64(0)
    assert lib.mdj_stream_emit(None, 0, 0, ctypes.byref(w)) == -1
    assert lib.mdj_stream_next(None, 10, ctypes.byref(w), ctypes.byref(first), ctypes.byref(n)) == -1
    assert lib.mdj_stream_rows(None) == 0
    lib.mdj_stream_close(None)


def test_transpose_add_argument_checks_need_no_gpu(lib):
    # n = 0 is a no-op; null pointers, unknown dtypes, n >= 2^32 and partial
    # overlap are rejected before any CUDA call
    assert lib.mdj_transpose_add(None, None, 0, 4, None) == 0
    assert lib.mdj_transpose_add(None, None, 5, 4, None) == -1
    assert lib.mdj_transpose_add(None, None, 5, 99, None) == -2
    assert lib.mdj_transpose_add(4096, 8192, 1 << 32, 4, None) == -3
    assert lib.mdj_transpose_add(4096, 4096 + 64, 8, 4, None) == -1
    assert lib.mdj_transpose_add(4097, 4097, 8, 4, None) == -1


def test_merge_host_argument_checks_need_no_gpu(lib):
    from paper_2101_08878_gb300.mdj import SINK_FN, MdjCol, MdjTable
    sink = SINK_FN(lambda piece, first, ctx: 0)
    total = ctypes.c_uint64(9)
    cols = (MdjCol * 1)()
    cols[0].dtype = 2
    t = MdjTable(cols, 1, 0)
    big_budget = 1 << 30
    # a budget below 64 MiB, a missing sink, a bad join type, P = 0, float keys, too many rows
    assert lib.mdj_merge_host(ctypes.byref(t), 0, ctypes.byref(t), 0, 8, 0, 1 << 20, sink, None, None, None,
                              ctypes.byref(total)) == -1
    assert lib.mdj_merge_host(ctypes.byref(t), 0, ctypes.byref(t), 0, 8, 0, big_budget, SINK_FN(), None, None,
                              None, ctypes.byref(total)) == -1
    assert lib.mdj_merge_host(ctypes.byref(t), 0, ctypes.byref(t), 0, 8, 7, big_budget, sink, None, None, None,
                              ctypes.byref(total)) == -1
    assert lib.mdj_merge_host(ctypes.byref(t), 0, ctypes.byref(t), 0, 0, 0, big_budget, sink, None, None, None,
                              ctypes.byref(total)) == -1
    fcols = (MdjCol * 1)()
    fcols[0].dtype = 4
    ft = MdjTable(fcols, 1, 0)
    assert lib.mdj_merge_host(ctypes.byref(ft), 0, ctypes.byref(ft), 0, 8, 0, big_budget, sink, None, None, None,
                              ctypes.byref(total)) == -2
    big = MdjTable(cols, 1, 1 << 32)
    assert lib.mdj_merge_host(ctypes.byref(big), 0, ctypes.byref(t), 0, 8, 0, big_budget, sink, None, None, None,
                              ctypes.byref(total)) == -3
    assert lib.mdj_status_string(-8) == b"stopped by the caller's sink"


def test_merge_multi_argument_checks_need_no_gpu(lib):
    from paper_2101_08878_gb300.mdj import MdjCol, MdjResult, MdjTable
    res = MdjResult()
    cols = (MdjCol * 2)()
    cols[0].dtype = 2
    cols[1].dtype = 1
    t = MdjTable(cols, 2, 0)
    k2 = (ctypes.c_int32 * 2)(0, 1)
    dup = (ctypes.c_int32 * 2)(0, 0)
    out_of_range = (ctypes.c_int32 * 2)(0, 5)
    assert lib.mdj_merge_multi(ctypes.byref(t), k2, ctypes.byref(t), k2, 0, 8, None, None, ctypes.byref(res)) == -1
    assert lib.mdj_merge_multi(ctypes.byref(t), k2, ctypes.byref(t), k2, 9, 8, None, None, ctypes.byref(res)) == -1
    assert lib.mdj_merge_multi(ctypes.byref(t), dup, ctypes.byref(t), k2, 2, 8, None, None, ctypes.byref(res)) == -1
    assert lib.mdj_merge_multi(ctypes.byref(t), k2, ctypes.byref(t), out_of_range, 2, 8, None, None,
                               ctypes.byref(res)) == -1
    swapped = (ctypes.c_int32 * 2)(1, 0)  # I64 against I32
    assert lib.mdj_merge_multi(ctypes.byref(t), k2, ctypes.byref(t), swapped, 2, 8, None, None,
                               ctypes.byref(res)) == -1
    fcols = (MdjCol * 2)()
    fcols[0].dtype = 4
    fcols[1].dtype = 1
    ft = MdjTable(fcols, 2, 0)
    assert lib.mdj_merge_multi(ctypes.byref(ft), k2, ctypes.byref(ft), k2, 2, 8, None, None, ctypes.byref(res)) == -2


def test_binding_rejects_bad_arguments_before_device_work(lib):
    import torch
    from paper_2101_08878_gb300 import mdj
    k = torch.arange(10, dtype=torch.int64)
    p = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError):
        mdj.MergeStream([k, p], [k, p], 8, how="sideways")
    with pytest.raises(ValueError):
        mdj.merge_host_chunked([k, p], [k, p], 8, 1 << 30, how="sideways")
    with pytest.raises(ValueError):
        mdj.transpose_add(torch.zeros((4, 4), dtype=torch.float64))   # not a CUDA tensor
    with pytest.raises(ValueError):
        mdj.mdj_merge_multi([k, p], [k, p], [0], [0], 8)              # not CUDA tensors
    assert mdj.HOW == {"inner": 0, "left": 1, "right": 2, "outer": 3}
    assert mdj.NO_ROW == 0xFFFFFFFF


def test_compaction_position_width_gate(tmp_path):
    # The key-tuple merge drops hash-collision candidates by a scan of m + 1
    # keep flags; 32-bit positions must give way to 64-bit ones before the
    # kept total can pass 2^32 - 1.  The gate is plain C++ (mdj_sizes.h), so it
    # is compiled and checked here with the host compiler.
    import shutil
    import subprocess
    if not shutil.which("g++"):
        pytest.skip("no host C++ compiler")
    src = tmp_path / "gate.cc"
    src.write_text(
        '#include "mdj_sizes.h"\n#include <stdio.h>\n'
        'int main() {\n'
        '  const unsigned long long m[] = {0ull, 1ull, 4294967293ull, 4294967294ull, 4294967295ull, 1ull << 40};\n'
        '  for (unsigned long long v : m) printf("%d\\n", (int)mdj::compaction_needs_u64_positions(v));\n'
        '  return 0;\n}\n')
    exe = tmp_path / "gate"
    csrc = os.path.join(ROOT, "paper_2101_08878_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17", "-I", csrc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    # 32-bit positions while the scan covers at most 2^32 - 1 flags
    assert out == ["0", "0", "0", "0", "1", "1"]


def test_workspace_give_back_keeps_arena_chunks(tmp_path):
    # Workspace (the library's per-call device memory) carves small buffers out
    # of arena chunks; the first buffer of a chunk has the chunk's address, and
    # giving it back early must not free the chunk the later buffers live in.
    # Host code only: compiled with nvcc, run with a fake allocator that
    # tracks live blocks (no GPU).
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if not nvcc:
        pytest.skip("no nvcc")
    csrc = os.path.join(ROOT, "paper_2101_08878_gb300", "csrc")
    src = tmp_path / "ws_test.cu"
    src.write_text(
        '#include <stdio.h>\n#include <set>\n#include "mdj_internal.cuh"\n'
        'static std::set<void *> live;\n'
        'static void *fa(size_t b, void *, void *) { void *p = malloc(b); live.insert(p); return p; }\n'
        'static void fr(void *p, void *, void *) { live.erase(p); free(p); }\n'
        'int main() {\n'
        '  mdj_allocator a = {fa, fr, nullptr};\n'
        '  {\n'
        '    mdj::Workspace ws(&a, nullptr);\n'
        '    void *s1 = ws.get(64);\n'
        '    void *big = ws.get(4u << 20);\n'
        '    ws.give_back(s1);\n'
        '    void *s2 = ws.get(64);\n'
        '    printf("%d %d %d\\n", (int)live.size(), (int)live.count(s1), s2 != nullptr);\n'
        '    ws.give_back(big);\n'
        '    printf("%d\\n", (int)live.size());\n'
        '  }\n'
        '  printf("%d\\n", (int)live.size());\n'
        '  return 0;\n}\n')
    exe = tmp_path / "ws_test"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", csrc, str(src), os.path.join(csrc, "mdj_runtime.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    # chunk + large buffer live, the chunk (at s1's address) kept; then the
    # large buffer alone released; nothing left after the workspace
    assert out == ["2", "1", "1", "1", "0"]


def test_merge_multi_how_refuses_bad_arguments_before_device_work(lib):
    # an unknown join type, or no key columns, is refused before any device
    # work (the column pointers are stand-ins, never dereferenced)
    from paper_2101_08878_gb300.mdj import MdjCol, MdjResult, MdjTable
    cols = (MdjCol * 2)()
    cols[0].data = ctypes.c_void_p(0x1000)
    cols[0].dtype = 2
    cols[1].data = ctypes.c_void_p(0x2000)
    cols[1].dtype = 4
    tab = MdjTable(cols, 2, 1000)
    keys = (ctypes.c_int32 * 1)(0)
    out = MdjResult()
    for how in (-1, 4, 99):
        assert lib.mdj_merge_multi_how(ctypes.byref(tab), keys, ctypes.byref(tab), keys, 1, 8, how, None, None,
                                       ctypes.byref(out)) == -1
    assert lib.mdj_merge_multi_how(ctypes.byref(tab), keys, ctypes.byref(tab), keys, 0, 8, 3, None, None,
                                   ctypes.byref(out)) == -1
    assert out.nrows == 0


def test_noalloc_size_limit_at_p8(lib):
    # mdj_partition_noalloc's fixed array holds P*T + ceil(P*T/4096) + P + 1
    # words (T = ceil(nrows / 4096)) of 4 Mi; at P = 8 that admits
    # 2,146,951,168 rows.  One row more is refused before any device work, so
    # the call needs no GPU and no buffers of that size (the pointers below are
    # never dereferenced).
    from paper_2101_08878_gb300.mdj import MdjCol, MdjTable

    def words(n, P):
        nh = P * ((n + 4095) // 4096)
        return nh + (nh + 4095) // 4096 + P + 1

    limit = 2_146_951_168
    assert words(limit, 8) <= 4 << 20 < words(limit + 1, 8)
    cols = (MdjCol * 2)()
    cols[0].data = ctypes.c_void_p(0x1000)  # stand-ins: refused before use
    cols[0].dtype = 2
    cols[1].data = ctypes.c_void_p(0x2000)
    cols[1].dtype = 4
    outs = (ctypes.c_void_p * 2)(0x3000, 0x4000)
    off = ctypes.c_void_p(0x5000)
    over = MdjTable(cols, 2, limit + 1)
    assert lib.mdj_partition_noalloc(ctypes.byref(over), 0, 8, outs, None, off, None) == -3
    assert lib.mdj_partition_noalloc(ctypes.byref(MdjTable(cols, 2, 16_764_929)), 0, 1024, outs, None, off,
                                     None) == -3
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        return  # below the limit the call would start device work on the stand-in pointers
    # with no device, a size inside the limit gets past the gate and stops at
    # the first CUDA call instead
    fits = MdjTable(cols, 2, limit)
    assert lib.mdj_partition_noalloc(ctypes.byref(fits), 0, 8, outs, None, off, None) == -5
