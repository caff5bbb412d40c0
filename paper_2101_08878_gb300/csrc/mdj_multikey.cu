// The merge on several key columns (a merge variant: keys that are tuples).
//
// Each row's key tuple becomes one 64-bit surrogate, a hash of the columns'
// bits; the merge of mdj_merge runs on the surrogates, carrying the real key
// columns along as payloads; every candidate row then compares the two
// sides' key tuples column by column and rows whose tuples differ (hash
// collisions) are dropped.  Equal tuples always have equal surrogates, so no
// pair is lost, and the comparison removes every false one: the result is
// exactly the inner equi-join on all key columns.
#include <stdlib.h>
#include <string.h>

#include "mdj_internal.cuh"
#include "mdj_sizes.h"

namespace mdj {
namespace {

constexpr int kMaxKeys = 8;

struct KeyCols {
  const void *col[kMaxKeys];
  int32_t width[kMaxKeys];
  int32_t n;
};

__device__ __forceinline__ uint64_t col_bits(const void *c, int width, uint64_t i) {
  return width == 8 ? ((const uint64_t *)c)[i] : (uint64_t)((const uint32_t *)c)[i];
}

// Surrogate of row i: fmix64 chained over the key columns' bits (each column
// mixed with its position so that permuted tuples differ).  weak = 1 (test
// hook) uses the first column's bits alone, so that distinct tuples collide.
__global__ void k_tuple_hash(const __grid_constant__ KeyCols K, uint64_t n, int weak, uint64_t *__restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t h = 0x243F6A8885A308D3ULL;
    if (weak) {
      h = col_bits(K.col[0], K.width[0], i);
    } else {
      for (int j = 0; j < K.n; j++)
        h = fmix64(h ^ fmix64(col_bits(K.col[j], K.width[j], i) + 0x9E3779B97F4A7C15ULL * (j + 1)));
    }
    out[i] = h;
  }
}

// keep[i] = 1 if candidate row i's left and right key tuples are equal;
// *dropped counts the others.
__global__ void k_verify(const __grid_constant__ KeyCols Lk, const __grid_constant__ KeyCols Rk, uint64_t m,
                         uint32_t *__restrict__ keep, unsigned long long *dropped) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long local = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    bool eq = true;
    for (int j = 0; j < Lk.n; j++)
      eq = eq && col_bits(Lk.col[j], Lk.width[j], i) == col_bits(Rk.col[j], Rk.width[j], i);
    keep[i] = eq;
    local += !eq;
  }
  local = warp_sum(local);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(dropped, local);
}

// Rows with keep[i] move to position pos[i] (exclusive scan of keep).
template <typename PosT>
__global__ void k_compact_col(const void *__restrict__ src, void *__restrict__ dst, int width, uint64_t m,
                              const uint32_t *__restrict__ keep, const PosT *__restrict__ pos) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    if (!keep[i]) continue;
    if (width == 8)
      ((uint64_t *)dst)[pos[i]] = ((const uint64_t *)src)[i];
    else
      ((uint32_t *)dst)[pos[i]] = ((const uint32_t *)src)[i];
  }
}

__global__ void k_flags_u64(const uint32_t *__restrict__ keep, uint64_t m, uint64_t *__restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += stride) out[i] = i < m ? keep[i] : 0;
}

int weak_hash_for_tests() {
  const char *e = getenv("MDJ_TEST_WEAK_TUPLE_HASH");
  return e && e[0] == '1';
}

unsigned grid_of(uint64_t n) {
  const uint64_t g = (n + 255) / 256, most = (uint64_t)num_sms() * 8;
  return (unsigned)(g < 1 ? 1 : (g < most ? g : most));
}

int check_side(const mdj_table *t, const int32_t *keys, int32_t nkeys) {
  if (!t || !t->cols || t->ncols < 1 || t->ncols + 1 > MDJ_MAX_COLS) return MDJ_ERR_INVALID_ARG;
  if (t->nrows >= (1ull << 32)) return MDJ_ERR_TOO_LARGE;
  for (int j = 0; j < t->ncols; j++) {
    if (dtype_width(t->cols[j].dtype) == 0) return MDJ_ERR_UNSUPPORTED_DTYPE;
    if (t->nrows > 0 && !t->cols[j].data) return MDJ_ERR_INVALID_ARG;
  }
  for (int a = 0; a < nkeys; a++) {
    if (keys[a] < 0 || keys[a] >= t->ncols) return MDJ_ERR_INVALID_ARG;
    for (int b = 0; b < a; b++)
      if (keys[a] == keys[b]) return MDJ_ERR_INVALID_ARG;
    const int32_t d = t->cols[keys[a]].dtype;
    if (d != MDJ_I32 && d != MDJ_I64 && d != MDJ_U32 && d != MDJ_U64) return MDJ_ERR_UNSUPPORTED_DTYPE;
  }
  return MDJ_OK;
}

bool is_key(const int32_t *keys, int32_t nkeys, int j) {
  for (int a = 0; a < nkeys; a++)
    if (keys[a] == j) return true;
  return false;
}

int merge_multi_impl(const mdj_table *left, const int32_t *lkeys, const mdj_table *right, const int32_t *rkeys,
                     int32_t nkeys, uint32_t P, const mdj_allocator *alloc, void *stream, mdj_result *out) {
  if (!out || !lkeys || !rkeys || nkeys < 1 || nkeys > kMaxKeys) return MDJ_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  MDJ_TRY(check_side(left, lkeys, nkeys));
  MDJ_TRY(check_side(right, rkeys, nkeys));
  for (int a = 0; a < nkeys; a++)
    if (left->cols[lkeys[a]].dtype != right->cols[rkeys[a]].dtype) return MDJ_ERR_INVALID_ARG;
  if (P < 1 || P > MDJ_MAX_PARTITIONS) return MDJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws(alloc, s);

  // surrogate keys, then tables (surrogate, key columns, other columns)
  mdj_col lc[MDJ_MAX_COLS], rc[MDJ_MAX_COLS];
  const mdj_table *sides[2] = {left, right};
  const int32_t *keys[2] = {lkeys, rkeys};
  mdj_col *cols[2] = {lc, rc};
  mdj_table tabs[2];
  const int weak = weak_hash_for_tests();
  for (int side = 0; side < 2; side++) {
    const mdj_table *t = sides[side];
    uint64_t *sur = (uint64_t *)ws.get((size_t)(t->nrows ? t->nrows : 1) * 8);
    if (!sur) return MDJ_ERR_OOM;
    KeyCols K;
    memset(&K, 0, sizeof K);
    K.n = nkeys;
    for (int a = 0; a < nkeys; a++) {
      K.col[a] = t->cols[keys[side][a]].data;
      K.width[a] = dtype_width(t->cols[keys[side][a]].dtype);
    }
    if (t->nrows) {
      TraceScope tr("tuple_hash", s);
      k_tuple_hash<<<grid_of(t->nrows), 256, 0, s>>>(K, t->nrows, weak, sur);
    }
    MDJ_LAUNCH_CHECK();
    int c = 0;
    cols[side][c++] = {sur, MDJ_I64};
    for (int a = 0; a < nkeys; a++) cols[side][c++] = t->cols[keys[side][a]];
    for (int j = 0; j < t->ncols; j++)
      if (!is_key(keys[side], nkeys, j)) cols[side][c++] = t->cols[j];
    tabs[side] = {cols[side], c, t->nrows};
  }
  mdj_result cand;
  MDJ_TRY(mdj_merge(&tabs[0], 0, &tabs[1], 0, P, alloc, stream, &cand));
  // candidate columns: left_cols = [left keys..., left others...],
  // right_cols = [right keys..., right others...]; the key is the surrogate
  const uint64_t m = cand.nrows;
  uint32_t *keep = m ? (uint32_t *)ws.get((size_t)(m + 1) * 4) : nullptr;
  unsigned long long *dropped = (unsigned long long *)ws.get(8);
  int rc2 = (m && !keep) || !dropped ? MDJ_ERR_OOM : MDJ_OK;
  unsigned long long host_dropped = 0;
  if (rc2 == MDJ_OK && m) {
    KeyCols Lk, Rk;
    memset(&Lk, 0, sizeof Lk);
    memset(&Rk, 0, sizeof Rk);
    Lk.n = Rk.n = nkeys;
    for (int a = 0; a < nkeys; a++) {
      Lk.col[a] = cand.left_cols[a];
      Lk.width[a] = dtype_width(cand.left_dtypes[a]);
      Rk.col[a] = cand.right_cols[a];
      Rk.width[a] = dtype_width(cand.right_dtypes[a]);
    }
    rc2 = cuda_status(cudaMemsetAsync(dropped, 0, 8, s));
    if (rc2 == MDJ_OK) {
      TraceScope tr("tuple_verify", s);
      k_verify<<<grid_of(m), 256, 0, s>>>(Lk, Rk, m, keep, dropped);
      rc2 = cuda_status(cudaGetLastError());
    }
    if (rc2 == MDJ_OK) rc2 = cuda_status(cudaMemcpyAsync(&host_dropped, dropped, 8, cudaMemcpyDeviceToHost, s));
    if (rc2 == MDJ_OK) rc2 = cuda_status(cudaStreamSynchronize(s));
  }
  if (rc2 != MDJ_OK) {
    mdj_result_release(&cand, alloc, stream);
    return rc2;
  }
  // the result: row ids, the left key and other columns, the right others
  mdj_result r;
  memset(&r, 0, sizeof r);
  r.key_dtype = 0;
  r.n_left_cols = cand.n_left_cols;
  for (int j = 0; j < cand.n_left_cols; j++) r.left_dtypes[j] = cand.left_dtypes[j];
  r.n_right_cols = cand.n_right_cols - nkeys;
  for (int j = 0; j < r.n_right_cols; j++) r.right_dtypes[j] = cand.right_dtypes[nkeys + j];
  if (host_dropped == 0) {  // every candidate stands: keep its buffers
    r.nrows = m;
    r.left_row = cand.left_row;
    r.right_row = cand.right_row;
    for (int j = 0; j < r.n_left_cols; j++) r.left_cols[j] = cand.left_cols[j];
    for (int j = 0; j < r.n_right_cols; j++) r.right_cols[j] = cand.right_cols[nkeys + j];
    if (cand.key) ws.release_caller(cand.key);
    for (int a = 0; a < nkeys; a++)
      if (cand.right_cols[a]) ws.release_caller(cand.right_cols[a]);
    *out = r;
    return MDJ_OK;
  }
  // drop the colliding rows: positions by a scan of keep (64-bit positions
  // once m + 1 flags no longer fit a 32-bit total), then each column
  const bool wide = compaction_needs_u64_positions(m);
  uint32_t *pos = nullptr;
  uint64_t *pos64 = nullptr;
  if (wide) {
    pos64 = (uint64_t *)ws.get((size_t)(m + 1) * 8);
    rc2 = pos64 ? MDJ_OK : MDJ_ERR_OOM;
    if (rc2 == MDJ_OK) {
      TraceScope tr("tuple_flags_u64", s);
      k_flags_u64<<<grid_of(m + 1), 256, 0, s>>>(keep, m, pos64);
      rc2 = cuda_status(cudaGetLastError());
    }
    if (rc2 == MDJ_OK) rc2 = exclusive_scan_u64(ws, pos64, pos64, (size_t)m + 1);
  } else {
    pos = (uint32_t *)ws.get((size_t)(m + 1) * 4);
    rc2 = pos ? MDJ_OK : MDJ_ERR_OOM;
    if (rc2 == MDJ_OK) rc2 = cuda_status(cudaMemsetAsync(keep + m, 0, 4, s));
    if (rc2 == MDJ_OK) rc2 = exclusive_scan_u32(ws, keep, pos, (size_t)m + 1);
  }
  const uint64_t kept = m - host_dropped;
  r.nrows = kept;
  auto move = [&](const void *src, int width, void **dst) -> int {
    *dst = kept ? ws.get_owned_by_caller((size_t)kept * width) : nullptr;
    if (kept && !*dst) return MDJ_ERR_OOM;
    if (kept) {
      TraceScope tr("tuple_compact", s);
      if (wide)
        k_compact_col<uint64_t><<<grid_of(m), 256, 0, s>>>(src, *dst, width, m, keep, pos64);
      else
        k_compact_col<uint32_t><<<grid_of(m), 256, 0, s>>>(src, *dst, width, m, keep, pos);
    }
    return cuda_status(cudaGetLastError());
  };
  if (rc2 == MDJ_OK) rc2 = move(cand.left_row, 4, (void **)&r.left_row);
  if (rc2 == MDJ_OK) rc2 = move(cand.right_row, 4, (void **)&r.right_row);
  for (int j = 0; rc2 == MDJ_OK && j < r.n_left_cols; j++)
    rc2 = move(cand.left_cols[j], dtype_width(r.left_dtypes[j]), &r.left_cols[j]);
  for (int j = 0; rc2 == MDJ_OK && j < r.n_right_cols; j++)
    rc2 = move(cand.right_cols[nkeys + j], dtype_width(r.right_dtypes[j]), &r.right_cols[j]);
  mdj_result_release(&cand, alloc, stream);
  if (rc2 != MDJ_OK) {
    mdj_result_release(&r, alloc, stream);
    return rc2;
  }
  *out = r;
  return MDJ_OK;
}

// ------------------------------------------------ outer joins on tuples
//
// The inner merge's verified pairs mark the rows they use; the rows of a kept
// side that no pair uses follow the pairs, each once, with its own row id,
// NO_ROW for the other side and zeroed columns for it, and the key columns
// filled from the present side's tuple.

constexpr uint32_t kNoRowId = 0xFFFFFFFFu;

// flag[rows[i]] = 1 for every pair i (plain stores; equal values race benignly).
__global__ void k_mark_rows(const uint32_t *__restrict__ rows, uint64_t m, uint32_t *__restrict__ flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) flag[rows[i]] = 1u;
}

// flag[i] = 1 for the rows no pair used (i < n), flag[n] = 0: the scan input
// of their output positions.
__global__ void k_unmarked(uint32_t *__restrict__ flag, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride)
    flag[i] = i < n ? (flag[i] ^ 1u) : 0u;
}

struct EmitCols {
  const void *src[2 * MDJ_MAX_COLS];  // NULL: zero for these rows
  void *dst[2 * MDJ_MAX_COLS];
  int32_t width[2 * MDJ_MAX_COLS];
  int32_t n;
};

// Unmatched row i (pos[i + 1] != pos[i]) goes to base + pos[i].
__global__ void k_emit_unmatched(const uint32_t *__restrict__ pos, uint64_t n, uint64_t base,
                                 uint32_t *__restrict__ own_row, uint32_t *__restrict__ other_row,
                                 const __grid_constant__ EmitCols C) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t p = pos[i];
    if (pos[i + 1] == p) continue;
    const uint64_t o = base + p;
    own_row[o] = (uint32_t)i;
    other_row[o] = kNoRowId;
    for (int c = 0; c < C.n; c++) {
      if (C.width[c] == 8)
        ((uint64_t *)C.dst[c])[o] = C.src[c] ? ((const uint64_t *)C.src[c])[i] : 0ull;
      else
        ((uint32_t *)C.dst[c])[o] = C.src[c] ? ((const uint32_t *)C.src[c])[i] : 0u;
    }
  }
}

int merge_multi_how_impl(const mdj_table *left, const int32_t *lkeys, const mdj_table *right, const int32_t *rkeys,
                         int32_t nkeys, uint32_t P, int32_t how, const mdj_allocator *alloc, void *stream,
                         mdj_result *out) {
  if (how < MDJ_INNER || how > MDJ_OUTER) return MDJ_ERR_INVALID_ARG;
  mdj_result in;
  MDJ_TRY(merge_multi_impl(left, lkeys, right, rkeys, nkeys, P, alloc, stream, &in));
  if (how == MDJ_INNER) {
    *out = in;
    return MDJ_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Workspace ws(alloc, s);
  const bool keep_l = how == MDJ_LEFT || how == MDJ_OUTER, keep_r = how == MDJ_RIGHT || how == MDJ_OUTER;
  const uint64_t m = in.nrows;
  // unmatched rows of each kept side: marks, then positions by a scan
  uint32_t *pos[2] = {nullptr, nullptr};
  uint64_t cnt[2] = {0, 0};
  int rc = MDJ_OK;
  for (int side = 0; side < 2 && rc == MDJ_OK; side++) {
    if (!(side == 0 ? keep_l : keep_r)) continue;
    const uint64_t n = side == 0 ? left->nrows : right->nrows;
    uint32_t *flag = (uint32_t *)ws.get((size_t)(n + 1) * 4);
    pos[side] = (uint32_t *)ws.get((size_t)(n + 1) * 4);
    if (!flag || !pos[side]) rc = MDJ_ERR_OOM;
    if (rc == MDJ_OK) rc = cuda_status(cudaMemsetAsync(flag, 0, (size_t)(n + 1) * 4, s));
    if (rc == MDJ_OK && m) {
      TraceScope tr("tuple_mark", s);
      k_mark_rows<<<grid_of(m), 256, 0, s>>>(side == 0 ? in.left_row : in.right_row, m, flag);
      rc = cuda_status(cudaGetLastError());
    }
    if (rc == MDJ_OK) {
      k_unmarked<<<grid_of(n + 1), 256, 0, s>>>(flag, n);
      rc = cuda_status(cudaGetLastError());
    }
    if (rc == MDJ_OK) rc = exclusive_scan_u32(ws, flag, pos[side], (size_t)n + 1);
    uint32_t host_cnt = 0;
    if (rc == MDJ_OK) rc = cuda_status(cudaMemcpyAsync(&host_cnt, pos[side] + n, 4, cudaMemcpyDeviceToHost, s));
    if (rc == MDJ_OK) rc = cuda_status(cudaStreamSynchronize(s));
    cnt[side] = host_cnt;
  }
  // the result: the pairs, then left-only rows, then right-only rows
  mdj_result r;
  memset(&r, 0, sizeof r);
  r.key_dtype = 0;
  r.n_left_cols = in.n_left_cols;
  r.n_right_cols = in.n_right_cols;
  for (int j = 0; j < r.n_left_cols; j++) r.left_dtypes[j] = in.left_dtypes[j];
  for (int j = 0; j < r.n_right_cols; j++) r.right_dtypes[j] = in.right_dtypes[j];
  const uint64_t M = m + cnt[0] + cnt[1];
  r.nrows = M;
  auto alloc_copy = [&](void **dst, const void *src, int width) -> int {
    *dst = M ? ws.get_owned_by_caller((size_t)M * width) : nullptr;
    if (M && !*dst) return MDJ_ERR_OOM;
    if (m) return cuda_status(cudaMemcpyAsync(*dst, src, (size_t)m * width, cudaMemcpyDeviceToDevice, s));
    return MDJ_OK;
  };
  if (rc == MDJ_OK) rc = alloc_copy((void **)&r.left_row, in.left_row, 4);
  if (rc == MDJ_OK) rc = alloc_copy((void **)&r.right_row, in.right_row, 4);
  for (int j = 0; rc == MDJ_OK && j < r.n_left_cols; j++)
    rc = alloc_copy(&r.left_cols[j], in.left_cols[j], dtype_width(r.left_dtypes[j]));
  for (int j = 0; rc == MDJ_OK && j < r.n_right_cols; j++)
    rc = alloc_copy(&r.right_cols[j], in.right_cols[j], dtype_width(r.right_dtypes[j]));
  // source columns of the output, side by side: left output column c is the
  // left table's column lsrc[c] (keys in lkeys order, then the others); right
  // output column c is the right table's column rsrc[c]
  int lsrc[MDJ_MAX_COLS], rsrc[MDJ_MAX_COLS];
  {
    int c = 0;
    for (int a = 0; a < nkeys; a++) lsrc[c++] = lkeys[a];
    for (int j = 0; j < left->ncols; j++)
      if (!is_key(lkeys, nkeys, j)) lsrc[c++] = j;
    c = 0;
    for (int j = 0; j < right->ncols; j++)
      if (!is_key(rkeys, nkeys, j)) rsrc[c++] = j;
  }
  for (int side = 0; side < 2 && rc == MDJ_OK; side++) {
    if (!cnt[side]) continue;
    EmitCols C;
    memset(&C, 0, sizeof C);
    for (int c = 0; c < r.n_left_cols; c++) {
      C.dst[C.n] = r.left_cols[c];
      C.width[C.n] = dtype_width(r.left_dtypes[c]);
      if (side == 0)
        C.src[C.n] = left->cols[lsrc[c]].data;
      else
        C.src[C.n] = c < nkeys ? right->cols[rkeys[c]].data : nullptr;  // the right row's tuple
      C.n++;
    }
    for (int c = 0; c < r.n_right_cols; c++) {
      C.dst[C.n] = r.right_cols[c];
      C.width[C.n] = dtype_width(r.right_dtypes[c]);
      C.src[C.n] = side == 1 ? right->cols[rsrc[c]].data : nullptr;
      C.n++;
    }
    const uint64_t n = side == 0 ? left->nrows : right->nrows;
    const uint64_t base = side == 0 ? m : m + cnt[0];
    TraceScope tr("tuple_unmatched", s);
    k_emit_unmatched<<<grid_of(n), 256, 0, s>>>(pos[side], n, base, side == 0 ? r.left_row : r.right_row,
                                                side == 0 ? r.right_row : r.left_row, C);
    rc = cuda_status(cudaGetLastError());
  }
  if (rc == MDJ_OK) rc = cuda_status(cudaStreamSynchronize(s));
  mdj_result_release(&in, alloc, stream);
  if (rc != MDJ_OK) {
    mdj_result_release(&r, alloc, stream);
    return rc;
  }
  *out = r;
  return MDJ_OK;
}

}  // namespace
}  // namespace mdj

extern "C" int mdj_merge_multi_how(const mdj_table *left, const int32_t *left_keys, const mdj_table *right,
                                   const int32_t *right_keys, int32_t nkeys, uint32_t P, int32_t how,
                                   const mdj_allocator *alloc, void *stream, mdj_result *out) {
  if (out) memset(out, 0, sizeof *out);
  return mdj::merge_multi_how_impl(left, left_keys, right, right_keys, nkeys, P, how, alloc, stream, out);
}

extern "C" int mdj_merge_multi(const mdj_table *left, const int32_t *left_keys, const mdj_table *right,
                               const int32_t *right_keys, int32_t nkeys, uint32_t P, const mdj_allocator *alloc,
                               void *stream, mdj_result *out) {
  return mdj::merge_multi_impl(left, left_keys, right, right_keys, nkeys, P, alloc, stream, out);
}
