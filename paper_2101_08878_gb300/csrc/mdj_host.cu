// The merge of host-resident tables larger than device memory, streamed
// through the device in bounded pieces.  The paper's runtime splits messages
// larger than MPI's 2 GB count limit into 1 GB chunks (Sec. IV-B); on one
// GPU the same bound applies to the tables themselves.
//
// Phase 1, per side: the host table goes to the device chunk by chunk, each
// chunk is hash partitioned into B buckets (mdj_partition: h mod B, stable),
// and each bucket's slice returns to host storage with the rows' global row
// ids.  Equal keys land in the same bucket on both sides.
// Phase 2, per bucket: both sides' bucket b go to the device, their merge is
// opened as a stream (mdj_stream_open, any join type), and its rows are
// written window by window into one device buffer; each window's row ids are
// mapped back to the input tables and handed to the caller's sink.
//
// B and the chunk and window sizes come from the caller's device budget, so
// device memory stays bounded whatever the table sizes; a single key whose
// rows exceed a bucket's share of the budget gives MDJ_ERR_OOM.
#include <string.h>

#include <algorithm>
#include <vector>

#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr uint32_t kNoRow = 0xFFFFFFFFu;

// Bucket-local row ids of one window back to input row ids (kNoRow stays).
__global__ void k_map_rows(uint32_t *__restrict__ rows, uint64_t n, const uint32_t *__restrict__ global) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t r = rows[i];
    rows[i] = r == kNoRow ? kNoRow : global[r];
  }
}

// One side's buckets in host memory: per bucket, every column's bytes and
// the global row ids, in bucket order.
struct HostBuckets {
  std::vector<std::vector<std::vector<unsigned char>>> cols;  // [bucket][column]
  std::vector<std::vector<uint32_t>> rid;                     // [bucket]
};

// A device block for `bytes`, freed by the owning workspace.
unsigned char *dev_block(Workspace &ws, size_t bytes) { return (unsigned char *)ws.get(bytes ? bytes : 1); }

int partition_to_host(const mdj_table *t, int32_t key_col, uint32_t B, uint64_t chunk_rows, const mdj_allocator *alloc,
                      cudaStream_t s, HostBuckets *hb) {
  const int nc = t->ncols;
  int w[MDJ_MAX_COLS];
  for (int j = 0; j < nc; j++) w[j] = dtype_width(t->cols[j].dtype);
  hb->cols.assign(B, std::vector<std::vector<unsigned char>>(nc));
  hb->rid.assign(B, {});
  const uint64_t n = t->nrows;
  if (n == 0) return MDJ_OK;
  const uint64_t C = std::min<uint64_t>(chunk_rows, n);
  Workspace ws(alloc, s);
  unsigned char *din[MDJ_MAX_COLS], *dout[MDJ_MAX_COLS];
  for (int j = 0; j < nc; j++) {
    din[j] = dev_block(ws, C * w[j]);
    dout[j] = dev_block(ws, C * w[j]);
    if (!din[j] || !dout[j]) return MDJ_ERR_OOM;
  }
  uint32_t *drid = (uint32_t *)dev_block(ws, C * 4);
  int64_t *doff = (int64_t *)dev_block(ws, (size_t)(B + 1) * 8);
  if (!drid || !doff) return MDJ_ERR_OOM;
  std::vector<int64_t> off(B + 1);
  std::vector<uint32_t> rbuf;
  for (uint64_t c0 = 0; c0 < n; c0 += C) {
    const uint64_t cnt = std::min(C, n - c0);
    mdj_col cols[MDJ_MAX_COLS];
    void *outs[MDJ_MAX_COLS];
    for (int j = 0; j < nc; j++) {
      MDJ_CUDA_TRY(cudaMemcpyAsync(din[j], (const unsigned char *)t->cols[j].data + c0 * w[j], cnt * w[j],
                                   cudaMemcpyHostToDevice, s));
      cols[j].data = din[j];
      cols[j].dtype = t->cols[j].dtype;
      outs[j] = dout[j];
    }
    const mdj_table chunk = {cols, nc, cnt};
    MDJ_TRY(mdj_partition(&chunk, key_col, B, outs, drid, doff, alloc, s));
    MDJ_CUDA_TRY(cudaMemcpyAsync(off.data(), doff, (size_t)(B + 1) * 8, cudaMemcpyDeviceToHost, s));
    MDJ_CUDA_TRY(cudaStreamSynchronize(s));
    for (uint32_t b = 0; b < B; b++) {
      const uint64_t lo = (uint64_t)off[b], nb = (uint64_t)(off[b + 1] - off[b]);
      if (nb == 0) continue;
      for (int j = 0; j < nc; j++) {
        std::vector<unsigned char> &v = hb->cols[b][j];
        const size_t at = v.size();
        v.resize(at + nb * w[j]);
        MDJ_CUDA_TRY(cudaMemcpyAsync(v.data() + at, dout[j] + lo * w[j], nb * w[j], cudaMemcpyDeviceToHost, s));
      }
      rbuf.resize(nb);
      MDJ_CUDA_TRY(cudaMemcpyAsync(rbuf.data(), drid + lo, nb * 4, cudaMemcpyDeviceToHost, s));
      MDJ_CUDA_TRY(cudaStreamSynchronize(s));
      std::vector<uint32_t> &r = hb->rid[b];
      const size_t at = r.size();
      r.resize(at + nb);
      for (uint64_t i = 0; i < nb; i++) r[at + i] = rbuf[i] + (uint32_t)c0;  // chunk-local -> input row
    }
  }
  return MDJ_OK;
}

// Bucket b of one side on the device: every column and the global row ids.
int bucket_to_device(Workspace &ws, const mdj_table *t, const HostBuckets &hb, uint32_t b, mdj_col *cols,
                     mdj_table *out, uint32_t **rid) {
  const uint64_t nb = hb.rid[b].size();
  cudaStream_t s = ws.stream();
  for (int j = 0; j < t->ncols; j++) {
    const std::vector<unsigned char> &v = hb.cols[b][j];
    unsigned char *d = dev_block(ws, v.size());
    if (!d) return MDJ_ERR_OOM;
    if (!v.empty()) MDJ_CUDA_TRY(cudaMemcpyAsync(d, v.data(), v.size(), cudaMemcpyHostToDevice, s));
    cols[j].data = d;
    cols[j].dtype = t->cols[j].dtype;
  }
  *rid = (uint32_t *)dev_block(ws, nb * 4);
  if (!*rid) return MDJ_ERR_OOM;
  if (nb) MDJ_CUDA_TRY(cudaMemcpyAsync(*rid, hb.rid[b].data(), nb * 4, cudaMemcpyHostToDevice, s));
  *out = {cols, t->ncols, nb};
  return MDJ_OK;
}

// A whole host table on the device: one block and one copy per column.
int table_to_device(Workspace &ws, const mdj_table *t, mdj_col *cols, mdj_table *out) {
  for (int j = 0; j < t->ncols; j++) {
    const size_t bytes = t->nrows * (size_t)dtype_width(t->cols[j].dtype);
    unsigned char *d = dev_block(ws, bytes);
    if (!d) return MDJ_ERR_OOM;
    if (bytes) MDJ_CUDA_TRY(cudaMemcpyAsync(d, t->cols[j].data, bytes, cudaMemcpyHostToDevice, ws.stream()));
    cols[j].data = d;
    cols[j].dtype = t->cols[j].dtype;
  }
  *out = {cols, t->ncols, t->nrows};
  return MDJ_OK;
}

// Rows [q0, q0 + n) of a device result, as a piece pointing into it.
mdj_result result_piece(const mdj_result &r, uint64_t q0, uint64_t n) {
  mdj_result p = r;
  p.nrows = n;
  const int kw = dtype_width(r.key_dtype);
  if (r.key) p.key = (unsigned char *)r.key + q0 * kw;
  if (r.left_row) p.left_row = r.left_row + q0;
  if (r.right_row) p.right_row = r.right_row + q0;
  for (int j = 0; j < r.n_left_cols; j++)
    if (r.left_cols[j]) p.left_cols[j] = (unsigned char *)r.left_cols[j] + q0 * dtype_width(r.left_dtypes[j]);
  for (int j = 0; j < r.n_right_cols; j++)
    if (r.right_cols[j]) p.right_cols[j] = (unsigned char *)r.right_cols[j] + q0 * dtype_width(r.right_dtypes[j]);
  return p;
}

// Both tables fit one bucket of the budget: they go to the device once and
// are merged in place.  An inner merge runs mdj_merge and hands its result to
// the sink in windows that point into it; the other join types stream their
// rows through one window buffer.  Row ids are already input row ids.
int merge_resident(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P, int32_t how,
                   uint64_t window, mdj_sink sink, void *sink_ctx, const mdj_allocator *alloc, cudaStream_t s,
                   uint64_t *total_rows) {
  Workspace ws(alloc, s);
  mdj_col lc[MDJ_MAX_COLS], rc[MDJ_MAX_COLS];
  mdj_table lt, rt;
  MDJ_TRY(table_to_device(ws, left, lc, &lt));
  MDJ_TRY(table_to_device(ws, right, rc, &rt));
  uint64_t produced = 0;
  int rc2 = MDJ_OK;
  if (how == MDJ_INNER) {
    mdj_result res;
    MDJ_TRY(mdj_merge(&lt, lk, &rt, rk, P, alloc, (void *)s, &res));
    rc2 = cuda_status(cudaStreamSynchronize(s));
    for (uint64_t q0 = 0; q0 < res.nrows && rc2 == MDJ_OK; q0 += window) {
      const uint64_t n = std::min(window, res.nrows - q0);
      const mdj_result piece = result_piece(res, q0, n);
      if (sink(&piece, produced, sink_ctx) != 0) rc2 = MDJ_ERR_ABORTED;
      produced += n;
    }
    mdj_result_release(&res, alloc, (void *)s);
  } else {
    Workspace wbuf(alloc, s);
    mdj_result piece;
    memset(&piece, 0, sizeof piece);
    mdj_window win;
    memset(&win, 0, sizeof win);
    piece.key_dtype = left->cols[lk].dtype;
    win.key = piece.key = dev_block(wbuf, window * dtype_width(piece.key_dtype));
    win.left_row = piece.left_row = (uint32_t *)dev_block(wbuf, window * 4);
    win.right_row = piece.right_row = (uint32_t *)dev_block(wbuf, window * 4);
    if (!piece.key || !piece.left_row || !piece.right_row) return MDJ_ERR_OOM;
    for (int j = 0, c = 0; j < left->ncols; j++) {
      if (j == lk) continue;
      piece.left_dtypes[c] = left->cols[j].dtype;
      if (!(piece.left_cols[c] = win.left_cols[c] = dev_block(wbuf, window * dtype_width(left->cols[j].dtype))))
        return MDJ_ERR_OOM;
      piece.n_left_cols = ++c;
    }
    for (int j = 0, c = 0; j < right->ncols; j++) {
      if (j == rk) continue;
      piece.right_dtypes[c] = right->cols[j].dtype;
      if (!(piece.right_cols[c] = win.right_cols[c] = dev_block(wbuf, window * dtype_width(right->cols[j].dtype))))
        return MDJ_ERR_OOM;
      piece.n_right_cols = ++c;
    }
    mdj_stream *h = nullptr;
    uint64_t m = 0;
    MDJ_TRY(mdj_stream_open(&lt, lk, &rt, rk, P, how, alloc, (void *)s, &h, &m));
    for (uint64_t q0 = 0; q0 < m && rc2 == MDJ_OK; q0 += window) {
      const uint64_t n = std::min(window, m - q0);
      rc2 = mdj_stream_emit(h, q0, n, &win);
      if (rc2 == MDJ_OK) rc2 = cuda_status(cudaStreamSynchronize(s));
      if (rc2 != MDJ_OK) break;
      piece.nrows = n;
      if (sink(&piece, produced, sink_ctx) != 0) rc2 = MDJ_ERR_ABORTED;
      produced += n;
    }
    mdj_stream_close(h);
  }
  MDJ_TRY(rc2);
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  *total_rows = produced;
  return MDJ_OK;
}

uint64_t row_bytes(const mdj_table *t) {
  uint64_t b = 0;
  for (int j = 0; j < t->ncols; j++) b += dtype_width(t->cols[j].dtype);
  return b;
}

int merge_host_impl(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P, int32_t how,
                    uint64_t budget, mdj_sink sink, void *sink_ctx, const mdj_allocator *alloc, void *stream,
                    uint64_t *total_rows) {
  if (!total_rows || !sink) return MDJ_ERR_INVALID_ARG;
  *total_rows = 0;
  for (const mdj_table *t : {left, right}) {
    if (!t || !t->cols || t->ncols < 1 || t->ncols > MDJ_MAX_COLS) return MDJ_ERR_INVALID_ARG;
    if (t->nrows >= (1ull << 32)) return MDJ_ERR_TOO_LARGE;
    for (int j = 0; j < t->ncols; j++) {
      if (dtype_width(t->cols[j].dtype) == 0) return MDJ_ERR_UNSUPPORTED_DTYPE;
      if (t->nrows > 0 && !t->cols[j].data) return MDJ_ERR_INVALID_ARG;
    }
  }
  if (lk < 0 || lk >= left->ncols || rk < 0 || rk >= right->ncols) return MDJ_ERR_INVALID_ARG;
  const int32_t kd = left->cols[lk].dtype;
  if (kd != MDJ_I32 && kd != MDJ_I64) return MDJ_ERR_UNSUPPORTED_DTYPE;
  if (right->cols[rk].dtype != kd) return MDJ_ERR_INVALID_ARG;
  if (P < 1 || P > MDJ_MAX_PARTITIONS || how < MDJ_INNER || how > MDJ_OUTER) return MDJ_ERR_INVALID_ARG;
  if (budget < (64ull << 20)) return MDJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  // sizes from the budget: a bucket pair's rows (with row ids) take at most
  // a sixth of it (the stream open holds about four times its inputs), a
  // chunk of phase 1 a quarter, a window a sixth
  const uint64_t wl = row_bytes(left), wr = row_bytes(right);
  const uint64_t in_bytes = left->nrows * (wl + 4) + right->nrows * (wr + 4);
  uint64_t B = 1;
  while (B < MDJ_MAX_PARTITIONS && in_bytes > B * (budget / 6)) B *= 2;
  const uint64_t chunk_rows = std::max<uint64_t>(1, (budget / 4) / (2 * std::max(wl, wr) + 4));
  const uint64_t out_row = wl + wr + 8 - dtype_width(kd);  // key once, both row ids, every other column
  const uint64_t window = std::max<uint64_t>(1, (budget / 6) / out_row);

  if (B == 1) return merge_resident(left, lk, right, rk, P, how, window, sink, sink_ctx, alloc, s, total_rows);

  HostBuckets hl, hr;
  MDJ_TRY(partition_to_host(left, lk, (uint32_t)B, chunk_rows, alloc, s, &hl));
  MDJ_TRY(partition_to_host(right, rk, (uint32_t)B, chunk_rows, alloc, s, &hr));

  Workspace wbuf(alloc, s);  // one window, reused by every bucket
  mdj_result piece;
  memset(&piece, 0, sizeof piece);
  piece.key_dtype = kd;
  const int kw = dtype_width(kd);
  piece.key = dev_block(wbuf, window * kw);
  piece.left_row = (uint32_t *)dev_block(wbuf, window * 4);
  piece.right_row = (uint32_t *)dev_block(wbuf, window * 4);
  if (!piece.key || !piece.left_row || !piece.right_row) return MDJ_ERR_OOM;
  mdj_window win;
  memset(&win, 0, sizeof win);
  win.key = piece.key;
  win.left_row = piece.left_row;
  win.right_row = piece.right_row;
  for (int j = 0, c = 0; j < left->ncols; j++) {
    if (j == lk) continue;
    piece.left_dtypes[c] = left->cols[j].dtype;
    if (!(piece.left_cols[c] = win.left_cols[c] = dev_block(wbuf, window * dtype_width(left->cols[j].dtype))))
      return MDJ_ERR_OOM;
    piece.n_left_cols = ++c;
  }
  for (int j = 0, c = 0; j < right->ncols; j++) {
    if (j == rk) continue;
    piece.right_dtypes[c] = right->cols[j].dtype;
    if (!(piece.right_cols[c] = win.right_cols[c] = dev_block(wbuf, window * dtype_width(right->cols[j].dtype))))
      return MDJ_ERR_OOM;
    piece.n_right_cols = ++c;
  }

  const bool keep_left = how == MDJ_LEFT || how == MDJ_OUTER, keep_right = how == MDJ_RIGHT || how == MDJ_OUTER;
  // Every row of bucket b has h mod B = b.  For a power-of-two P <= B that
  // fixes h mod P = b mod P too, so all of a bucket's rows would fall in one of
  // its P partitions; such buckets are merged with one partition instead (the
  // merge's own sub-buckets come from the high hash bits, so the work still
  // spreads over the device).  The joined rows do not depend on P.
  const uint32_t Pb = ((P & (P - 1)) == 0 && (uint64_t)P <= B) ? 1u : P;
  uint64_t produced = 0;
  for (uint32_t b = 0; b < B; b++) {
    const uint64_t nl = hl.rid[b].size(), nr = hr.rid[b].size();
    if (!((nl && nr) || (nl && keep_left) || (nr && keep_right))) continue;
    Workspace ws(alloc, s);  // this bucket's tables, released before the next bucket
    mdj_col lc[MDJ_MAX_COLS], rc[MDJ_MAX_COLS];
    mdj_table lt, rt;
    uint32_t *lrid, *rrid;
    MDJ_TRY(bucket_to_device(ws, left, hl, b, lc, &lt, &lrid));
    MDJ_TRY(bucket_to_device(ws, right, hr, b, rc, &rt, &rrid));
    mdj_stream *h = nullptr;
    uint64_t m = 0;
    MDJ_TRY(mdj_stream_open(&lt, lk, &rt, rk, Pb, how, alloc, stream, &h, &m));
    int rc2 = MDJ_OK;
    for (uint64_t q0 = 0; q0 < m && rc2 == MDJ_OK; q0 += window) {
      const uint64_t n = std::min(window, m - q0);
      rc2 = mdj_stream_emit(h, q0, n, &win);
      if (rc2 != MDJ_OK) break;
      const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms() * 8);
      k_map_rows<<<grid, 256, 0, s>>>(piece.left_row, n, lrid);
      k_map_rows<<<grid, 256, 0, s>>>(piece.right_row, n, rrid);
      rc2 = cuda_status(cudaGetLastError());
      if (rc2 == MDJ_OK) rc2 = cuda_status(cudaStreamSynchronize(s));
      if (rc2 != MDJ_OK) break;
      piece.nrows = n;
      if (sink(&piece, produced, sink_ctx) != 0) rc2 = MDJ_ERR_ABORTED;
      produced += n;
    }
    mdj_stream_close(h);
    MDJ_TRY(rc2);
  }
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  *total_rows = produced;
  return MDJ_OK;
}

}  // namespace
}  // namespace mdj

extern "C" int mdj_merge_host(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
                              uint32_t P, int32_t how, uint64_t device_budget, mdj_sink sink, void *sink_ctx,
                              const mdj_allocator *alloc, void *stream, uint64_t *total_rows) {
  return mdj::merge_host_impl(left, left_key, right, right_key, P, how, device_budget, sink, sink_ctx, alloc, stream,
                              total_rows);
}
