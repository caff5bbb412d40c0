// The merge of host-resident tables larger than device memory, streamed
// through the device in bounded pieces.  The paper's runtime splits messages
// larger than MPI's 2 GB count limit into 1 GB chunks (Sec. IV-B); on one
// GPU the same bound applies to the tables themselves.
//
// Phase 1, per side: the host table goes to the device chunk by chunk, each
// chunk is hash partitioned into B buckets (mdj_partition: h mod B, stable),
// its row ids are made input row ids, and the partitioned chunk returns to
// a host staging area (one array per column, chunks in order) with its
// bucket offsets.  Chunk c's copy back runs on a second stream while chunk
// c + 1 is copied in and partitioned (two output buffer sets; every
// allocation stays on the caller's stream).
// Phase 2, per bucket: both sides' bucket b (its slice of every chunk) go to
// the device, their merge is opened as a stream (mdj_stream_open, any join
// type), and its rows are written window by window into one device buffer;
// each window's row ids are mapped back to the input tables and handed to the
// caller's sink.  Equal keys land in the same bucket on both sides.
//
// Host <-> device movement: where the device reads and writes pageable host
// memory through the host's page tables (a coherent CPU-GPU link), copies run
// as kernels, which never block the host thread and gather many slices per
// launch; elsewhere they are cudaMemcpyAsync calls.  The staging area's pages
// are touched by host threads before the device writes them (a device write
// that faults a page in costs far more than a host first touch).
//
// B and the chunk and window sizes come from the caller's device budget, so
// device memory stays bounded whatever the table sizes; a single key whose
// rows exceed a bucket's share of the budget gives MDJ_ERR_OOM.
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <thread>
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

// Chunk-local row ids to input row ids.
__global__ void k_add_rows(uint32_t *__restrict__ rows, uint64_t n, uint32_t base) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) rows[i] += base;
}

// ---- copies between host and device memory

// One contiguous copy; a launch carries up to kMaxSegs of them.
struct Seg {
  const unsigned char *src;
  unsigned char *dst;
  uint64_t bytes;
};
constexpr int kMaxSegs = 96;
struct SegList {
  Seg seg[kMaxSegs];
  int n;
};

// Block row y copies segment y: 16-byte words when both ends and the size
// allow, else bytes.  Grid-stride over the segment in x.
__global__ void __launch_bounds__(512) k_copy_segs(SegList L) {
  const Seg sg = L.seg[blockIdx.y];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((((uintptr_t)sg.src | (uintptr_t)sg.dst | sg.bytes) & 15) == 0) {
    const uint4 *__restrict__ s = (const uint4 *)sg.src;
    uint4 *__restrict__ d = (uint4 *)sg.dst;
    const uint64_t n = sg.bytes >> 4;
    uint64_t i = t0;
    for (; i + 3 * stride < n; i += 4 * stride) {  // four loads in flight per thread
      const uint4 a = s[i], b = s[i + stride], c = s[i + 2 * stride], e = s[i + 3 * stride];
      d[i] = a;
      d[i + stride] = b;
      d[i + 2 * stride] = c;
      d[i + 3 * stride] = e;
    }
    for (; i < n; i += stride) d[i] = s[i];
  } else {
    for (uint64_t i = t0; i < sg.bytes; i += stride) sg.dst[i] = sg.src[i];
  }
}

// The device reads and writes pageable host memory directly (and coherently).
// MDJ_TEST_HOST_MEMCPY=1 (test hook) takes the cudaMemcpyAsync path anyway.
bool direct_host_access() {
  const char *e = getenv("MDJ_TEST_HOST_MEMCPY");
  if (e && e[0] == '1') return false;
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) return false;
  return v == 1;
}

// Issues copies between host and device memory on `s`: batched into copy
// kernels when `direct`, else one cudaMemcpyAsync each (kind cudaMemcpyDefault).
class Copier {
 public:
  Copier(bool direct, cudaStream_t s) : direct_(direct), s_(s) { L_.n = 0; }
  int add(void *dst, const void *src, uint64_t bytes) {
    if (!bytes) return MDJ_OK;
    if (!direct_) return cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s_));
    L_.seg[L_.n++] = {(const unsigned char *)src, (unsigned char *)dst, bytes};
    total_ += bytes;
    return L_.n == kMaxSegs ? flush() : MDJ_OK;
  }
  int flush() {
    if (!L_.n) return MDJ_OK;
    // about four blocks per SM over all segments (copies over the host link
    // are latency bound: many loads in flight), at least 32 KB per block
    const uint64_t per = total_ / L_.n;
    const uint64_t want = std::max<uint64_t>(1, (uint64_t)4 * num_sms() / L_.n);
    const unsigned bx = (unsigned)std::min<uint64_t>(std::min(want, std::max<uint64_t>(per >> 15, 1)), 128);
    k_copy_segs<<<dim3(bx, L_.n), 512, 0, s_>>>(L_);
    L_.n = 0;
    total_ = 0;
    return cuda_status(cudaGetLastError());
  }

 private:
  bool direct_;
  cudaStream_t s_;
  SegList L_;
  uint64_t total_ = 0;
};

// Touches the pages of host staging memory from background threads, task by
// task in order (a task: the byte ranges one phase-1 chunk writes), so that
// the device never writes a page the host has not faulted in and the host
// faults pages in while the device works on earlier chunks.  Every touched
// byte lies inside its own task's ranges, so touching never races with a
// device copy into another task's ranges.  Runs in the calling thread when
// threads cannot be started.
class PageToucher {
 public:
  struct Range {
    unsigned char *p;
    size_t bytes;
  };
  // Ranges of task `task` (tasks numbered 0, 1, ... in the order they are added).
  void add(size_t task, unsigned char *p, size_t bytes) {
    if (!bytes) return;
    if (task >= tasks_.size()) tasks_.resize(task + 1);
    // granules of at most 4 MiB, so that threads share large ranges
    for (size_t off = 0; off < bytes; off += kGranule)
      tasks_[task].push_back({p + off, std::min(kGranule, bytes - off)});
  }
  void start() {
    const long pg = sysconf(_SC_PAGESIZE);
    page_ = pg > 0 ? (size_t)pg : 4096;
    for (size_t t = 0; t < tasks_.size(); t++)
      for (const Range &r : tasks_[t]) gran_.push_back({r, t});
    left_.reset(new std::atomic<size_t>[tasks_.size()]);
    for (size_t t = 0; t < tasks_.size(); t++) left_[t].store(tasks_[t].size());
    unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 16u));
    try {
      for (unsigned i = 0; i < nt; i++) th_.emplace_back([this] { work(); });
    } catch (...) {
    }
    if (th_.empty()) work();
  }
  // Blocks until every page of task `task` is touched.
  void wait(size_t task) {
    if (task >= tasks_.size()) return;
    while (left_[task].load(std::memory_order_acquire) != 0) std::this_thread::yield();
  }
  ~PageToucher() {
    stop_.store(true);
    for (auto &t : th_) t.join();
  }

 private:
  static constexpr size_t kGranule = 4u << 20;
  struct Gran {
    Range r;
    size_t task;
  };
  void work() {
    for (;;) {
      if (stop_.load(std::memory_order_relaxed)) return;
      const size_t g = next_.fetch_add(1);
      if (g >= gran_.size()) return;
      const Range r = gran_[g].r;
      volatile unsigned char *v = r.p;
      // one byte in every page the range overlaps, the range's own byte
      const uintptr_t a = (uintptr_t)r.p;
      const uintptr_t first_page = a - a % page_;
      for (uintptr_t q = first_page; q < a + r.bytes; q += page_) v[(q < a ? a : q) - a] = 0;
      left_[gran_[g].task].fetch_sub(1, std::memory_order_release);
    }
  }
  std::vector<std::vector<Range>> tasks_;
  std::vector<Gran> gran_;
  std::unique_ptr<std::atomic<size_t>[]> left_;
  std::atomic<size_t> next_{0};
  std::atomic<bool> stop_{false};
  std::vector<std::thread> th_;
  size_t page_ = 4096;
};

// One side's buckets in host memory: the partitioned chunks in chunk order,
// each column (and the input row ids) as one array of nrows elements; chunk c
// holds rows [c * chunk_rows, ...) and offs[c * (B + 1) + b] is the start of
// its bucket b, relative to the chunk.
struct HostStage {
  unsigned char *mem = nullptr;
  unsigned char *col[MDJ_MAX_COLS] = {};
  uint32_t *rid = nullptr;
  std::vector<int64_t> offs;
  uint64_t chunk_rows = 0, nchunks = 0;
  HostStage() = default;
  HostStage(const HostStage &) = delete;
  HostStage &operator=(const HostStage &) = delete;
  ~HostStage() { free(mem); }
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// A device block for `bytes`, freed by the owning workspace.
unsigned char *dev_block(Workspace &ws, size_t bytes) { return (unsigned char *)ws.get(bytes ? bytes : 1); }

// One side's staging area (uninitialised host memory) for chunks of
// `chunk_rows` rows; chunk c's ranges become toucher task task0 + c.
int stage_alloc(const mdj_table *t, uint32_t B, uint64_t chunk_rows, HostStage *hs, PageToucher &pt, size_t task0) {
  const int nc = t->ncols;
  const uint64_t n = t->nrows;
  hs->nchunks = 0;
  if (n == 0) return MDJ_OK;
  const uint64_t C = std::min<uint64_t>(chunk_rows, n);
  hs->chunk_rows = C;
  hs->nchunks = (n + C - 1) / C;
  hs->offs.assign(hs->nchunks * (B + 1), 0);
  size_t bytes = align256((size_t)n * 4);
  for (int j = 0; j < nc; j++) bytes += align256((size_t)n * dtype_width(t->cols[j].dtype));
  hs->mem = (unsigned char *)malloc(bytes);
  if (!hs->mem) return MDJ_ERR_OOM;
  size_t at = 0;
  for (int j = 0; j < nc; j++) {
    hs->col[j] = hs->mem + at;
    at += align256((size_t)n * dtype_width(t->cols[j].dtype));
  }
  hs->rid = (uint32_t *)(hs->mem + at);
  for (uint64_t c = 0; c < hs->nchunks; c++) {
    const uint64_t c0 = c * C, cnt = std::min(C, n - c0);
    for (int j = 0; j < nc; j++) {
      const int w = dtype_width(t->cols[j].dtype);
      pt.add(task0 + c, hs->col[j] + c0 * w, cnt * w);
    }
    pt.add(task0 + c, (unsigned char *)(hs->rid + c0), cnt * 4);
  }
  return MDJ_OK;
}

// Phase 1 of one side into its staging area.  Chunk c is copied in and
// partitioned on the caller's stream `s`; its copy back runs on a second
// stream after its pages are touched, issued once chunk c + 1's work is
// queued (a copy into pageable memory may hold the host thread until it
// ends), through the copy engines, so that it overlaps the partition kernels
// (which fill every SM).  Two output buffer sets alternate.
int partition_to_host(const mdj_table *t, int32_t key_col, uint32_t B, const mdj_allocator *alloc, cudaStream_t s,
                      bool direct, HostStage *hs, PageToucher &pt, size_t task0) {
  const int nc = t->ncols;
  int w[MDJ_MAX_COLS];
  for (int j = 0; j < nc; j++) w[j] = dtype_width(t->cols[j].dtype);
  const uint64_t n = t->nrows, nchunks = hs->nchunks, C = hs->chunk_rows;
  if (nchunks == 0) return MDJ_OK;

  Workspace ws(alloc, s);
  unsigned char *din[MDJ_MAX_COLS], *dout[2][MDJ_MAX_COLS];
  uint32_t *drid[2];
  int64_t *doff[2];
  for (int j = 0; j < nc; j++)
    if (!(din[j] = dev_block(ws, C * w[j]))) return MDJ_ERR_OOM;
  for (int k = 0; k < 2; k++) {
    for (int j = 0; j < nc; j++)
      if (!(dout[k][j] = dev_block(ws, C * w[j]))) return MDJ_ERR_OOM;
    drid[k] = (uint32_t *)dev_block(ws, C * 4);
    doff[k] = (int64_t *)dev_block(ws, (size_t)(B + 1) * 8);
    if (!drid[k] || !doff[k]) return MDJ_ERR_OOM;
  }
  // copy-back stream and its events; freed on every path
  struct Side2 {
    cudaStream_t sc = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    ~Side2() {
      for (int k = 0; k < 2; k++) {
        if (ready[k]) cudaEventDestroy(ready[k]);
        if (done[k]) cudaEventDestroy(done[k]);
      }
      if (sc) cudaStreamDestroy(sc);
    }
  } x;
  MDJ_CUDA_TRY(cudaStreamCreateWithFlags(&x.sc, cudaStreamNonBlocking));
  for (int k = 0; k < 2; k++) {
    MDJ_CUDA_TRY(cudaEventCreateWithFlags(&x.ready[k], cudaEventDisableTiming));
    MDJ_CUDA_TRY(cudaEventCreateWithFlags(&x.done[k], cudaEventDisableTiming));
  }
  Copier in(direct, s), back(false, x.sc);
  auto copy_back = [&](uint64_t c) {
    const int k = (int)(c & 1);
    const uint64_t c0 = c * C, cnt = std::min(C, n - c0);
    pt.wait(task0 + c);
    int rc = cuda_status(cudaStreamWaitEvent(x.sc, x.ready[k], 0));
    for (int j = 0; j < nc && rc == MDJ_OK; j++) rc = back.add(hs->col[j] + c0 * w[j], dout[k][j], cnt * w[j]);
    if (rc == MDJ_OK) rc = back.add(hs->rid + c0, drid[k], cnt * 4);
    if (rc == MDJ_OK) rc = back.add(&hs->offs[c * (B + 1)], doff[k], (size_t)(B + 1) * 8);
    if (rc == MDJ_OK) rc = cuda_status(cudaEventRecord(x.done[k], x.sc));
    return rc;
  };
  int rc = MDJ_OK;
  for (uint64_t c = 0; c < nchunks && rc == MDJ_OK; c++) {
    const int k = (int)(c & 1);
    const uint64_t c0 = c * C, cnt = std::min(C, n - c0);
    if (c >= 2) rc = cuda_status(cudaStreamWaitEvent(s, x.done[k], 0));  // chunk c - 2's copy back is done
    mdj_col cols[MDJ_MAX_COLS];
    void *outs[MDJ_MAX_COLS];
    for (int j = 0; j < nc && rc == MDJ_OK; j++) {
      rc = in.add(din[j], (const unsigned char *)t->cols[j].data + c0 * w[j], cnt * w[j]);
      cols[j].data = din[j];
      cols[j].dtype = t->cols[j].dtype;
      outs[j] = dout[k][j];
    }
    if (rc == MDJ_OK) rc = in.flush();
    const mdj_table chunk = {cols, nc, cnt};
    if (rc == MDJ_OK) rc = mdj_partition(&chunk, key_col, B, outs, drid[k], doff[k], alloc, s);
    if (rc == MDJ_OK && c0) {
      const unsigned g = (unsigned)std::min<uint64_t>((cnt + 511) / 512, (uint64_t)num_sms() * 4);
      k_add_rows<<<g, 512, 0, s>>>(drid[k], cnt, (uint32_t)c0);
      rc = cuda_status(cudaGetLastError());
    }
    if (rc == MDJ_OK) rc = cuda_status(cudaEventRecord(x.ready[k], s));
    if (rc == MDJ_OK && c >= 1) rc = copy_back(c - 1);
  }
  if (rc == MDJ_OK) rc = copy_back(nchunks - 1);
  // the caller's stream (and the release of this workspace) follows the
  // copies back; the host reads the offsets after them
  const int k_last = (int)((nchunks - 1) & 1);
  if (rc == MDJ_OK) rc = cuda_status(cudaStreamWaitEvent(s, x.done[k_last], 0));
  if (nchunks >= 2 && rc == MDJ_OK) rc = cuda_status(cudaStreamWaitEvent(s, x.done[k_last ^ 1], 0));
  const int rs = cuda_status(cudaStreamSynchronize(x.sc));
  return rc != MDJ_OK ? rc : rs;
}

// Rows of bucket b in every chunk of one side.
uint64_t bucket_rows(const HostStage &hs, uint32_t B, uint32_t b) {
  uint64_t nb = 0;
  for (uint64_t c = 0; c < hs.nchunks; c++) nb += (uint64_t)(hs.offs[c * (B + 1) + b + 1] - hs.offs[c * (B + 1) + b]);
  return nb;
}

// Bucket b of one side on the device: every column and the input row ids
// (allocated in `ws`, on the caller's stream).
int bucket_alloc(Workspace &ws, const mdj_table *t, const HostStage &hs, uint32_t B, uint32_t b, mdj_col *cols,
                 mdj_table *out, uint32_t **rid) {
  const uint64_t nb = bucket_rows(hs, B, b);
  const int nc = t->ncols;
  for (int j = 0; j < nc; j++) {
    unsigned char *d = dev_block(ws, nb * dtype_width(t->cols[j].dtype));
    if (!d) return MDJ_ERR_OOM;
    cols[j].data = d;
    cols[j].dtype = t->cols[j].dtype;
  }
  *rid = (uint32_t *)dev_block(ws, nb * 4);
  if (!*rid) return MDJ_ERR_OOM;
  *out = {cols, nc, nb};
  return MDJ_OK;
}

// Gathers bucket b's slice of every chunk into the buffers bucket_alloc gave.
int bucket_copy(Copier &cp, const mdj_table *t, const HostStage &hs, uint32_t B, uint32_t b, const mdj_col *cols,
                uint32_t *rid) {
  const int nc = t->ncols;
  uint64_t pos = 0;
  for (uint64_t c = 0; c < hs.nchunks; c++) {
    const int64_t *o = &hs.offs[c * (B + 1)];
    const uint64_t lo = c * hs.chunk_rows + (uint64_t)o[b], cnt = (uint64_t)(o[b + 1] - o[b]);
    if (!cnt) continue;
    for (int j = 0; j < nc; j++) {
      const int w = dtype_width(t->cols[j].dtype);
      MDJ_TRY(cp.add((unsigned char *)cols[j].data + pos * w, hs.col[j] + lo * w, cnt * w));
    }
    MDJ_TRY(cp.add(rid + pos, hs.rid + lo, cnt * 4));
    pos += cnt;
  }
  return cp.flush();
}

// Both sides' bucket b on the device, in a workspace of its own.
struct BucketPair {
  Workspace ws;
  mdj_col lc[MDJ_MAX_COLS], rc[MDJ_MAX_COLS];
  mdj_table lt, rt;
  uint32_t *lrid = nullptr, *rrid = nullptr;
  uint32_t b = 0;
  BucketPair(const mdj_allocator *a, cudaStream_t s) : ws(a, s) {}
};

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

// The right table's copies in, issued on their own stream once the left
// side's partition is queued (merge_steps' hook): the link carries them while
// the device partitions the left side.
struct LateRight {
  const mdj_table *host;
  mdj_col *cols;
  cudaStream_t s, sc;
  cudaEvent_t alloced, ready;
};
int copy_right_in(void *ctx) {
  LateRight &x = *(LateRight *)ctx;
  MDJ_CUDA_TRY(cudaStreamWaitEvent(x.sc, x.alloced, 0));
  for (int j = 0; j < x.host->ncols; j++) {
    const size_t bytes = x.host->nrows * (size_t)dtype_width(x.host->cols[j].dtype);
    if (bytes)
      MDJ_CUDA_TRY(cudaMemcpyAsync((void *)x.cols[j].data, x.host->cols[j].data, bytes, cudaMemcpyHostToDevice, x.sc));
  }
  MDJ_CUDA_TRY(cudaEventRecord(x.ready, x.sc));
  MDJ_CUDA_TRY(cudaStreamWaitEvent(x.s, x.ready, 0));
  return MDJ_OK;
}

// Both tables fit one bucket of the budget: they go to the device once and
// are merged in place.  An inner merge runs mdj_merge's steps, the right
// table's copies overlapping the left side's partition, and hands its result
// to the sink in windows that point into it; the other join types stream
// their rows through one window buffer.  Row ids are already input row ids.
int merge_resident(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P, int32_t how,
                   uint64_t window, mdj_sink sink, void *sink_ctx, const mdj_allocator *alloc, cudaStream_t s,
                   uint64_t *total_rows) {
  // the copy stream and events; drained before the workspace releases the
  // right table's buffers (declared after it, destroyed first)
  Workspace ws(alloc, s);
  struct CopyStream {
    cudaStream_t sc = nullptr;
    cudaEvent_t alloced = nullptr, ready = nullptr;
    ~CopyStream() {
      if (sc) cudaStreamSynchronize(sc);
      if (alloced) cudaEventDestroy(alloced);
      if (ready) cudaEventDestroy(ready);
      if (sc) cudaStreamDestroy(sc);
    }
  } cs;
  mdj_col lc[MDJ_MAX_COLS], rc[MDJ_MAX_COLS];
  mdj_table lt, rt;
  MDJ_TRY(table_to_device(ws, left, lc, &lt));
  uint64_t produced = 0;
  int rc2 = MDJ_OK;
  if (how == MDJ_INNER) {
    for (int j = 0; j < right->ncols; j++) {
      unsigned char *d = dev_block(ws, right->nrows * (size_t)dtype_width(right->cols[j].dtype));
      if (!d) return MDJ_ERR_OOM;
      rc[j].data = d;
      rc[j].dtype = right->cols[j].dtype;
    }
    rt = {rc, right->ncols, right->nrows};
    MDJ_CUDA_TRY(cudaStreamCreateWithFlags(&cs.sc, cudaStreamNonBlocking));
    MDJ_CUDA_TRY(cudaEventCreateWithFlags(&cs.alloced, cudaEventDisableTiming));
    MDJ_CUDA_TRY(cudaEventCreateWithFlags(&cs.ready, cudaEventDisableTiming));
    MDJ_CUDA_TRY(cudaEventRecord(cs.alloced, s));  // the blocks may have served earlier work of s
    LateRight late = {right, rc, s, cs.sc, cs.alloced, cs.ready};
    mdj_result res;
    MDJ_TRY(merge_steps(&lt, lk, &rt, rk, P, alloc, (void *)s, &res, copy_right_in, &late));
    rc2 = cuda_status(cudaStreamSynchronize(s));
    for (uint64_t q0 = 0; q0 < res.nrows && rc2 == MDJ_OK; q0 += window) {
      const uint64_t n = std::min(window, res.nrows - q0);
      const mdj_result piece = result_piece(res, q0, n);
      if (sink(&piece, produced, sink_ctx) != 0) rc2 = MDJ_ERR_ABORTED;
      produced += n;
    }
    mdj_result_release(&res, alloc, (void *)s);
  } else {
    MDJ_TRY(table_to_device(ws, right, rc, &rt));
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
  // a seventh of it (the stream open holds about four times its inputs, the
  // next bucket pair is copied in meanwhile), a chunk of phase 1 a quarter, a
  // window a seventh
  const uint64_t wl = row_bytes(left), wr = row_bytes(right);
  const uint64_t in_bytes = left->nrows * (wl + 4) + right->nrows * (wr + 4);
  uint64_t B = 1;
  while (B < MDJ_MAX_PARTITIONS && in_bytes > B * (budget / 7)) B *= 2;
  // a chunk's input, two output sets and their row ids: a quarter of the
  // budget; a multiple of 16 rows, so every chunk's columns start 16-byte
  // aligned in the staging area
  const uint64_t chunk_rows =
      std::max<uint64_t>(16, ((budget / 4) / (3 * std::max(wl, wr) + 8)) & ~(uint64_t)15);
  const uint64_t out_row = wl + wr + 8 - dtype_width(kd);  // key once, both row ids, every other column
  const uint64_t window = std::max<uint64_t>(1, (budget / 7) / out_row);

  if (B == 1) return merge_resident(left, lk, right, rk, P, how, window, sink, sink_ctx, alloc, s, total_rows);

  const bool direct = direct_host_access();
  HostStage hl, hr;
  {
    PageToucher pt;  // destroyed (threads joined) before the staging areas
    MDJ_TRY(stage_alloc(left, (uint32_t)B, chunk_rows, &hl, pt, 0));
    MDJ_TRY(stage_alloc(right, (uint32_t)B, chunk_rows, &hr, pt, hl.nchunks));
    pt.start();
    MDJ_TRY(partition_to_host(left, lk, (uint32_t)B, alloc, s, direct, &hl, pt, 0));
    MDJ_TRY(partition_to_host(right, rk, (uint32_t)B, alloc, s, direct, &hr, pt, hl.nchunks));
  }

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
  std::vector<uint32_t> todo;  // buckets with output
  for (uint32_t b = 0; b < B; b++) {
    const uint64_t nl = bucket_rows(hl, (uint32_t)B, b), nr = bucket_rows(hr, (uint32_t)B, b);
    if ((nl && nr) || (nl && keep_left) || (nr && keep_right)) todo.push_back(b);
  }
  // Bucket i + 1 is allocated on the caller's stream and copied in on a
  // prefetch stream while bucket i merges.  The guard drains the prefetch
  // stream before any bucket's buffers are released (it is destroyed first).
  std::unique_ptr<BucketPair> cur, nxt;
  struct Prefetch {
    cudaStream_t sp = nullptr;
    cudaEvent_t alloced = nullptr, ready[2] = {nullptr, nullptr};
    ~Prefetch() {
      if (sp) cudaStreamSynchronize(sp);
      if (alloced) cudaEventDestroy(alloced);
      for (int k = 0; k < 2; k++)
        if (ready[k]) cudaEventDestroy(ready[k]);
      if (sp) cudaStreamDestroy(sp);
    }
  } pf;
  MDJ_CUDA_TRY(cudaStreamCreateWithFlags(&pf.sp, cudaStreamNonBlocking));
  MDJ_CUDA_TRY(cudaEventCreateWithFlags(&pf.alloced, cudaEventDisableTiming));
  for (int k = 0; k < 2; k++) MDJ_CUDA_TRY(cudaEventCreateWithFlags(&pf.ready[k], cudaEventDisableTiming));
  auto prefetch = [&](std::unique_ptr<BucketPair> &bp, uint32_t b, int slot) {
    bp.reset(new BucketPair(alloc, s));
    bp->b = b;
    MDJ_TRY(bucket_alloc(bp->ws, left, hl, (uint32_t)B, b, bp->lc, &bp->lt, &bp->lrid));
    MDJ_TRY(bucket_alloc(bp->ws, right, hr, (uint32_t)B, b, bp->rc, &bp->rt, &bp->rrid));
    // the blocks may have served earlier work of the caller's stream
    MDJ_CUDA_TRY(cudaEventRecord(pf.alloced, s));
    MDJ_CUDA_TRY(cudaStreamWaitEvent(pf.sp, pf.alloced, 0));
    Copier cp(direct, pf.sp);
    MDJ_TRY(bucket_copy(cp, left, hl, (uint32_t)B, b, bp->lc, bp->lrid));
    MDJ_TRY(bucket_copy(cp, right, hr, (uint32_t)B, b, bp->rc, bp->rrid));
    MDJ_CUDA_TRY(cudaEventRecord(pf.ready[slot], pf.sp));
    return (int)MDJ_OK;
  };
  uint64_t produced = 0;
  if (!todo.empty()) MDJ_TRY(prefetch(cur, todo[0], 0));
  for (size_t i = 0; i < todo.size(); i++) {
    if (i + 1 < todo.size()) MDJ_TRY(prefetch(nxt, todo[i + 1], (int)((i + 1) & 1)));
    MDJ_CUDA_TRY(cudaStreamWaitEvent(s, pf.ready[i & 1], 0));
    mdj_stream *h = nullptr;
    uint64_t m = 0;
    MDJ_TRY(mdj_stream_open(&cur->lt, lk, &cur->rt, rk, Pb, how, alloc, stream, &h, &m));
    int rc2 = MDJ_OK;
    for (uint64_t q0 = 0; q0 < m && rc2 == MDJ_OK; q0 += window) {
      const uint64_t n = std::min(window, m - q0);
      rc2 = mdj_stream_emit(h, q0, n, &win);
      if (rc2 != MDJ_OK) break;
      const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms() * 8);
      k_map_rows<<<grid, 256, 0, s>>>(piece.left_row, n, cur->lrid);
      k_map_rows<<<grid, 256, 0, s>>>(piece.right_row, n, cur->rrid);
      rc2 = cuda_status(cudaGetLastError());
      if (rc2 == MDJ_OK) rc2 = cuda_status(cudaStreamSynchronize(s));
      if (rc2 != MDJ_OK) break;
      piece.nrows = n;
      if (sink(&piece, produced, sink_ctx) != 0) rc2 = MDJ_ERR_ABORTED;
      produced += n;
    }
    mdj_stream_close(h);
    MDJ_TRY(rc2);
    cur = std::move(nxt);  // this bucket's tables go back on the caller's stream
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
