// Runtime pieces of libmdj: the stream-ordered workspace, launch tracing,
// status strings and small host helpers.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "mdj_internal.cuh"

namespace mdj {

extern thread_local char g_last_cuda_error[256];

// ----------------------------------------------------------------- workspace

void *Workspace::raw_alloc(size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (alloc_ && alloc_->alloc) return alloc_->alloc(bytes, alloc_->ctx, (void *)stream_);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, stream_) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void Workspace::raw_free(void *p) {
  if (!p) return;
  if (alloc_ && alloc_->release) {
    alloc_->release(p, alloc_->ctx, (void *)stream_);
    return;
  }
  if (!(alloc_ && alloc_->alloc)) cudaFreeAsync(p, stream_);
}

void *Workspace::get(size_t bytes) {
  if (bytes <= kArenaMax) {
    const size_t need = ((bytes ? bytes : 1) + 255) & ~(size_t)255;
    if (!arena_ || arena_used_ + need > kArenaChunk) {
      void *c = raw_alloc(kArenaChunk);
      if (!c) return nullptr;
      chunks_.push_back(c);
      arena_ = (unsigned char *)c;
      arena_used_ = 0;
    }
    void *p = arena_ + arena_used_;
    arena_used_ += need;
    return p;
  }
  void *p = raw_alloc(bytes);
  if (p) owned_.push_back(p);
  return p;
}

// Only buffers allocated on their own go back early; a small buffer lives in
// an arena chunk (whose base may equal the buffer's address) until
// release_all.
void Workspace::give_back(void *p) {
  for (size_t i = 0; i < owned_.size(); i++)
    if (owned_[i] == p) {
      raw_free(p);
      owned_.erase(owned_.begin() + i);
      return;
    }
}

void *Workspace::get_owned_by_caller(size_t bytes) { return raw_alloc(bytes); }
void Workspace::release_caller(void *p) { raw_free(p); }

void Workspace::release_all() {
  for (size_t i = owned_.size(); i-- > 0;) raw_free(owned_[i]);
  owned_.clear();
  for (size_t i = chunks_.size(); i-- > 0;) raw_free(chunks_[i]);
  chunks_.clear();
  arena_ = nullptr;
  arena_used_ = 0;
}

// ------------------------------------------------------------------- helpers

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

thread_local char g_last_cuda_error[256];

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MDJ_OK;
  snprintf(g_last_cuda_error, sizeof g_last_cuda_error, "%s", cudaGetErrorString(e));
  return MDJ_ERR_CUDA;
}

BucketSpec make_spec(uint32_t P, uint32_t S, uint32_t div) {
  BucketSpec b;
  b.P = P;
  b.M = UINT64_MAX / P;
  b.S = S;
  b.S1 = S / div;
  b.div = div;
  b.dmul = 1;
  b.dmod = 1;
  b.pow2 = (P & (P - 1)) == 0;
  b.digit_mode = 0;
  return b;
}

BucketSpec make_digit_spec(uint32_t P, uint32_t dmul, uint32_t dmod) {
  BucketSpec b = make_spec(P, 1, 1);
  b.dmul = dmul;
  b.dmod = dmod;
  b.digit_mode = 1;
  return b;
}

// ------------------------------------------------------------------- tracing

namespace {
struct TraceEntry {
  std::string name;
  uint64_t launches = 0;
  double total_ms = 0;
};
struct Pending {
  int entry;
  cudaEvent_t a, b;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceEntry> g_entries;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;

cudaEvent_t take_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int entry_index(const char *name) {
  for (size_t i = 0; i < g_entries.size(); i++)
    if (g_entries[i].name == name) return (int)i;
  g_entries.push_back(TraceEntry{name, 0, 0.0});
  return (int)g_entries.size() - 1;
}
}  // namespace

TraceScope::TraceScope(const char *name, cudaStream_t s) : name_(name), s_(s), slot_(-1) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (!g_trace_on) return;
  Pending p;
  p.entry = entry_index(name);
  p.a = take_event();
  p.b = take_event();
  if (!p.a || !p.b) return;
  cudaEventRecord(p.a, s);
  g_pending.push_back(p);
  slot_ = (int)g_pending.size() - 1;
}

TraceScope::~TraceScope() {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (slot_ >= 0 && slot_ < (int)g_pending.size()) cudaEventRecord(g_pending[slot_].b, s_);
}

}  // namespace mdj

using namespace mdj;

extern "C" {

void mdj_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_on = on != 0;
}

void mdj_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (auto &p : g_pending) {
    cudaEventSynchronize(p.b);
    g_free_events.push_back(p.a);
    g_free_events.push_back(p.b);
  }
  g_pending.clear();
  g_entries.clear();
}

int mdj_profile_collect(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  int rc = MDJ_OK;
  for (auto &p : g_pending) {
    cudaError_t e = cudaEventSynchronize(p.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) {
      rc = cuda_status(e);
    } else {
      g_entries[p.entry].launches += 1;
      g_entries[p.entry].total_ms += ms;
    }
    g_free_events.push_back(p.a);
    g_free_events.push_back(p.b);
  }
  g_pending.clear();
  return rc;
}

int mdj_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  return (int)g_entries.size();
}

int mdj_profile_get(int i, const char **name, uint64_t *launches, double *total_ms) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (i < 0 || i >= (int)g_entries.size()) return MDJ_ERR_INVALID_ARG;
  if (name) *name = g_entries[i].name.c_str();
  if (launches) *launches = g_entries[i].launches;
  if (total_ms) *total_ms = g_entries[i].total_ms;
  return MDJ_OK;
}

const char *mdj_status_string(int status) {
  switch (status) {
    case MDJ_OK: return "ok";
    case MDJ_ERR_INVALID_ARG: return "invalid argument";
    case MDJ_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype";
    case MDJ_ERR_TOO_LARGE: return "too many rows (row ids are uint32)";
    case MDJ_ERR_OOM: return "out of device memory (allocator returned NULL)";
    case MDJ_ERR_CUDA: return "CUDA runtime error";
    case MDJ_ERR_DEVICE_TIMEOUT: return "bounded device-side wait expired";
    case MDJ_ERR_INTERNAL: return "internal consistency check failed";
    case MDJ_ERR_ABORTED: return "stopped by the caller's sink";
    default: return "unknown status";
  }
}

int mdj_version(void) { return MDJ_VERSION; }

const char *mdj_last_error(void) { return g_last_cuda_error[0] ? g_last_cuda_error : ""; }

void mdj_result_release(mdj_result *res, const mdj_allocator *alloc, void *stream) {
  if (!res) return;
  Workspace ws(alloc, (cudaStream_t)stream);
  ws.release_caller(res->key);
  ws.release_caller(res->left_row);
  ws.release_caller(res->right_row);
  for (int j = 0; j < res->n_left_cols && j < MDJ_MAX_COLS; j++) ws.release_caller(res->left_cols[j]);
  for (int j = 0; j < res->n_right_cols && j < MDJ_MAX_COLS; j++) ws.release_caller(res->right_cols[j]);
  memset(res, 0, sizeof *res);
}

}  // extern "C"
