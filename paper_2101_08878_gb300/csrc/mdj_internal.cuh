// Internal declarations shared by the libmdj translation units.
//
// Device-side helpers: the key hash (MurmurHash3's 64-bit finalizer, written
// from its published description), the partition / sub-bucket functions, and
// small warp/block primitives.  Host-side helpers: the stream-ordered
// workspace that owns every temporary buffer of one call, launch tracing, and
// the plan that decides how a join is bucketed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "mdj.h"

namespace mdj {

// ------------------------------------------------------------------ limits

constexpr uint32_t kMaxFanout = 1024;     // buckets of one stable scatter pass
constexpr uint32_t kMergeFanout = 256;    // pass-1 buckets of a two-pass join plan
constexpr uint32_t kMaxSubBuckets = 49152;  // final buckets of a two-pass plan
constexpr uint32_t kPass2SpanMax = 1024;  // local buckets of one pass-2 tile

// ------------------------------------------------------------------ hashing

// MurmurHash3 64-bit finalizer: xor-shift 33, multiply, xor-shift 33,
// multiply, xor-shift 33.
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t h) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdULL;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ULL;
  h ^= h >> 33;
  return h;
}

// Key bits: sign-extended to 64 bits, so equal int32/int64 values hash equal.
__device__ __forceinline__ uint64_t key_bits(int32_t k) { return (uint64_t)(int64_t)k; }
__device__ __forceinline__ uint64_t key_bits(int64_t k) { return (uint64_t)k; }

// How a row's hash h selects its bucket.
//   p  = h mod P                                (the partition / "worker")
//   sb = p * S + floor(hi32(h) * S / 2^32)      (final sub-bucket, p-major)
//   FB mode:    bucket = sb / div                (div = 1: the sub-bucket)
//   DIGIT mode: bucket = (p / dmul) % dmod       (LSD digit of p)
// With S = S1 * div, floor(x*S/2^32) / div = floor(x*S1/2^32) for any 32-bit x
// (write x*S1 = s1*2^32 + lo: then x*S/2^32 = s1*div + lo*div/2^32 and
// lo*div/2^32 < div), so the pass-1 bucket sb / div = p*S1 + floor(x*S1/2^32)
// needs no division.
struct BucketSpec {
  uint64_t P;
  uint64_t M;  // floor((2^64 - 1) / P), for the quotient estimate of h / P
  uint32_t S;
  uint32_t S1;  // S / div
  uint32_t div;
  uint32_t dmul;
  uint32_t dmod;
  int pow2;     // P is a power of two: h mod P = h & (P - 1)
  int digit_mode;
};

// h mod P by a one-correction Barrett reduction: q = umulhi(h, M) is the true
// quotient or one less, so one conditional subtraction finishes.
__device__ __forceinline__ uint32_t mod_p(uint64_t h, const BucketSpec &bs) {
  if (bs.pow2) return (uint32_t)h & (uint32_t)(bs.P - 1);
  uint64_t q = __umul64hi(h, bs.M);
  uint64_t r = h - q * bs.P;
  if (r >= bs.P) r -= bs.P;
  return (uint32_t)r;
}

__device__ __forceinline__ uint32_t sub_bucket_of(uint64_t h, const BucketSpec &bs) {
  uint32_t p = mod_p(h, bs);
  return p * bs.S + __umulhi((uint32_t)(h >> 32), bs.S);
}

__device__ __forceinline__ uint32_t bucket_of(uint64_t h, const BucketSpec &bs) {
  uint32_t p = mod_p(h, bs);
  if (bs.digit_mode) return (p / bs.dmul) % bs.dmod;
  return p * bs.S1 + __umulhi((uint32_t)(h >> 32), bs.S1);
}

// A tile of a segmented (batched) partition: rows [row0, row0 + rows) of one segment.
struct SegTile {
  uint32_t row0, rows, seg;
};

BucketSpec make_spec(uint32_t P, uint32_t S, uint32_t div);
BucketSpec make_digit_spec(uint32_t P, uint32_t dmul, uint32_t dmod);

// Partition-only spec built on the device (one per segment of a batch).
__device__ __forceinline__ BucketSpec make_spec_dev(uint32_t P) {
  BucketSpec b;
  b.P = P;
  b.M = 0xFFFFFFFFFFFFFFFFull / P;
  b.S = 1;
  b.S1 = 1;
  b.div = 1;
  b.dmul = 1;
  b.dmod = 1;
  b.pow2 = (P & (P - 1)) == 0;
  b.digit_mode = 0;
  return b;
}

// ------------------------------------------------------------ primitives

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Device time in nanoseconds (bounds every device-side wait).
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive scan of one value per thread.  `scratch` holds one T
// per warp plus one.  Returns the exclusive prefix; *total gets the block sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *scratch, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  T inc = warp_inclusive_scan(v);
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? scratch[lane] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane < nw) scratch[lane] = wi - w;
    if (lane == nw - 1) scratch[32] = wi;
  }
  __syncthreads();
  T res = scratch[warp] + inc - v;
  *total = scratch[32];
  __syncthreads();
  return res;
}

// In-place exclusive scan of a shared-memory array a[0..n).  `scratch` holds
// 33 uint32.  All threads of the block must call it.
__device__ __forceinline__ void block_scan_array(uint32_t *a, uint32_t n, uint32_t *scratch) {
  const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
  const uint32_t beg = threadIdx.x * per;
  uint32_t s = 0;
  for (uint32_t i = 0; i < per; i++)
    if (beg + i < n) s += a[beg + i];
  uint32_t tot;
  uint32_t run = block_exclusive_scan<uint32_t>(s, scratch, &tot);
  for (uint32_t i = 0; i < per; i++)
    if (beg + i < n) {
      uint32_t c = a[beg + i];
      a[beg + i] = run;
      run += c;
    }
  __syncthreads();
}

// Bits of element i of a 4- or 8-byte column (0 for a missing column).
__device__ __forceinline__ uint64_t pay_bits(const void *col, int width, uint32_t i) {
  if (!col) return 0;
  return width == 8 ? ((const uint64_t *)col)[i] : (uint64_t)((const uint32_t *)col)[i];
}

// The two terms of mdj_count_checksum's checksum (defined in mdj.h):
// f(l) for a left row l with key bits kbits and first-payload bits pbits,
// g(r) for a right row r; the checksum is the sum of f(l) g(r) over pairs.
__device__ __forceinline__ uint64_t term_f(uint64_t kbits, uint32_t lrow, uint64_t pbits) {
  return fmix64(kbits ^ (0x9E3779B97F4A7C15ULL * ((uint64_t)lrow + 1)) ^ pbits);
}
__device__ __forceinline__ uint64_t term_g(uint32_t rrow, uint64_t pbits) {
  return fmix64((0xC2B2AE3D27D4EB4FULL * ((uint64_t)rrow + 1)) ^ pbits);
}

// ------------------------------------------------------------ host helpers

inline int dtype_width(int32_t dt) {
  switch (dt) {
    case MDJ_I32: case MDJ_F32: case MDJ_U32: return 4;
    case MDJ_I64: case MDJ_F64: case MDJ_U64: return 8;
    default: return 0;
  }
}

// Every temporary buffer of one call, from the caller's allocator (or
// cudaMallocAsync), released in stream order when the call ends.  Requests of
// at most kArenaMax bytes are carved from kArenaChunk-byte chunks (one
// allocator call per chunk, not per buffer; give_back of such a piece is a
// no-op until the call ends), larger ones are allocated one by one.
class Workspace {
 public:
  Workspace(const mdj_allocator *a, cudaStream_t s) : alloc_(a), stream_(s) {}
  ~Workspace() { release_all(); }
  Workspace(const Workspace &) = delete;
  Workspace &operator=(const Workspace &) = delete;

  void *get(size_t bytes);           // NULL on failure
  void give_back(void *p);           // release one buffer early
  void *get_owned_by_caller(size_t bytes);  // not released by this workspace
  void release_caller(void *p);      // release a caller-owned buffer (error paths)
  void release_all();
  cudaStream_t stream() const { return stream_; }
  const mdj_allocator *allocator() const { return alloc_; }

 private:
  void *raw_alloc(size_t bytes);
  void raw_free(void *p);
  const mdj_allocator *alloc_;
  cudaStream_t stream_;
  std::vector<void *> owned_;       // buffers allocated on their own
  std::vector<void *> chunks_;      // arena chunks for small buffers
  unsigned char *arena_ = nullptr;  // current chunk
  size_t arena_used_ = 0;
  static constexpr size_t kArenaMax = 1u << 20;
  static constexpr size_t kArenaChunk = 8u << 20;
};

// Launch tracing (mdj_profile_*): events around each launch when enabled.
struct TraceScope {
  TraceScope(const char *name, cudaStream_t s);
  ~TraceScope();
  const char *name_;
  cudaStream_t s_;
  int slot_;
};

int num_sms();
int cuda_status(cudaError_t e);  // MDJ_OK or MDJ_ERR_CUDA (and records the text)

// Set-up that must run once on every device that uses it, with that device
// current (for example cudaFuncSetAttribute, which applies to the current
// device only).  Thread-safe: concurrent first calls on one device run `fn`
// once; a failed `fn` is retried by the next call.
constexpr int kMaxDevicesOnce = 64;
struct PerDeviceOnce {
  std::mutex mu;
  bool done[kMaxDevicesOnce] = {};
};
template <typename Fn>
int once_per_device(PerDeviceOnce &once, Fn &&fn) {
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kMaxDevicesOnce) return MDJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(once.mu);
  if (once.done[dev]) return MDJ_OK;
  const int rc = fn();
  if (rc == MDJ_OK) once.done[dev] = true;
  return rc;
}

// ------------------------------------------------------------- side buffers

// One table side as the join kernels see it: `key` plus payload columns, with
// rows grouped into `nbuckets` buckets by bucket offsets `off` (uint32,
// nbuckets + 1 entries, device).  `rid` maps a row to its input row index;
// NULL means the identity (an unpartitioned side).
struct Side {
  const void *key;
  int32_t key_dtype;
  int32_t ncols;                   // non-key columns
  const void *cols[MDJ_MAX_COLS];
  int32_t widths[MDJ_MAX_COLS];
  int32_t dtypes[MDJ_MAX_COLS];
  const uint32_t *rid;
  const uint32_t *off;
  uint64_t nrows;
};

// How a join is bucketed: P partitions, each split into S sub-buckets so that
// a sub-bucket's build side fits one shared-memory hash table.
struct Plan {
  uint32_t P = 1;
  uint32_t S = 1;        // sub-buckets per partition
  uint32_t F1 = 1;       // buckets of pass 1 (P * S / F2)
  uint32_t F2 = 1;       // pass-2 split of each pass-1 bucket (1 = single pass)
  uint32_t nbuckets = 1; // final buckets (P * S)
  bool lsd = false;      // P > kMaxFanout: two stable digit passes on p
  bool partition = true; // false: no partitioning at all (P = 1, small build side)
  bool stable = false;   // stable passes (rows keep input order in a bucket)
  uint32_t cap = 4096;   // build rows per shared-memory table
  uint32_t join_threads = 512;  // threads of a join block (256 or 512); probe rows per item = 8x
};

Plan make_plan(uint64_t n_build, uint32_t P, uint32_t cap, bool force_partition);

// Partition one side (key + every column + row ids) according to `plan` into
// freshly allocated workspace buffers; fills `out` (offsets per final bucket).
int partition_side(Workspace &ws, const mdj_table *t, int32_t key_col, const Plan &plan,
                   Side *out);

// Segmented partition of a batch: segment i = rows [seg_off[i], seg_off[i+1])
// (host array) is split into seg_nb[i] = P_i * S_i buckets numbered from
// seg_base[i]: bucket p * S_i + floor(hi32(h) * S_i / 2^32), p = h mod P_i,
// h = fmix64(key) (all host arrays).  nbuckets = sum of seg_nb.
int partition_side_segmented(Workspace &ws, const mdj_table *t, int32_t key_col, const uint64_t *seg_off,
                             uint32_t nseg, const uint32_t *seg_base, const uint32_t *seg_nb, const uint32_t *seg_P,
                             uint32_t nbuckets, Side *out);

// Stable partition into caller buffers (the mdj_partition body).
int stable_partition(Workspace &ws, const mdj_table *t, int32_t key_col, uint32_t P,
                     void *const *out_cols, uint32_t *out_rid, int64_t *out_offsets);

// Allocation-free variants (caller-provided device scratch), used only by
// mdj_partition_noalloc: words of scratch needed, and the calls themselves.
size_t scan_scratch_words(size_t n);
int exclusive_scan_u32_scratch(const uint32_t *in, uint32_t *out, size_t n, uint32_t *sums, cudaStream_t s);
size_t stable_partition_scratch_words(uint64_t n, uint32_t P);
int stable_partition_scratch(const mdj_table *t, int32_t key_col, uint32_t P, void *const *out_cols,
                             uint32_t *out_rid, int64_t *out_offsets, uint32_t *scratch, size_t scratch_words,
                             cudaStream_t s);

// mdj_merge's steps with a hook between the two sides' partitions
// (csrc/mdj_join.cu).
int merge_steps(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P,
                const mdj_allocator *alloc, void *stream, mdj_result *out, int (*after_left)(void *), void *ctx);

// mdj_count_checksum: the pair count and checksum of the inner join, from
// the streamed output's grouping (every key group of the build side gathered
// once, each probe row told its group): count = sum of the probe rows' group
// sizes, checksum = sum over probe rows r of g(r) times the sum of f over r's
// group (a prefix sum over the grouped build rows).
int grouped_count_checksum(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P,
                           const mdj_allocator *alloc, void *stream, uint64_t *count, uint64_t *checksum);

// Exclusive scans (out may equal in).  n may be 0.
int exclusive_scan_u32(Workspace &ws, const uint32_t *in, uint32_t *out, size_t n);
int exclusive_scan_u64(Workspace &ws, const uint64_t *in, uint64_t *out, size_t n);

}  // namespace mdj

#define MDJ_TRY(expr)                 \
  do {                                \
    int _rc = (expr);                 \
    if (_rc != MDJ_OK) return _rc;    \
  } while (0)

#define MDJ_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::mdj::cuda_status(_e);    \
  } while (0)

#define MDJ_LAUNCH_CHECK() MDJ_CUDA_TRY(cudaGetLastError())
