// Device-wide exclusive scan (prefix sum), used for partition offsets, the
// per-(bucket, tile) scatter bases, work-item offsets and output offsets.
//
// Up to kSmallScanMax elements: one launch of one block (each warp reduces
// its span, a block scan of the warp sums, each warp rescans its span).
// Larger: three launches, no inter-block waits: (1) each block reduces one
// chunk, (2) one block scans the chunk sums, (3) each block rescans its chunk
// and adds its chunk's base.  Each element is read twice and written once.
#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T *__restrict__ in, size_t n, T *__restrict__ sums) {
  __shared__ T scratch[33];
  const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++)
    if (base + i < n) s += in[base + i];
  T tot;
  block_exclusive_scan<T>(s, scratch, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block: exclusive scan of `sums[0..m)` in place, chunk by chunk with a
// running carry.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(T *__restrict__ sums, size_t m) {
  __shared__ T scratch[33];
  T carry = 0;
  for (size_t c0 = 0; c0 < m; c0 += kScanThreads) {
    size_t i = c0 + threadIdx.x;
    T v = i < m ? sums[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(v, scratch, &tot);
    if (i < m) sums[i] = carry + ex;
    carry += tot;
  }
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const T *__restrict__ in, T *__restrict__ out, size_t n,
                                                            const T *__restrict__ sums) {
  __shared__ T scratch[33];
  const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    v[i] = base + i < n ? in[base + i] : T(0);
    s += v[i];
  }
  T tot;
  T run = block_exclusive_scan<T>(s, scratch, &tot) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; i++)
    if (base + i < n) {
      out[base + i] = run;
      run += v[i];
    }
}

constexpr int kSmallScanThreads = 1024;
constexpr size_t kSmallScanMax = 1u << 15;
constexpr int kSmallRows = 8;  // 32-element rows a warp loads per step

// One block.  Warp w owns [w * per, (w + 1) * per); a step loads kSmallRows
// rows of 32 consecutive elements (coalesced, all loads in flight at once).
// `in` may equal `out`: every lane reads its elements before writing them.
template <typename T>
__global__ void __launch_bounds__(kSmallScanThreads) k_scan_small(const T *in, T *out, size_t n) {
  __shared__ T scratch[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr size_t step = 32 * kSmallRows;
  const size_t per = ((n + 31) / 32 + step - 1) / step * step;
  const size_t lo = min(n, (size_t)warp * per), hi = min(n, lo + per);
  T s = 0;
  for (size_t i0 = lo; i0 < hi; i0 += step) {
    T v[kSmallRows];
#pragma unroll
    for (int j = 0; j < kSmallRows; j++) {
      const size_t i = i0 + j * 32 + lane;
      v[j] = i < hi ? in[i] : T(0);
    }
#pragma unroll
    for (int j = 0; j < kSmallRows; j++) s += v[j];
  }
  const T wt = __shfl_sync(0xffffffffu, warp_inclusive_scan(s), 31);
  T tot;
  T carry = block_exclusive_scan<T>(lane == 31 ? wt : T(0), scratch, &tot);  // the warps before this one
  for (size_t i0 = lo; i0 < hi; i0 += step) {
    T v[kSmallRows];
#pragma unroll
    for (int j = 0; j < kSmallRows; j++) {
      const size_t i = i0 + j * 32 + lane;
      v[j] = i < hi ? in[i] : T(0);
    }
#pragma unroll
    for (int j = 0; j < kSmallRows; j++) {
      const T inc = warp_inclusive_scan(v[j]);
      const size_t i = i0 + j * 32 + lane;
      if (i < hi) out[i] = carry + inc - v[j];
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
}

template <typename T>
int exclusive_scan(Workspace &ws, const T *in, T *out, size_t n) {
  if (n == 0) return MDJ_OK;
  if (n <= kSmallScanMax) {
    TraceScope tr("scan_small", ws.stream());
    k_scan_small<T><<<1, kSmallScanThreads, 0, ws.stream()>>>(in, out, n);
    MDJ_LAUNCH_CHECK();
    return MDJ_OK;
  }
  const size_t nb = (n + kScanChunk - 1) / kScanChunk;
  T *sums = (T *)ws.get(nb * sizeof(T));
  if (!sums) return MDJ_ERR_OOM;
  cudaStream_t s = ws.stream();
  {
    TraceScope tr("scan_reduce", s);
    k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  }
  {
    TraceScope tr("scan_sums", s);
    k_scan_sums<T><<<1, kScanThreads, 0, s>>>(sums, nb);
  }
  {
    TraceScope tr("scan_down", s);
    k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  }
  MDJ_LAUNCH_CHECK();
  ws.give_back(sums);
  return MDJ_OK;
}

}  // namespace

int exclusive_scan_u32(Workspace &ws, const uint32_t *in, uint32_t *out, size_t n) {
  return exclusive_scan<uint32_t>(ws, in, out, n);
}

int exclusive_scan_u64(Workspace &ws, const uint64_t *in, uint64_t *out, size_t n) {
  return exclusive_scan<uint64_t>(ws, in, out, n);
}

}  // namespace mdj

namespace mdj {

// Scan with caller-provided scratch for the chunk sums (no allocation):
// scan_scratch_words(n) words at `sums`.  Used by the allocation-free
// partition entry point.
size_t scan_scratch_words(size_t n) { return n ? (n + kScanChunk - 1) / kScanChunk : 0; }

int exclusive_scan_u32_scratch(const uint32_t *in, uint32_t *out, size_t n, uint32_t *sums, cudaStream_t s) {
  if (n == 0) return MDJ_OK;
  const size_t nb = (n + kScanChunk - 1) / kScanChunk;
  k_scan_reduce<uint32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  k_scan_sums<uint32_t><<<1, kScanThreads, 0, s>>>(sums, nb);
  k_scan_down<uint32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

}  // namespace mdj
