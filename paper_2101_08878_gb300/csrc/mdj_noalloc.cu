// mdj_partition_noalloc: the stable hash partition of mdj_partition for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they want to partition: code running inside another framework's memory pool
// that owns the whole device budget, latency-critical loops where an
// allocation could block the device or fail part-way, or plugins whose host
// process forbids them from touching the device allocator.  They already own
// the input and output buffers; what they cannot provide is the partition's
// temporary working memory.  This entry point takes that working memory from a
// fixed-size array compiled into the library instead.
//
// The scratch array below (16 MiB) exists once per GPU that loads this
// library, for the lifetime of the process.  Every call on a device reuses the
// same array and leaves its contents behind; calls whose work overlaps on the
// GPU (different streams, or different host threads without ordering) race on
// it and must be serialised by the caller.  Every scratch word this path reads
// is first written by the same call, so nothing needs clearing between calls.
#include <mutex>

#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr size_t kNoallocScratchWords = (size_t)4 << 20;  // 4 Mi uint32 = 16 MiB

// Histogram matrix, scan partials and bucket starts of one partition call.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t *g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch(uint32_t **out) {
  int dev = 0;
  MDJ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MDJ_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    g_noalloc_ptr[dev] = (uint32_t *)p;
  }
  *out = g_noalloc_ptr[dev];
  return MDJ_OK;
}

int check_noalloc_args(const mdj_table *in, int32_t key_col, uint32_t P, void *const *out_cols,
                       const int64_t *out_offsets) {
  if (!in || !in->cols || in->ncols < 1 || in->ncols > MDJ_MAX_COLS) return MDJ_ERR_INVALID_ARG;
  if (key_col < 0 || key_col >= in->ncols) return MDJ_ERR_INVALID_ARG;
  if (in->nrows >= (1ull << 32)) return MDJ_ERR_TOO_LARGE;
  for (int j = 0; j < in->ncols; j++) {
    if (dtype_width(in->cols[j].dtype) == 0) return MDJ_ERR_UNSUPPORTED_DTYPE;
    if (in->nrows > 0 && !in->cols[j].data) return MDJ_ERR_INVALID_ARG;
  }
  const int32_t kd = in->cols[key_col].dtype;
  if (kd != MDJ_I32 && kd != MDJ_I64) return MDJ_ERR_UNSUPPORTED_DTYPE;
  if (P < 1 || P > kMaxFanout || !out_cols || !out_offsets) return MDJ_ERR_INVALID_ARG;
  if (in->nrows > 0)
    for (int j = 0; j < in->ncols; j++)
      if (!out_cols[j]) return MDJ_ERR_INVALID_ARG;
  return MDJ_OK;
}

}  // namespace
}  // namespace mdj

using namespace mdj;

extern "C" int mdj_partition_noalloc(const mdj_table *in, int32_t key_col, uint32_t P, void *const *out_cols,
                                     uint32_t *out_row_ids, int64_t *out_offsets, void *stream) {
  MDJ_TRY(check_noalloc_args(in, key_col, P, out_cols, out_offsets));
  if (stable_partition_scratch_words(in->nrows, P) > kNoallocScratchWords) return MDJ_ERR_TOO_LARGE;
  uint32_t *scratch = nullptr;
  MDJ_TRY(noalloc_scratch(&scratch));
  return stable_partition_scratch(in, key_col, P, out_cols, out_row_ids, out_offsets, scratch,
                                  kNoallocScratchWords, (cudaStream_t)stream);
}
