// The per-partition merge: an inner hash join of co-partitioned tables
// (Sec. V-B: "a merge operation is carried out" after the shuffle).
//
// Both sides are bucketed with the same hash (partition p, then sub-bucket),
// so equal keys share a bucket.  A work item is (bucket, chunk of at most
// `cap` build rows); one block builds a hash table of that chunk in shared
// memory and streams the bucket's probe rows past it.  Two passes:
//
//   count  - matches per item (and, for mdj_count_checksum, the pair checksum);
//            an exclusive scan of the counts gives every item's output offset,
//            and the grand total is the one value read back to the host
//   write  - the same build + probe, each probe row writing its matches at its
//            block-scanned position (output columns are structure-of-arrays)
//
// Table layout (per block, shared memory): build keys keys_s[cap]; slot words
// (tag16 << 16 | head+1) over 2^k >= 2*rows slots with linear probing; one
// slot per DISTINCT key, with its member count cnt[] and a member chain nxt[]
// through the build rows, so duplicate keys cost one slot and the probe finds a
// key in O(1) however many copies it has.
#include <string.h>

#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr int kJoinThreads = 512;
constexpr uint32_t kDefaultCap = 4096;
constexpr uint32_t kMaxCap = 16384;
constexpr uint32_t kRightChunk = 65536;  // probe rows per work item
constexpr int MODE_COUNT = 0, MODE_CHECKSUM = 1, MODE_WRITE = 2;

struct JSide {
  const void *key;
  const uint32_t *rid;  // NULL: identity
  const uint32_t *off;  // bucket offsets [nbuckets + 1]
  const void *cols[MDJ_MAX_COLS];
  int32_t width[MDJ_MAX_COLS];
  int32_t ncols;
};

struct JOut {
  void *key;
  uint32_t *lrow;
  uint32_t *rrow;
  void *lcols[MDJ_MAX_COLS];
  void *rcols[MDJ_MAX_COLS];
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename KeyT>
size_t join_smem_bytes(uint32_t cap, int mode) {
  const size_t t = 2 * (size_t)cap;
  size_t b = align16((size_t)cap * sizeof(KeyT) + (size_t)cap * 2) + t * 8;
  if (mode == MODE_CHECKSUM) b += t * 8;
  return b;
}

__device__ __forceinline__ uint64_t pay_bits(const void *col, int width, uint32_t i) {
  if (!col) return 0;
  return width == 8 ? ((const uint64_t *)col)[i] : (uint64_t)((const uint32_t *)col)[i];
}

// checksum terms (mdj_count_checksum)
__device__ __forceinline__ uint64_t term_f(uint64_t kbits, uint32_t lrow, uint64_t pbits) {
  return fmix64(kbits ^ (0x9E3779B97F4A7C15ULL * ((uint64_t)lrow + 1)) ^ pbits);
}
__device__ __forceinline__ uint64_t term_g(uint32_t rrow, uint64_t pbits) {
  return fmix64((0xC2B2AE3D27D4EB4FULL * ((uint64_t)rrow + 1)) ^ pbits);
}

// Work items of bucket b: ceil(nl / cap) build chunks x ceil(nr / kRightChunk)
// probe chunks (0 when either side is empty).
__global__ void k_items(const uint32_t *__restrict__ offL, const uint32_t *__restrict__ offR, uint32_t nb, uint32_t cap,
                        uint64_t *__restrict__ items) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) {
    uint64_t nl = offL[b + 1] - offL[b], nr = offR[b + 1] - offR[b];
    items[b] = (nl && nr) ? ((nl + cap - 1) / cap) * ((nr + kRightChunk - 1) / kRightChunk) : 0ull;
  } else if (b == nb) {
    items[nb] = 0;
  }
}

template <typename KeyT, int MODE>
__global__ void __launch_bounds__(kJoinThreads, 2)
    k_join(JSide L, JSide R, const uint64_t *__restrict__ item_off, uint32_t nb, uint32_t nitems, uint32_t cap,
           uint64_t *__restrict__ item_cnt, unsigned long long *__restrict__ chk, const uint64_t *__restrict__ out_off,
           JOut out) {
  extern __shared__ __align__(16) unsigned char smem[];
  KeyT *keys_s = (KeyT *)smem;
  uint16_t *nxt = (uint16_t *)(smem + (size_t)cap * sizeof(KeyT));
  uint32_t *slots = (uint32_t *)(smem + align16((size_t)cap * sizeof(KeyT) + (size_t)cap * 2));
  uint32_t *cnt = slots + 2 * cap;
  uint64_t *fsum = (uint64_t *)(cnt + 2 * cap);
  __shared__ uint32_t s_item[3];
  __shared__ uint32_t scratch32[33];
  __shared__ uint64_t scratch64[33];

  const KeyT *__restrict__ Lkey = (const KeyT *)L.key;
  const KeyT *__restrict__ Rkey = (const KeyT *)R.key;
  for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    if (threadIdx.x == 0) {
      uint32_t lo = 0, hi = nb - 1;  // last bucket b with item_off[b] <= it
      while (lo < hi) {
        uint32_t mid = (lo + hi + 1) / 2;
        if (item_off[mid] <= it)
          lo = mid;
        else
          hi = mid - 1;
      }
      const uint32_t local = (uint32_t)(it - item_off[lo]);
      const uint32_t nr = R.off[lo + 1] - R.off[lo];
      const uint32_t nrc = (nr + kRightChunk - 1) / kRightChunk;
      s_item[0] = lo;
      s_item[1] = local / nrc;
      s_item[2] = local % nrc;
    }
    __syncthreads();
    const uint32_t b = s_item[0], lc = s_item[1], rc = s_item[2];
    const uint32_t lbeg = L.off[b] + lc * cap;
    const uint32_t lend = (uint32_t)min((uint64_t)lbeg + cap, (uint64_t)L.off[b + 1]);
    const uint32_t nl = lend - lbeg;
    const uint32_t rbeg = R.off[b] + rc * kRightChunk;
    const uint32_t rend = (uint32_t)min((uint64_t)rbeg + kRightChunk, (uint64_t)R.off[b + 1]);
    uint32_t logt = 5;
    while ((1u << logt) < 2 * nl) logt++;
    const uint32_t tsz = 1u << logt, mask = tsz - 1;

    // ---- build
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) keys_s[i] = Lkey[lbeg + i];
    for (uint32_t s = threadIdx.x; s < tsz; s += blockDim.x) {
      slots[s] = 0;
      cnt[s] = 0;
      if (MODE == MODE_CHECKSUM) fsum[s] = 0;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) {
      const KeyT k = keys_s[i];
      const uint64_t h = fmix64(key_bits(k));
      const uint32_t tag = (uint32_t)(h >> 32) & 0xFFFFu;
      const uint32_t w = (tag << 16) | (i + 1);
      uint32_t s = (uint32_t)h >> (32 - logt);
      for (uint32_t probe = 0; probe < tsz; probe++) {
        uint32_t cur = slots[s];
        if (cur == 0) {
          uint32_t prev = atomicCAS(&slots[s], 0u, w);
          if (prev == 0) {
            nxt[i] = 0;
            break;
          }
          cur = prev;
        }
        if ((cur >> 16) == tag && keys_s[(cur & 0xFFFFu) - 1] == k) {
          uint32_t prev = atomicExch(&slots[s], w);
          nxt[i] = (uint16_t)(prev & 0xFFFFu);
          break;
        }
        s = (s + 1) & mask;
      }
      atomicAdd(&cnt[s], 1u);
      if (MODE == MODE_CHECKSUM) {
        const uint32_t lr = L.rid ? L.rid[lbeg + i] : lbeg + i;
        const uint64_t pb = L.ncols > 0 ? pay_bits(L.cols[0], L.width[0], lbeg + i) : 0ull;
        atomicAdd((unsigned long long *)&fsum[s], (unsigned long long)term_f(key_bits(k), lr, pb));
      }
    }
    __syncthreads();

    // ---- probe
    if (MODE != MODE_WRITE) {
      uint64_t acc = 0, csum = 0;
      for (uint32_t r = rbeg + threadIdx.x; r < rend; r += blockDim.x) {
        const KeyT k = Rkey[r];
        const uint64_t h = fmix64(key_bits(k));
        const uint32_t tag = (uint32_t)(h >> 32) & 0xFFFFu;
        uint32_t s = (uint32_t)h >> (32 - logt);
        for (uint32_t probe = 0; probe < tsz; probe++) {
          const uint32_t w = slots[s];
          if (w == 0) break;
          if ((w >> 16) == tag && keys_s[(w & 0xFFFFu) - 1] == k) {
            acc += cnt[s];
            if (MODE == MODE_CHECKSUM) {
              const uint32_t rr = R.rid ? R.rid[r] : r;
              const uint64_t pb = R.ncols > 0 ? pay_bits(R.cols[0], R.width[0], r) : 0ull;
              csum += term_g(rr, pb) * fsum[s];
            }
            break;
          }
          s = (s + 1) & mask;
        }
      }
      acc = warp_sum(acc);
      if (MODE == MODE_CHECKSUM) csum = warp_sum(csum);
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      if (lane == 0) {
        scratch64[warp] = acc;
        if (MODE == MODE_CHECKSUM) scratch64[16 + warp] = csum;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint64_t a = 0, c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
          a += scratch64[w];
          if (MODE == MODE_CHECKSUM) c += scratch64[16 + w];
        }
        item_cnt[it] = a;
        if (MODE == MODE_CHECKSUM) atomicAdd(chk, (unsigned long long)c);
      }
    } else {
      uint64_t base = out_off[it];
      KeyT *okey = (KeyT *)out.key;
      for (uint32_t r0 = rbeg; r0 < rend; r0 += blockDim.x) {
        const uint32_t r = r0 + threadIdx.x;
        uint32_t c = 0, head = 0;
        KeyT k = KeyT(0);
        if (r < rend) {
          k = Rkey[r];
          const uint64_t h = fmix64(key_bits(k));
          const uint32_t tag = (uint32_t)(h >> 32) & 0xFFFFu;
          uint32_t s = (uint32_t)h >> (32 - logt);
          for (uint32_t probe = 0; probe < tsz; probe++) {
            const uint32_t w = slots[s];
            if (w == 0) break;
            if ((w >> 16) == tag && keys_s[(w & 0xFFFFu) - 1] == k) {
              c = cnt[s];
              head = w & 0xFFFFu;
              break;
            }
            s = (s + 1) & mask;
          }
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<uint32_t>(c, scratch32, &tot);
        if (c) {
          const uint64_t pos0 = base + ex;
          const uint32_t rr = R.rid ? R.rid[r] : r;
          uint32_t li = head - 1;
          for (uint32_t q = 0; q < c; q++) {
            const uint64_t pos = pos0 + q;
            const uint32_t lrow = lbeg + li;
            okey[pos] = k;
            out.lrow[pos] = L.rid ? L.rid[lrow] : lrow;
            out.rrow[pos] = rr;
            for (int j = 0; j < L.ncols; j++) {
              if (L.width[j] == 8)
                ((uint64_t *)out.lcols[j])[pos] = ((const uint64_t *)L.cols[j])[lrow];
              else
                ((uint32_t *)out.lcols[j])[pos] = ((const uint32_t *)L.cols[j])[lrow];
            }
            for (int j = 0; j < R.ncols; j++) {
              if (R.width[j] == 8)
                ((uint64_t *)out.rcols[j])[pos] = ((const uint64_t *)R.cols[j])[r];
              else
                ((uint32_t *)out.rcols[j])[pos] = ((const uint32_t *)R.cols[j])[r];
            }
            li = (uint32_t)nxt[li] - 1;
          }
        }
        base += tot;
      }
    }
    __syncthreads();
  }
}

JSide to_jside(const Side &s) {
  JSide j;
  memset(&j, 0, sizeof j);
  j.key = s.key;
  j.rid = s.rid;
  j.off = s.off;
  j.ncols = s.ncols;
  for (int c = 0; c < s.ncols; c++) {
    j.cols[c] = s.cols[c];
    j.width[c] = s.widths[c];
  }
  return j;
}

template <typename KeyT>
int set_join_attrs(uint32_t cap) {
  static uint32_t done_cap = 0;
  if (done_cap >= cap) return MDJ_OK;
  MDJ_CUDA_TRY(cudaFuncSetAttribute(k_join<KeyT, MODE_COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)join_smem_bytes<KeyT>(cap, MODE_COUNT)));
  MDJ_CUDA_TRY(cudaFuncSetAttribute(k_join<KeyT, MODE_WRITE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)join_smem_bytes<KeyT>(cap, MODE_WRITE)));
  MDJ_CUDA_TRY(cudaFuncSetAttribute(k_join<KeyT, MODE_CHECKSUM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)join_smem_bytes<KeyT>(cap, MODE_CHECKSUM)));
  done_cap = cap;
  return MDJ_OK;
}

int join_grid(size_t smem, uint32_t max_items) {
  int per_sm = (int)((227 * 1024) / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  uint64_t g = (uint64_t)num_sms() * per_sm;
  if (g > max_items) g = max_items;
  return (int)(g ? g : 1);
}

// count (or checksum) pass + scan + readback; then the write pass.
template <typename KeyT>
int run_join(Workspace &ws, const Side &Ls, const Side &Rs, const Plan &plan, bool checksum_mode,
             mdj_result *res, uint64_t *count, uint64_t *checksum) {
  cudaStream_t s = ws.stream();
  const uint32_t nb = plan.nbuckets, cap = plan.cap;
  MDJ_TRY(set_join_attrs<KeyT>(cap));
  const JSide L = to_jside(Ls), R = to_jside(Rs);

  uint64_t *item_off = (uint64_t *)ws.get((size_t)(nb + 1) * 8);
  if (!item_off) return MDJ_ERR_OOM;
  {
    TraceScope tr("join_items", s);
    k_items<<<(nb + 1 + 255) / 256, 256, 0, s>>>(Ls.off, Rs.off, nb, cap, item_off);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u64(ws, item_off, item_off, nb + 1));
  uint64_t nitems = 0;
  MDJ_CUDA_TRY(cudaMemcpyAsync(&nitems, item_off + nb, 8, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (nitems >= (1ull << 31)) return MDJ_ERR_TOO_LARGE;
  const uint64_t max_items = nitems;

  uint64_t *item_cnt = (uint64_t *)ws.get((size_t)(max_items + 1) * 8);
  unsigned long long *chk = (unsigned long long *)ws.get(16);
  if (!item_cnt || !chk) return MDJ_ERR_OOM;
  MDJ_CUDA_TRY(cudaMemsetAsync(item_cnt, 0, (size_t)(max_items + 1) * 8, s));
  MDJ_CUDA_TRY(cudaMemsetAsync(chk, 0, 16, s));

  JOut none;
  memset(&none, 0, sizeof none);
  if (checksum_mode) {
    const size_t sm = join_smem_bytes<KeyT>(cap, MODE_CHECKSUM);
    TraceScope tr("join_checksum", s);
    k_join<KeyT, MODE_CHECKSUM><<<join_grid(sm, (uint32_t)max_items), kJoinThreads, sm, s>>>(
        L, R, item_off, nb, (uint32_t)nitems, cap, item_cnt, chk, nullptr, none);
  } else {
    const size_t sm = join_smem_bytes<KeyT>(cap, MODE_COUNT);
    TraceScope tr("join_count", s);
    k_join<KeyT, MODE_COUNT><<<join_grid(sm, (uint32_t)max_items), kJoinThreads, sm, s>>>(
        L, R, item_off, nb, (uint32_t)nitems, cap, item_cnt, nullptr, nullptr, none);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u64(ws, item_cnt, item_cnt, max_items + 1));

  uint64_t host[2] = {0, 0};
  MDJ_CUDA_TRY(cudaMemcpyAsync(&host[0], item_cnt + max_items, 8, cudaMemcpyDeviceToHost, s));
  if (checksum_mode) MDJ_CUDA_TRY(cudaMemcpyAsync(&host[1], chk, 8, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  const uint64_t m = host[0];
  if (checksum_mode) {
    *count = m;
    *checksum = host[1];
    return MDJ_OK;
  }
  if (count) *count = m;

  // ---- outputs (owned by the caller)
  mdj_result r;
  memset(&r, 0, sizeof r);
  r.nrows = m;
  r.key_dtype = Ls.key_dtype;
  r.n_left_cols = Ls.ncols;
  r.n_right_cols = Rs.ncols;
  for (int j = 0; j < Ls.ncols; j++) r.left_dtypes[j] = Ls.dtypes[j];
  for (int j = 0; j < Rs.ncols; j++) r.right_dtypes[j] = Rs.dtypes[j];
  if (m > 0) {
    bool ok = true;
    r.key = ws.get_owned_by_caller(m * sizeof(KeyT));
    r.left_row = (uint32_t *)ws.get_owned_by_caller(m * 4);
    r.right_row = (uint32_t *)ws.get_owned_by_caller(m * 4);
    ok = r.key && r.left_row && r.right_row;
    for (int j = 0; ok && j < Ls.ncols; j++) ok = (r.left_cols[j] = ws.get_owned_by_caller(m * Ls.widths[j])) != nullptr;
    for (int j = 0; ok && j < Rs.ncols; j++) ok = (r.right_cols[j] = ws.get_owned_by_caller(m * Rs.widths[j])) != nullptr;
    if (!ok) {
      mdj_result_release(&r, ws.allocator(), (void *)s);
      return MDJ_ERR_OOM;
    }
    JOut o;
    memset(&o, 0, sizeof o);
    o.key = r.key;
    o.lrow = r.left_row;
    o.rrow = r.right_row;
    for (int j = 0; j < Ls.ncols; j++) o.lcols[j] = r.left_cols[j];
    for (int j = 0; j < Rs.ncols; j++) o.rcols[j] = r.right_cols[j];
    const size_t sm = join_smem_bytes<KeyT>(cap, MODE_WRITE);
    {
      TraceScope tr("join_write", s);
      k_join<KeyT, MODE_WRITE><<<join_grid(sm, (uint32_t)max_items), kJoinThreads, sm, s>>>(
          L, R, item_off, nb, (uint32_t)nitems, cap, nullptr, nullptr, item_cnt, o);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      mdj_result_release(&r, ws.allocator(), (void *)s);
      return cuda_status(e);
    }
  }
  *res = r;
  return MDJ_OK;
}

// ------------------------------------------------------------- validation

int check_table(const mdj_table *t, int32_t key_col) {
  if (!t || !t->cols || t->ncols < 1 || t->ncols > MDJ_MAX_COLS) return MDJ_ERR_INVALID_ARG;
  if (key_col < 0 || key_col >= t->ncols) return MDJ_ERR_INVALID_ARG;
  if (t->nrows >= (1ull << 32)) return MDJ_ERR_TOO_LARGE;
  for (int j = 0; j < t->ncols; j++) {
    if (dtype_width(t->cols[j].dtype) == 0) return MDJ_ERR_UNSUPPORTED_DTYPE;
    if (t->nrows > 0 && !t->cols[j].data) return MDJ_ERR_INVALID_ARG;
  }
  const int32_t kd = t->cols[key_col].dtype;
  if (kd != MDJ_I32 && kd != MDJ_I64) return MDJ_ERR_UNSUPPORTED_DTYPE;
  return MDJ_OK;
}

uint32_t cap_from_env() {
  static uint32_t cap = 0;
  if (!cap) {
    cap = kDefaultCap;
    const char *e = getenv("MDJ_TABLE_ROWS");
    if (e) {
      long v = atol(e);
      if (v >= 256 && v <= (long)kMaxCap) cap = (uint32_t)v;
    }
  }
  return cap;
}

int merge_impl(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P,
               const mdj_allocator *alloc, void *stream, mdj_result *out, bool checksum_mode, uint64_t *count,
               uint64_t *checksum) {
  MDJ_TRY(check_table(left, lk));
  MDJ_TRY(check_table(right, rk));
  if (P < 1 || P > MDJ_MAX_PARTITIONS) return MDJ_ERR_INVALID_ARG;
  if (left->cols[lk].dtype != right->cols[rk].dtype) return MDJ_ERR_INVALID_ARG;
  if (!checksum_mode && !out) return MDJ_ERR_INVALID_ARG;
  if (checksum_mode && (!count || !checksum)) return MDJ_ERR_INVALID_ARG;
  if (out) memset(out, 0, sizeof *out);

  Workspace ws(alloc, (cudaStream_t)stream);
  const Plan plan = make_plan(left->nrows, P, cap_from_env(), P > 1);
  Side L, R;
  MDJ_TRY(partition_side(ws, left, lk, plan, &L));
  MDJ_TRY(partition_side(ws, right, rk, plan, &R));
  if (left->cols[lk].dtype == MDJ_I64) return run_join<int64_t>(ws, L, R, plan, checksum_mode, out, count, checksum);
  return run_join<int32_t>(ws, L, R, plan, checksum_mode, out, count, checksum);
}

}  // namespace
}  // namespace mdj

using namespace mdj;

extern "C" {

int mdj_partition(const mdj_table *in, int32_t key_col, uint32_t P, void *const *out_cols, uint32_t *out_row_ids,
                  int64_t *out_offsets, const mdj_allocator *alloc, void *stream) {
  MDJ_TRY(check_table(in, key_col));
  if (P < 1 || P > MDJ_MAX_PARTITIONS || !out_cols || !out_offsets) return MDJ_ERR_INVALID_ARG;
  if (in->nrows > 0)
    for (int j = 0; j < in->ncols; j++)
      if (!out_cols[j]) return MDJ_ERR_INVALID_ARG;
  Workspace ws(alloc, (cudaStream_t)stream);
  return stable_partition(ws, in, key_col, P, out_cols, out_row_ids, out_offsets);
}

int mdj_join(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
             const mdj_allocator *alloc, void *stream, mdj_result *out) {
  return merge_impl(left, left_key, right, right_key, 1, alloc, stream, out, false, nullptr, nullptr);
}

int mdj_merge(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key, uint32_t P,
              const mdj_allocator *alloc, void *stream, mdj_result *out) {
  return merge_impl(left, left_key, right, right_key, P, alloc, stream, out, false, nullptr, nullptr);
}

int mdj_count_checksum(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
                       uint32_t P, const mdj_allocator *alloc, void *stream, uint64_t *count, uint64_t *checksum) {
  return merge_impl(left, left_key, right, right_key, P, alloc, stream, nullptr, true, count, checksum);
}

}  // extern "C"
