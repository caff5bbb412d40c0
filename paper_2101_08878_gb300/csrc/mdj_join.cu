// The per-partition merge: an inner hash join of co-partitioned tables
// (Sec. V-B: the benchmark merges the shuffled data frames).
//
// Both sides are bucketed with the same hash (partition p, then sub-bucket),
// so equal keys share a bucket.  A work item is (bucket, chunk of at most `cap`
// build rows, chunk of probe rows); one block builds a hash table of the build
// chunk in shared memory and probes the probe chunk against it.
//
// Output (the two phases of a count-then-write materialisation, fused per
// item): an item first counts its matches (block scan over its probe rows),
// then learns where its rows go from the items before it by a decoupled
// look-back over per-item counts (items are taken in order from an atomic
// ticket, so every predecessor is already running; every wait is bounded), and
// writes them there.  The output buffer is sized optimistically (max(n_L, n_R)
// rows, exact whenever build keys are unique); if the join is larger, the
// counts are already known, so one exact write pass at the recorded item
// offsets follows.  The grand total is the one value read back to the host.
//
// Table layout (per block, shared memory): build keys keys_s[cap]; slot words
// (tag16 << 16 | head+1) over 2^k >= 2*rows slots with linear probing; one
// slot per DISTINCT key, with its member count cnt[] and a member chain nxt[]
// through the build rows, so duplicate keys cost one slot and the probe finds a
// key in O(1) however many copies it has.  Slots and tags come from a cheap
// multiplicative hash of the key: bucket membership was already randomised by
// the partition hash.
#include <string.h>

#include "mdj_internal.cuh"
#include "mdj_join_dev.cuh"
#include "mdj_shuffle_dev.cuh"
#include "mdj_tma.cuh"

namespace mdj {
namespace {


template <typename KeyT>
size_t join_smem_bytes(uint32_t cap, bool fsum) {
  size_t t = 32;
  while (t < 2 * (size_t)cap) t *= 2;  // slots of the largest table
  size_t b = align16((size_t)cap * sizeof(KeyT) + (size_t)cap * 2) + t * 8;
  if (fsum) b += t * 8;
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

// In-table position: top logt bits of key * golden-ratio constant; tag: bits 32..47.
__device__ __forceinline__ void slot_tag(uint64_t kb, uint32_t logt, uint32_t &slot, uint32_t &tag) {
  const uint64_t g = kb * 0x9E3779B97F4A7C15ULL;
  slot = (uint32_t)(g >> (64 - logt));
  tag = (uint32_t)(g >> 32) & 0xFFFFu;
}

// ------------------------------------------------------------- work items

// Items of bucket b: ceil(nl / cap) build chunks x ceil(nr / rch) probe chunks
// (0 when either side is empty).
__global__ void k_items(const uint32_t *__restrict__ offL, const uint32_t *__restrict__ offR, uint32_t nb, uint32_t cap,
                        uint32_t rch, uint64_t *__restrict__ items) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) {
    uint64_t nl = offL[b + 1] - offL[b], nr = offR[b + 1] - offR[b];
    items[b] = (nl && nr) ? ((nl + cap - 1) / cap) * ((nr + rch - 1) / rch) : 0ull;
  } else if (b == nb) {
    items[nb] = 0;
  }
}

// One descriptor per item: its build and probe row ranges.
__global__ void k_expand(const uint32_t *__restrict__ offL, const uint32_t *__restrict__ offR, uint32_t nb,
                         uint32_t cap, uint32_t rch, const uint64_t *__restrict__ item_off, uint32_t nitems,
                         Item *__restrict__ desc) {
  for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < nitems; it += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = nb - 1;  // last bucket b with item_off[b] <= it
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) / 2;
      if (item_off[mid] <= it)
        lo = mid;
      else
        hi = mid - 1;
    }
    const uint32_t local = (uint32_t)(it - item_off[lo]);
    const uint32_t nl = offL[lo + 1] - offL[lo], nr = offR[lo + 1] - offR[lo];
    const uint32_t nrc = (nr + rch - 1) / rch;
    const uint32_t lc = local / nrc, rc = local % nrc;
    Item d;
    d.lbeg = offL[lo] + lc * cap;
    d.nl = min(cap, nl - lc * cap);
    d.rbeg = offR[lo] + rc * rch;
    d.nr = min(rch, nr - rc * rch);
    desc[it] = d;
  }
}

// ------------------------------------------------------------ table build

template <typename KeyT>
__device__ __forceinline__ uint32_t table_log(uint32_t nl) {
  uint32_t logt = 5;
  while ((1u << logt) < 2 * nl) logt++;
  return logt;
}

// Loads the build keys into shared memory and clears 2^logt slots.
template <typename KeyT, bool FSUM>
__device__ __forceinline__ void load_and_clear(const KeyT *__restrict__ Lkey, uint32_t lbeg, uint32_t nl, uint32_t tsz,
                                               KeyT *keys_s, uint32_t *slots, uint32_t *cnt, uint64_t *fsum) {
  const uint32_t nthr = blockDim.x, tid = threadIdx.x;
  for (uint32_t i0 = 0; i0 < nl; i0 += 4 * nthr) {
    KeyT v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t i = i0 + u * nthr + tid;
      v[u] = i < nl ? Lkey[lbeg + i] : KeyT(0);
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t i = i0 + u * nthr + tid;
      if (i < nl) keys_s[i] = v[u];
    }
  }
  uint4 z = make_uint4(0, 0, 0, 0);
  for (uint32_t s = tid * 4; s < tsz; s += nthr * 4) {
    *(uint4 *)(slots + s) = z;
    *(uint4 *)(cnt + s) = z;
  }
  if (FSUM)
    for (uint32_t s = tid * 2; s < tsz; s += nthr * 2) *(uint4 *)(fsum + s) = z;
}

// One slot per distinct key; rows of a key are chained through nxt[] (head =
// the slot word's index, most recent insert first) and counted in cnt[].
template <typename KeyT, bool FSUM>
__device__ __forceinline__ void build_table(const KeyT *keys_s, uint32_t nl, uint32_t logt, uint32_t *slots,
                                            uint32_t *cnt, uint16_t *nxt, uint64_t *fsum, const JSide &L,
                                            uint32_t lbeg) {
  const uint32_t mask = (1u << logt) - 1;
  for (uint32_t i = threadIdx.x; i < nl; i += blockDim.x) {
    const KeyT k = keys_s[i];
    uint32_t s, tag;
    slot_tag(key_bits(k), logt, s, tag);
    const uint32_t w = (tag << 16) | (i + 1);
    for (uint32_t probe = 0; probe <= mask; probe++) {
      uint32_t cur = slots[s];
      if (cur == 0) {
        const uint32_t prev = atomicCAS(&slots[s], 0u, w);
        if (prev == 0) {
          nxt[i] = 0;
          break;
        }
        cur = prev;
      }
      if ((cur >> 16) == tag && keys_s[(cur & 0xFFFFu) - 1] == k) {
        const uint32_t prev = atomicExch(&slots[s], w);
        nxt[i] = (uint16_t)(prev & 0xFFFFu);
        break;
      }
      s = (s + 1) & mask;
    }
    atomicAdd(&cnt[s], 1u);
    if (FSUM) {
      const uint32_t lr = L.rid ? L.rid[lbeg + i] : lbeg + i;
      const uint64_t pb = L.ncols > 0 ? pay_bits(L.cols[0], L.width[0], lbeg + i) : 0ull;
      atomicAdd((unsigned long long *)&fsum[s], (unsigned long long)term_f(key_bits(k), lr, pb));
    }
  }
}

// Probe: slot of key k (or where the search ended) and the chain head (0: absent).
template <typename KeyT>
__device__ __forceinline__ uint32_t probe_table(const KeyT k, const KeyT *keys_s, const uint32_t *slots, uint32_t logt,
                                                uint32_t &slot_out) {
  const uint32_t mask = (1u << logt) - 1;
  uint32_t s, tag;
  slot_tag(key_bits(k), logt, s, tag);
  uint32_t head = 0;
  for (uint32_t probe = 0; probe <= mask; probe++) {
    const uint32_t w = slots[s];
    if (w == 0) break;
    if ((w >> 16) == tag && keys_s[(w & 0xFFFFu) - 1] == k) {
      head = w & 0xFFFFu;
      break;
    }
    s = (s + 1) & mask;
  }
  slot_out = s;
  return head;
}

__device__ __forceinline__ uint32_t next_ticket(uint32_t *ticket, uint32_t *s_it) {
  if (threadIdx.x == 0) *s_it = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t it = *s_it;
  __syncthreads();
  return it;
}

// ---------------------------------------------------- count (+ checksum)

// Pair count (and pair checksum) of every item, summed into totals[0..1].
template <typename KeyT, bool CHECKSUM>
__global__ void __launch_bounds__(kJoinThreads, 2)
    k_join_count(JSide L, JSide R, const Item *__restrict__ desc, uint32_t nitems, uint32_t *ticket,
                 unsigned long long *totals) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_it;
  const KeyT *__restrict__ Lkey = (const KeyT *)L.key;
  const KeyT *__restrict__ Rkey = (const KeyT *)R.key;
  const uint32_t nthr = blockDim.x, tid = threadIdx.x;
  for (;;) {
    const uint32_t it = next_ticket(ticket, &s_it);
    if (it >= nitems) break;
    const Item d = desc[it];
    const uint32_t logt = table_log<KeyT>(d.nl), tsz = 1u << logt;
    KeyT *keys_s = (KeyT *)smem;
    uint16_t *nxt = (uint16_t *)(smem + (size_t)d.nl * sizeof(KeyT));
    uint32_t *slots = (uint32_t *)(smem + align16((size_t)d.nl * (sizeof(KeyT) + 2)));
    uint32_t *cnt = slots + tsz;
    uint64_t *fsum = (uint64_t *)(cnt + tsz);
    load_and_clear<KeyT, CHECKSUM>(Lkey, d.lbeg, d.nl, tsz, keys_s, slots, cnt, fsum);
    __syncthreads();
    build_table<KeyT, CHECKSUM>(keys_s, d.nl, logt, slots, cnt, nxt, fsum, L, d.lbeg);
    __syncthreads();
    uint64_t acc = 0, csum = 0;
    for (uint32_t r0 = d.rbeg; r0 < d.rbeg + d.nr; r0 += kPF * nthr) {
      KeyT rk[kPF];
#pragma unroll
      for (int j = 0; j < kPF; j++) {
        const uint32_t r = r0 + j * nthr + tid;
        rk[j] = r < d.rbeg + d.nr ? Rkey[r] : KeyT(0);
      }
#pragma unroll
      for (int j = 0; j < kPF; j++) {
        const uint32_t r = r0 + j * nthr + tid;
        if (r < d.rbeg + d.nr) {
          uint32_t slot;
          if (probe_table<KeyT>(rk[j], keys_s, slots, logt, slot)) {
            acc += cnt[slot];
            if (CHECKSUM) {
              const uint32_t rr = R.rid ? R.rid[r] : r;
              const uint64_t pb = R.ncols > 0 ? pay_bits(R.cols[0], R.width[0], r) : 0ull;
              csum += term_g(rr, pb) * fsum[slot];
            }
          }
        }
      }
    }
    acc = warp_sum(acc);
    if (CHECKSUM) csum = warp_sum(csum);
    if ((tid & 31) == 0) {
      if (acc) atomicAdd(&totals[0], (unsigned long long)acc);
      if (CHECKSUM && csum) atomicAdd(&totals[1], (unsigned long long)csum);
    }
    __syncthreads();
  }
}

template <typename KeyT, bool HAVE_OFFSETS>
__global__ void __launch_bounds__(kWT, 2)
    k_join_write(JSide L, JSide R, const Item *__restrict__ desc, uint32_t nitems, uint32_t cap, uint32_t *ticket,
                 unsigned long long *state, uint64_t *__restrict__ item_off, unsigned long long *total,
                 uint64_t capacity, int *flags, int withhold_first, int ordered, JOut out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Item s_item;
  __shared__ uint32_t s_it;
  __shared__ JoinShared js;
  const uint32_t tid = threadIdx.x;
  const Resv rs = {state, item_off, total, capacity, flags, withhold_first, ordered};
  if (tid == 0) {
    s_it = atomicAdd(ticket, 1u);
    if (s_it < nitems) s_item = desc[s_it];
  }
  __syncthreads();
  for (;;) {
    const uint32_t it = s_it;
    if (it >= nitems) break;
    const Item d = s_item;
    // next ticket: fetched now, published at the end of this item
    uint32_t nx = 0;
    Item dn = {0, 0, 0, 0};
    if (tid == 0) {
      nx = atomicAdd(ticket, 1u);
      if (nx < nitems) dn = desc[nx];
    }
    join_item<KeyT, HAVE_OFFSETS>(smem, cap, L, R, d, it, rs, out, js);
    if (tid == 0) {
      s_it = nx;
      if (nx < nitems) s_item = dn;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- host

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

template <typename KernelT>
int resident_grid(KernelT kernel, size_t smem, uint64_t nitems, int *grid, int threads = kJoinThreads) {
  int per_sm = 0;
  MDJ_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  MDJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  if (per_sm < 1) return MDJ_ERR_INTERNAL;
  uint64_t g = (uint64_t)num_sms() * per_sm;
  if (g > nitems) g = nitems;
  *grid = (int)(g ? g : 1);
  return MDJ_OK;
}

// Work items of the whole join, with `rch` probe rows per item at most.
int make_items(Workspace &ws, const Side &Ls, const Side &Rs, uint32_t nb, uint32_t cap, uint32_t rch, Item **desc,
               uint32_t *nitems_out, uint64_t **bucket_items = nullptr) {
  cudaStream_t s = ws.stream();
  uint64_t *item_off = (uint64_t *)ws.get((size_t)(nb + 1) * 8);
  if (!item_off) return MDJ_ERR_OOM;
  {
    TraceScope tr("join_items", s);
    k_items<<<(nb + 1 + 255) / 256, 256, 0, s>>>(Ls.off, Rs.off, nb, cap, rch, item_off);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u64(ws, item_off, item_off, nb + 1));
  uint64_t nitems = 0;
  int part_flag = 0;
  MDJ_CUDA_TRY(cudaMemcpyAsync(&nitems, item_off + nb, 8, cudaMemcpyDeviceToHost, s));
  if (ws.flag_word_if_any()) MDJ_CUDA_TRY(cudaMemcpyAsync(&part_flag, ws.flag_word_if_any(), 4, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (part_flag) return MDJ_ERR_DEVICE_TIMEOUT;  // a partition pass gave up on a copy wait
  if (nitems >= (1ull << 31)) return MDJ_ERR_TOO_LARGE;
  *nitems_out = (uint32_t)nitems;
  *desc = (Item *)ws.get((size_t)(nitems ? nitems : 1) * sizeof(Item));
  if (!*desc) return MDJ_ERR_OOM;
  if (nitems) {
    TraceScope tr("join_expand", s);
    const uint64_t want = (nitems + 255) / 256, most = (uint64_t)num_sms() * 8;
    const unsigned g = (unsigned)(want < most ? want : most);
    k_expand<<<g, 256, 0, s>>>(Ls.off, Rs.off, nb, cap, rch, item_off, (uint32_t)nitems, *desc);
  }
  MDJ_LAUNCH_CHECK();
  if (bucket_items)
    *bucket_items = item_off;
  else
    ws.give_back(item_off);
  return MDJ_OK;
}

template <typename KeyT>
int run_count(Workspace &ws, const Side &Ls, const Side &Rs, const Plan &plan, uint64_t *count, uint64_t *checksum) {
  cudaStream_t s = ws.stream();
  Item *desc;
  uint32_t nitems;
  const uint32_t cap = plan.cap < kCountCapMax ? plan.cap : kCountCapMax;
  MDJ_TRY(make_items(ws, Ls, Rs, plan.nbuckets, cap, kCountChunk, &desc, &nitems));
  unsigned long long *tot = (unsigned long long *)ws.get(32);
  if (!tot) return MDJ_ERR_OOM;
  MDJ_CUDA_TRY(cudaMemsetAsync(tot, 0, 32, s));
  uint32_t *ticket = (uint32_t *)(tot + 2);
  if (nitems) {
    const size_t sm = join_smem_bytes<KeyT>(cap, true);
    int grid;
    MDJ_TRY(resident_grid(k_join_count<KeyT, true>, sm, nitems, &grid));
    TraceScope tr("join_checksum", s);
    k_join_count<KeyT, true><<<grid, kJoinThreads, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems, ticket, tot);
  }
  MDJ_LAUNCH_CHECK();
  unsigned long long host[2] = {0, 0};
  MDJ_CUDA_TRY(cudaMemcpyAsync(host, tot, 16, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  *count = host[0];
  *checksum = host[1];
  return MDJ_OK;
}

int alloc_result(Workspace &ws, const Side &Ls, const Side &Rs, size_t key_width, uint64_t rows, mdj_result *r,
                 JOut *o) {
  memset(r, 0, sizeof *r);
  r->key_dtype = Ls.key_dtype;
  r->n_left_cols = Ls.ncols;
  r->n_right_cols = Rs.ncols;
  for (int j = 0; j < Ls.ncols; j++) r->left_dtypes[j] = Ls.dtypes[j];
  for (int j = 0; j < Rs.ncols; j++) r->right_dtypes[j] = Rs.dtypes[j];
  memset(o, 0, sizeof *o);
  if (rows == 0) return MDJ_OK;
  bool ok = (r->key = ws.get_owned_by_caller(rows * key_width)) != nullptr;
  ok = ok && (r->left_row = (uint32_t *)ws.get_owned_by_caller(rows * 4)) != nullptr;
  ok = ok && (r->right_row = (uint32_t *)ws.get_owned_by_caller(rows * 4)) != nullptr;
  for (int j = 0; ok && j < Ls.ncols; j++) ok = (r->left_cols[j] = ws.get_owned_by_caller(rows * Ls.widths[j])) != nullptr;
  for (int j = 0; ok && j < Rs.ncols; j++) ok = (r->right_cols[j] = ws.get_owned_by_caller(rows * Rs.widths[j])) != nullptr;
  if (!ok) {
    mdj_result_release(r, ws.allocator(), (void *)ws.stream());
    return MDJ_ERR_OOM;
  }
  o->key = r->key;
  o->lrow = r->left_row;
  o->rrow = r->right_row;
  for (int j = 0; j < Ls.ncols; j++) o->lcols[j] = r->left_cols[j];
  for (int j = 0; j < Rs.ncols; j++) o->rcols[j] = r->right_cols[j];
  return MDJ_OK;
}

// Test hook: MDJ_TEST_WITHHOLD_FIRST_ITEM=1 makes item 0 of the fused write
// pass never publish its count, so every look-back wait must run out and the
// call must report MDJ_ERR_DEVICE_TIMEOUT with the context still usable.
int test_withhold_first() {
  const char *e = getenv("MDJ_TEST_WITHHOLD_FIRST_ITEM");
  return e && e[0] == '1';
}


// MDJ_ORDERED_OUTPUT=1: item output ranges follow item order (decoupled
// look-back), so the same inputs give byte-identical outputs.  Default: each
// item reserves its range with one atomicAdd (same rows, item order not
// reproducible), which never waits on other items.
int ordered_output() {
  const char *e = getenv("MDJ_ORDERED_OUTPUT");
  return e && e[0] == '1';
}

// Rows of the optimistic output buffer of the fused pass: max(n_L, n_R), the
// exact bound when build keys are unique (MDJ_OUTPUT_ROWS overrides).
uint64_t output_capacity_hint(uint64_t nl, uint64_t nr) {
  uint64_t c = nl > nr ? nl : nr;
  const char *e = getenv("MDJ_OUTPUT_ROWS");
  if (e) {
    long long v = atoll(e);
    if (v >= 0) c = (uint64_t)v;
  }
  return c;
}

// Batch bookkeeping returned by run_join: per-bucket item prefix, per-item
// output offsets (valid in ordered mode) and the item count.
struct ItemMap {
  uint64_t *bucket_items = nullptr;
  uint64_t *item_out = nullptr;
  uint32_t nitems = 0;
};

template <typename KeyT>
int run_join(Workspace &ws, const Side &Ls, const Side &Rs, const Plan &plan, mdj_result *res,
             bool force_ordered = false, ItemMap *map = nullptr) {
  cudaStream_t s = ws.stream();
  // the optimistic output buffer first: its allocation overlaps the device
  // work still queued, before make_items waits for the item count
  const uint64_t cap_rows = output_capacity_hint(Ls.nrows, Rs.nrows);
  mdj_result r;
  JOut o;
  MDJ_TRY(alloc_result(ws, Ls, Rs, sizeof(KeyT), cap_rows, &r, &o));
  Item *desc;
  uint32_t nitems;
  int rc = make_items(ws, Ls, Rs, plan.nbuckets, plan.cap, kWriteChunk, &desc, &nitems,
                      map ? &map->bucket_items : nullptr);
  // state[nitems] | item_off[nitems] | total | ticket | flags
  const size_t words = 2 * (size_t)nitems + 4;
  unsigned long long *state = rc == MDJ_OK ? (unsigned long long *)ws.get(words * 8) : nullptr;
  if (rc == MDJ_OK && !state) rc = MDJ_ERR_OOM;
  if (rc == MDJ_OK) rc = cuda_status(cudaMemsetAsync(state, 0, words * 8, s));
  if (rc != MDJ_OK) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    return rc;
  }
  uint64_t *item_off = (uint64_t *)(state + nitems);
  unsigned long long *total = state + 2 * (size_t)nitems;
  uint32_t *ticket = (uint32_t *)(total + 1);
  int *flags = (int *)(total + 2);

  const size_t sm = WriteLayout<KeyT>(plan.cap).total;  // ~105 KB at cap 4096: two blocks per SM
  if (nitems) {
    int grid;
    MDJ_TRY(resident_grid(k_join_write<KeyT, false>, sm, nitems, &grid, kWT));
    TraceScope tr("join_write", s);
    k_join_write<KeyT, false><<<grid, kWT, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems, plan.cap, ticket,
                                                    state, item_off, total, cap_rows, flags, test_withhold_first(),
                                                    force_ordered ? 1 : ordered_output(), o);
  }
  cudaError_t e = cudaGetLastError();
  unsigned long long host_total = 0;
  int host_flags[FLAG_WORDS] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host_total, total, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_flags, flags, sizeof host_flags, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    return cuda_status(e);
  }
  if (host_flags[FLAG_TIMEOUT]) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    return MDJ_ERR_DEVICE_TIMEOUT;
  }
  const uint64_t m = host_total;
  if (m > cap_rows || m == 0) {
    // the join outgrew the optimistic buffer (or is empty): exact buffers,
    // then one write pass at the offsets the fused pass recorded
    mdj_result_release(&r, ws.allocator(), (void *)s);
    MDJ_TRY(alloc_result(ws, Ls, Rs, sizeof(KeyT), m, &r, &o));
    if (m > 0) {
      int grid;
      MDJ_TRY(resident_grid(k_join_write<KeyT, true>, sm, nitems, &grid, kWT));
      MDJ_CUDA_TRY(cudaMemsetAsync(ticket, 0, 4, s));
      {
        TraceScope tr("join_write_exact", s);
        k_join_write<KeyT, true><<<grid, kWT, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems, plan.cap, ticket,
                                                       state, item_off, total, m, flags, 0, 0, o);
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) {
        mdj_result_release(&r, ws.allocator(), (void *)s);
        return cuda_status(e);
      }
    }
  }
  r.nrows = m;
  *res = r;
  if (map) {
    map->item_out = item_off;
    map->nitems = nitems;
  }
  return MDJ_OK;
}

// ------------------------------------------------- fused pass 2 + join
//
// For a two-level plan the pass-2 copy of every side is written once and read
// once by the join.  k_fused keeps it in L2 instead: pass-1 bucket w (a
// "wave") is split by pass 2 into scratch slot w % kFuseSlots, and its join
// items read the slot right after.  One persistent kernel runs both kinds of
// work units, taken in a fixed order from one ticket:
//   P2(0), P2(1), ..., P2(lag - 1), then P2(w), J(w - lag) for w = lag.. ,
// where P2(w) = the pass-2 tiles of wave w (left side, then right side) and
// J(w) = the join items of wave w.  J(w) waits until every P2(w) tile is done;
// P2(w) waits until every J(w - kFuseSlots) item is done (its slot is free).
// Each wait is on units with smaller tickets, all held by running blocks, so
// the order cannot deadlock; every wait is still bounded (kFuseWaitNs of
// %globaltimer time, then FLAG_TIMEOUT + FLAG_ABORT and the block stops).
// Join units read the slot through L2 only (join_item's COHERENT mode).

constexpr uint32_t kFuseSlots = 4;
constexpr uint32_t kFuseLag = 2;
constexpr uint64_t kFuseWaitNs = 2000000000ull;
constexpr uint32_t kFuseTile = shuffle_tile<kShuffleNT>();
static_assert(kFuseLag < kFuseSlots, "a wave's slot is reused only after its items ran");

struct FuseWave {
  uint32_t row0[2], rows[2];  // the wave's rows on each side (pass-1 order = final region)
  uint32_t tiles[2];          // pass-2 tiles per side
  uint32_t item0, nitems;     // its join items
};

// Scratch columns of one side in one slot: key, first payload, row ids.
struct FuseSideSlot {
  size_t key, pay, rid;  // byte offsets in the side's part of a slot
  size_t bytes;          // the side's part of a slot
};

struct FuseArgs {
  const ColMove *moves;   // [slot][side]: pass-1 copy -> the slot's scratch columns
  const JSide *jsides;    // [slot][side]: the slot's scratch columns as join sides
  const FuseWave *waves;
  const uint32_t *seg_start;  // first unit of each segment (2 * (F1 + lag) + 1 entries)
  uint32_t nseg, F1, F2;
  const Item *desc;
  uint32_t *ticket;
  uint32_t *p2_done, *j_done;  // per wave
  uint32_t *cursors[2];        // absolute sub-bucket cursors per side
  const void *p1_key[2], *p1_pay[2];
  const uint32_t *p1_rid[2];
  int key_w, pay_w[2];         // widths (pay_w 0: no payload column)
  unsigned char *slots;
  size_t slot_bytes;
  FuseSideSlot side[2];
  BucketSpec sub;
  uint32_t cap;
};

// Thread 0 waits until *ctr >= target; false when the wait ran out or another
// block gave up.
__device__ bool fuse_wait(const uint32_t *ctr, uint32_t target, int *flags) {
  volatile const uint32_t *v = ctr;
  if (*v >= target) {
    __threadfence();
    return true;
  }
  const uint64_t t0 = globaltimer_ns();
  while (*v < target) {
    if (((volatile int *)flags)[FLAG_ABORT]) return false;
    if (globaltimer_ns() - t0 > kFuseWaitNs) {
      atomicExch(&flags[FLAG_TIMEOUT], 1);
      atomicExch(&flags[FLAG_ABORT], 1);
      return false;
    }
    __nanosleep(200);
  }
  __threadfence();
  return true;
}

// The waves, the unit order (segment starts) and the largest wave per side
// (out[0], out[1]) and the unit count (out[2]); one block of 1024 threads.
__global__ void __launch_bounds__(1024)
    k_fuse_plan(const uint32_t *__restrict__ offL, const uint32_t *__restrict__ offR,
                const uint64_t *__restrict__ bucket_items, uint32_t F1, uint32_t F2, FuseWave *__restrict__ waves,
                uint32_t *__restrict__ seg_start, uint32_t *__restrict__ out) {
  __shared__ uint32_t scratch[40];
  __shared__ uint32_t mx[2];
  if (threadIdx.x < 2) mx[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t w = threadIdx.x; w < F1; w += blockDim.x) {
    FuseWave v;
    const uint32_t a = w * F2, b = (w + 1) * F2;
    v.row0[0] = offL[a];
    v.rows[0] = offL[b] - offL[a];
    v.row0[1] = offR[a];
    v.rows[1] = offR[b] - offR[a];
    v.tiles[0] = (v.rows[0] + kFuseTile - 1) / kFuseTile;
    v.tiles[1] = (v.rows[1] + kFuseTile - 1) / kFuseTile;
    v.item0 = (uint32_t)bucket_items[a];
    v.nitems = (uint32_t)(bucket_items[b] - bucket_items[a]);
    waves[w] = v;
    atomicMax(&mx[0], v.rows[0]);
    atomicMax(&mx[1], v.rows[1]);
  }
  __syncthreads();
  // segment sizes in unit order, then an in-place exclusive scan
  const uint32_t nseg = 2 * (F1 + kFuseLag);
  for (uint32_t s = threadIdx.x; s <= nseg; s += blockDim.x) {
    const uint32_t q = s / 2;
    uint32_t size = 0;
    if (s == nseg) {
      size = 0;
    } else if (s % 2 == 0) {
      if (q < F1) size = waves[q].tiles[0] + waves[q].tiles[1];
    } else if (q >= kFuseLag && q - kFuseLag < F1) {
      size = waves[q - kFuseLag].nitems;
    }
    seg_start[s] = size;
  }
  __syncthreads();
  block_scan_array(seg_start, nseg + 1, scratch);  // seg_start[nseg] = units (its input was 0)
  if (threadIdx.x == 0) {
    out[0] = mx[0];
    out[1] = mx[1];
    out[2] = seg_start[nseg];
  }
}

// Segment of unit u (the last s with seg_start[s] <= u) and u's index in it.
__device__ __forceinline__ void fuse_decode(const FuseArgs &a, uint32_t u, uint32_t *seg, uint32_t *local) {
  uint32_t lo = 0, hi = a.nseg - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) / 2;
    if (a.seg_start[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  *seg = lo;
  *local = u - a.seg_start[lo];
}

// The counter a unit of segment `seg` waits for and its target (ctr = NULL:
// no wait): items of wave w wait for its pass-2 tiles, pass-2 tiles of wave
// w >= kFuseSlots for the items of wave w - kFuseSlots.
__device__ __forceinline__ const uint32_t *fuse_dep(const FuseArgs &a, uint32_t seg, uint32_t *target) {
  const uint32_t q = seg / 2;
  if (seg % 2 == 0) {
    if (q < kFuseSlots) return nullptr;
    *target = a.waves[q - kFuseSlots].nitems;
    return &a.j_done[q - kFuseSlots];
  }
  const FuseWave &wv = a.waves[q - kFuseLag];
  *target = wv.tiles[0] + wv.tiles[1];
  return &a.p2_done[q - kFuseLag];
}

// Thread 0: the unit's dependency already met (one read, no waiting)?
__device__ __forceinline__ int fuse_ready_now(const FuseArgs &a, uint32_t seg) {
  uint32_t target = 0;
  const uint32_t *ctr = fuse_dep(a, seg, &target);
  if (!ctr) return 1;
  if (*(volatile const uint32_t *)ctr < target) return 0;
  __threadfence();
  return 1;
}

template <typename KeyT>
__global__ void __launch_bounds__(kShuffleNT, 2)
    k_fused(FuseArgs a, Resv rs, JOut out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ JoinShared js;
  __shared__ uint32_t s_unit, s_seg, s_local;
  __shared__ int s_ready, s_ok;
  const uint32_t tid = threadIdx.x;
  const uint32_t nunits = a.seg_start[a.nseg];
  // the block's first unit; every later one is fetched while the previous
  // unit runs, and decoded and checked while the block finishes it
  if (tid == 0) {
    s_unit = atomicAdd(a.ticket, 1u);
    if (s_unit < nunits) {
      fuse_decode(a, s_unit, &s_seg, &s_local);
      s_ready = fuse_ready_now(a, s_seg);
    }
  }
  __syncthreads();
  for (;;) {
    const uint32_t u = s_unit;
    if (u >= nunits) break;
    const uint32_t seg = s_seg, local = s_local;
    const int ready = s_ready;
    uint32_t nx = 0;
    if (tid == 0) nx = atomicAdd(a.ticket, 1u);
    if (!ready) {  // s_ready was read by every thread above; the wait reports in s_ok
      if (tid == 0) {
        uint32_t target = 0;
        const uint32_t *ctr = fuse_dep(a, seg, &target);
        s_ok = fuse_wait(ctr, target, rs.flags);
      }
      __syncthreads();
      if (!s_ok) break;
    }
    const uint32_t q = seg / 2;
    uint32_t w;
    if (seg % 2 == 0) {
      // ---- a pass-2 tile of wave q
      w = q;
      const FuseWave wv = a.waves[w];
      const int side = local < wv.tiles[0] ? 0 : 1;
      const uint32_t k = side ? local - wv.tiles[0] : local;
      const uint32_t row0 = wv.row0[side] + k * kFuseTile;
      const uint32_t rend = min(row0 + kFuseTile, wv.row0[side] + wv.rows[side]);
      const ColMove &cm = a.moves[(w % kFuseSlots) * 2 + side];
      const int reg_col = a.pay_w[side] ? 1 : -1;
      KeyT kv[kRPL];
      uint64_t pv[kRPL];
      uint32_t rv[kRPL];
      KeyT kf, kl;
      const KeyT *keys = (const KeyT *)a.p1_key[side];
      shuffle_load<KeyT, true>(keys, row0, rend, cm, reg_col, a.pay_w[side], a.p1_rid[side], kv, pv, rv, kf, kl);
      shuffle_clear_counters<kShuffleNT>(smem);  // the shared memory held a join item before
      __syncthreads();
      shuffle_one_tile<kShuffleNT, KeyT, true, false>(smem, keys, row0, rend, w * a.F2, a.F2, a.sub,
                                                      a.cursors[side], wv.row0[side], cm, reg_col, a.pay_w[side],
                                                      a.p1_rid[side], (uint32_t *)cm.dst[2], kv, pv, rv, 0u, 0u, kf,
                                                      kl, 0);
    } else {
      // ---- a join item of wave q - lag
      w = q - kFuseLag;
      const FuseWave wv = a.waves[w];
      const uint32_t it = wv.item0 + local;
      Item d = a.desc[it];
      d.lbeg -= wv.row0[0];
      d.rbeg -= wv.row0[1];
      const JSide *jside = a.jsides + (w % kFuseSlots) * 2;
      join_item<KeyT, false, true>(smem, a.cap, jside[0], jside[1], d, it, rs, out, js);
    }
    uint32_t nseg = 0, nlocal = 0;
    int nready = 0;
    if (tid == 0 && nx < nunits) {
      fuse_decode(a, nx, &nseg, &nlocal);
      nready = fuse_ready_now(a, nseg);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(seg % 2 == 0 ? &a.p2_done[w] : &a.j_done[w], 1u);
      s_unit = nx;
      s_seg = nseg;
      s_local = nlocal;
      s_ready = nready;
    }
    __syncthreads();
  }
}

// Resident blocks of k_fused (grid), and its dynamic shared memory.
template <typename KeyT>
int fused_launch_shape(uint32_t cap, size_t *smem, int *grid) {
  const size_t a = shuffle_smem_bytes<kShuffleNT>(), b = WriteLayout<KeyT>(cap).total;
  *smem = a > b ? a : b;
  int per_sm = 0;
  MDJ_CUDA_TRY(cudaFuncSetAttribute(k_fused<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
  MDJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<KeyT>, kShuffleNT, *smem));
  if (per_sm < 1) return MDJ_ERR_INTERNAL;
  *grid = num_sms() * per_sm;
  return MDJ_OK;
}

// MDJ_FUSED=1 turns the fused pass-2 + join path on.  Measured on GB300 for
// the 100M x 100M merge it is slower than pass 2 + k_join_write (5.1-5.7 vs
// 3.3 ms): join units wait on pass-2 tiles still in flight, and the slot
// ring (4 x 16 MB) does not stay in L2 beside the streaming traffic.
bool fused_enabled() {
  const char *e = getenv("MDJ_FUSED");
  return e && e[0] == '1';
}

constexpr size_t kFuseSlotBudget = 1ull << 30;  // scratch bytes at most (else the unfused path)

// The fused pass 2 + join of a two-level plan from both sides' pass-1 copies.
// *fallback = true (and no result) when the scratch would exceed its budget
// or the output outgrew the optimistic buffer: the caller then runs pass 2
// and the join separately.
template <typename KeyT>
int run_fused(Workspace &ws, const Side1 &L1, const Side1 &R1, const Plan &plan, mdj_result *res, bool *fallback) {
  cudaStream_t s = ws.stream();
  *fallback = false;
  const Side &Ls = L1.p1, &Rs = R1.p1;
  const uint32_t nb = plan.nbuckets, F1 = plan.F1, F2 = plan.F2;
  const uint64_t cap_rows = output_capacity_hint(Ls.nrows, Rs.nrows);
  mdj_result r;
  JOut o;
  MDJ_TRY(alloc_result(ws, Ls, Rs, sizeof(KeyT), cap_rows, &r, &o));
  auto fail = [&](int rc) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    return rc;
  };
  // items per final sub-bucket, the waves and the unit order
  uint64_t *bucket_items = (uint64_t *)ws.get((size_t)(nb + 1) * 8);
  const uint32_t nseg = 2 * (F1 + kFuseLag);
  FuseWave *waves = (FuseWave *)ws.get((size_t)F1 * sizeof(FuseWave));
  uint32_t *seg = (uint32_t *)ws.get((size_t)(nseg + 1) * 4);
  uint32_t *pout = (uint32_t *)ws.get(16);
  if (!bucket_items || !waves || !seg || !pout) return fail(MDJ_ERR_OOM);
  {
    TraceScope tr("join_items", s);
    k_items<<<(nb + 1 + 255) / 256, 256, 0, s>>>(Ls.off, Rs.off, nb, plan.cap, kWriteChunk, bucket_items);
  }
  if (cudaGetLastError() != cudaSuccess) return fail(MDJ_ERR_CUDA);
  int rc = exclusive_scan_u64(ws, bucket_items, bucket_items, nb + 1);
  if (rc != MDJ_OK) return fail(rc);
  {
    TraceScope tr("fuse_plan", s);
    k_fuse_plan<<<1, 1024, 0, s>>>(Ls.off, Rs.off, bucket_items, F1, F2, waves, seg, pout);
  }
  uint64_t nitems = 0;
  uint32_t hp[4] = {0, 0, 0, 0};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nitems, bucket_items + nb, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp, pout, 12, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(cuda_status(e));
  if (nitems >= (1ull << 31)) return fail(MDJ_ERR_TOO_LARGE);

  FuseArgs a;
  memset(&a, 0, sizeof a);
  a.key_w = (int)sizeof(KeyT);
  const Side *sd[2] = {&Ls, &Rs};
  const uint32_t maxrows[2] = {hp[0], hp[1]};
  auto part = [](size_t bytes) { return (bytes + 255) & ~(size_t)255; };
  for (int i = 0; i < 2; i++) {
    a.pay_w[i] = sd[i]->ncols ? sd[i]->widths[0] : 0;
    a.side[i].key = 0;
    a.side[i].pay = part((size_t)maxrows[i] * sizeof(KeyT));
    a.side[i].rid = a.side[i].pay + part((size_t)maxrows[i] * (a.pay_w[i] ? a.pay_w[i] : 0));
    a.side[i].bytes = a.side[i].rid + part((size_t)maxrows[i] * 4);
    a.p1_key[i] = sd[i]->key;
    a.p1_pay[i] = sd[i]->ncols ? sd[i]->cols[0] : nullptr;
    a.p1_rid[i] = sd[i]->rid;
  }
  a.slot_bytes = a.side[0].bytes + a.side[1].bytes;
  if (a.slot_bytes * kFuseSlots > kFuseSlotBudget || nitems == 0) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    *fallback = true;
    return MDJ_OK;
  }
  Item *desc = (Item *)ws.get((size_t)nitems * sizeof(Item));
  a.slots = (unsigned char *)ws.get(a.slot_bytes * kFuseSlots);
  // p2_done[F1] | j_done[F1] | ticket | cursors L[nb] | cursors R[nb]
  const size_t cwords = 2 * (size_t)F1 + 1 + 2 * (size_t)nb;
  uint32_t *cw = (uint32_t *)ws.get(cwords * 4);
  // item_off[nitems] | total | flags
  unsigned long long *st = (unsigned long long *)ws.get(((size_t)nitems + 3) * 8);
  if (!desc || !a.slots || !cw || !st) return fail(MDJ_ERR_OOM);
  {
    TraceScope tr("join_expand", s);
    const uint64_t want = (nitems + 255) / 256, most = (uint64_t)num_sms() * 8;
    k_expand<<<(unsigned)(want < most ? want : most), 256, 0, s>>>(Ls.off, Rs.off, nb, plan.cap, kWriteChunk,
                                                                   bucket_items, (uint32_t)nitems, desc);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(cw, 0, (2 * (size_t)F1 + 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cw + 2 * F1 + 1, Ls.off, (size_t)nb * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cw + 2 * F1 + 1 + nb, Rs.off, (size_t)nb * 4, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, ((size_t)nitems + 3) * 8, s);
  if (e != cudaSuccess) return fail(cuda_status(e));
  // per (slot, side): the pass-2 column move (key, payload, and the row ids
  // as dst[2]) and the join side over the slot's scratch columns
  ColMove hm[kFuseSlots * 2];
  JSide hj[kFuseSlots * 2];
  memset(hm, 0, sizeof hm);
  memset(hj, 0, sizeof hj);
  for (uint32_t k = 0; k < kFuseSlots; k++)
    for (int i = 0; i < 2; i++) {
      unsigned char *base = a.slots + (size_t)k * a.slot_bytes + (i ? a.side[0].bytes : 0);
      ColMove &m = hm[k * 2 + i];
      m.n = a.pay_w[i] ? 2 : 1;
      m.key_index = 0;
      m.src[0] = a.p1_key[i];
      m.dst[0] = base + a.side[i].key;
      m.width[0] = (int)sizeof(KeyT);
      m.src[1] = a.p1_pay[i];
      m.dst[1] = base + a.side[i].pay;
      m.width[1] = a.pay_w[i];
      m.dst[2] = base + a.side[i].rid;
      JSide &j = hj[k * 2 + i];
      j.key = base + a.side[i].key;
      j.rid = (const uint32_t *)(base + a.side[i].rid);
      j.cols[0] = base + a.side[i].pay;
      j.width[0] = a.pay_w[i];
      j.ncols = a.pay_w[i] ? 1 : 0;
    }
  ColMove *dm = (ColMove *)ws.get(sizeof hm);
  JSide *dj = (JSide *)ws.get(sizeof hj);
  if (!dm || !dj) return fail(MDJ_ERR_OOM);
  e = cudaMemcpyAsync(dm, hm, sizeof hm, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dj, hj, sizeof hj, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(cuda_status(e));
  a.moves = dm;
  a.jsides = dj;
  a.waves = waves;
  a.seg_start = seg;
  a.nseg = nseg;
  a.F1 = F1;
  a.F2 = F2;
  a.desc = desc;
  a.p2_done = cw;
  a.j_done = cw + F1;
  a.ticket = cw + 2 * F1;
  a.cursors[0] = cw + 2 * F1 + 1;
  a.cursors[1] = cw + 2 * F1 + 1 + nb;
  a.sub = make_spec(plan.P, plan.S, 1);
  a.cap = plan.cap;
  unsigned long long *total = st + nitems;
  int *flags = (int *)(st + nitems + 1);
  const Resv rs = {nullptr, (uint64_t *)st, total, cap_rows, flags, 0, 0};
  size_t smem = 0;
  int grid = 0;
  rc = fused_launch_shape<KeyT>(plan.cap, &smem, &grid);
  if (rc != MDJ_OK) return fail(rc);
  {
    TraceScope tr("fused_p2_join", s);
    k_fused<KeyT><<<grid, kShuffleNT, smem, s>>>(a, rs, o);
  }
  unsigned long long host_total = 0;
  int host_flags[FLAG_WORDS] = {0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host_total, total, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_flags, flags, sizeof host_flags, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(cuda_status(e));
  if (host_flags[FLAG_TIMEOUT]) return fail(MDJ_ERR_DEVICE_TIMEOUT);
  if (host_total > cap_rows) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    *fallback = true;
    return MDJ_OK;
  }
  r.nrows = host_total;
  *res = r;
  return MDJ_OK;
}

// pair_off[i] = output offset of pair i's first item (or of the next pair's,
// for a pair without items); pair_off[npairs] = total rows.
__global__ void k_pair_offsets(const uint32_t *__restrict__ seg_base, uint32_t npairs, uint32_t nb,
                               const uint64_t *__restrict__ bucket_items, const uint64_t *__restrict__ item_out,
                               uint32_t nitems, uint64_t total, uint64_t *__restrict__ pair_off) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > npairs) return;
  const uint32_t b = i < npairs ? seg_base[i] : nb;
  const uint64_t idx = bucket_items[b];
  pair_off[i] = (i < npairs && idx < nitems) ? item_out[idx] : total;
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
  Plan plan = make_plan(left->nrows, P, cap_from_env(), P > 1);
  // ordered output is deterministic only over stable partition passes
  plan.stable = ordered_output() != 0;
  const bool k64 = left->cols[lk].dtype == MDJ_I64;
  if (!checksum_mode && fused_enabled() && merge_shuffle_unstable() && plan.partition && !plan.lsd &&
      !plan.stable && plan.F2 > 1 && left->ncols <= 2 && right->ncols <= 2) {
    // two-level plan: pass 2 and the join fused through L2-resident scratch
    Side1 L1, R1;
    MDJ_TRY(partition_side_pass1(ws, left, lk, plan, &L1));
    MDJ_TRY(partition_side_pass1(ws, right, rk, plan, &R1));
    bool fallback = false;
    MDJ_TRY(k64 ? run_fused<int64_t>(ws, L1, R1, plan, out, &fallback)
                : run_fused<int32_t>(ws, L1, R1, plan, out, &fallback));
    if (!fallback) return MDJ_OK;
    Side L, R;
    MDJ_TRY(partition_side_pass2(ws, left, lk, plan, L1, &L));
    MDJ_TRY(partition_side_pass2(ws, right, rk, plan, R1, &R));
    return k64 ? run_join<int64_t>(ws, L, R, plan, out) : run_join<int32_t>(ws, L, R, plan, out);
  }
  Side L, R;
  MDJ_TRY(partition_side(ws, left, lk, plan, &L));
  MDJ_TRY(partition_side(ws, right, rk, plan, &R));
  if (checksum_mode)
    return k64 ? run_count<int64_t>(ws, L, R, plan, count, checksum) : run_count<int32_t>(ws, L, R, plan, count, checksum);
  return k64 ? run_join<int64_t>(ws, L, R, plan, out) : run_join<int32_t>(ws, L, R, plan, out);
}


// A batch of independent merges (P given) or joins (P NULL, i.e. all 1): segment
// i = rows [lo[i], lo[i+1]) of `left` and [ro[i], ro[i+1]) of `right`, hash
// split into P_i partitions of S_i sub-buckets each; all buckets joined by one
// persistent kernel in ordered mode, so segment i's rows come out contiguous.
int batch_impl(const mdj_table *left, int32_t left_key, const uint64_t *left_offsets, const mdj_table *right,
               int32_t right_key, const uint64_t *right_offsets, int32_t npairs, const uint32_t *P,
               const mdj_tuning *tuning, const mdj_allocator *alloc, void *stream, mdj_result *out,
               uint64_t *pair_offsets) {
  MDJ_TRY(check_table(left, left_key));
  MDJ_TRY(check_table(right, right_key));
  if (left->cols[left_key].dtype != right->cols[right_key].dtype) return MDJ_ERR_INVALID_ARG;
  if (npairs < 1 || !left_offsets || !right_offsets || !out || !pair_offsets) return MDJ_ERR_INVALID_ARG;
  if (left_offsets[0] != 0 || right_offsets[0] != 0 || left_offsets[npairs] != left->nrows ||
      right_offsets[npairs] != right->nrows)
    return MDJ_ERR_INVALID_ARG;
  for (int32_t i = 0; i < npairs; i++) {
    if (left_offsets[i + 1] < left_offsets[i] || right_offsets[i + 1] < right_offsets[i]) return MDJ_ERR_INVALID_ARG;
    if (P && (P[i] < 1 || P[i] > kPass2SpanMax)) return MDJ_ERR_INVALID_ARG;
  }
  memset(out, 0, sizeof *out);
  uint32_t cap = cap_from_env();
  uint32_t fill = 85;
  if (tuning) {
    if (tuning->table_rows) {
      if (tuning->table_rows < 256 || tuning->table_rows > kMaxCap) return MDJ_ERR_INVALID_ARG;
      cap = tuning->table_rows;
    }
    if (tuning->fill_pct) {
      if (tuning->fill_pct < 10 || tuning->fill_pct > 100) return MDJ_ERR_INVALID_ARG;
      fill = tuning->fill_pct;
    }
  }
  const uint64_t target = std::max<uint64_t>(1, (uint64_t)cap * fill / 100);
  std::vector<uint32_t> seg_nb(npairs), seg_base(npairs), seg_P(npairs);
  uint64_t nb = 0;
  for (int32_t i = 0; i < npairs; i++) {
    const uint64_t nl = left_offsets[i + 1] - left_offsets[i], nr = right_offsets[i + 1] - right_offsets[i];
    const uint32_t Pi = P ? P[i] : 1u;
    // the shuffle of a merge always runs; a join of an empty side needs no buckets
    uint64_t S = (nl && nr) ? (nl + target * Pi - 1) / (target * Pi) : 1;
    S = std::min<uint64_t>(std::max<uint64_t>(S, 1), kPass2SpanMax / Pi);
    seg_P[i] = Pi;
    seg_nb[i] = (uint32_t)(Pi * S);
    seg_base[i] = (uint32_t)nb;
    nb += seg_nb[i];
  }
  if (nb >= (1ull << 31)) return MDJ_ERR_TOO_LARGE;
  Workspace ws(alloc, (cudaStream_t)stream);
  cudaStream_t s = (cudaStream_t)stream;
  Side L, R;
  MDJ_TRY(partition_side_segmented(ws, left, left_key, left_offsets, npairs, seg_base.data(), seg_nb.data(),
                                   seg_P.data(), (uint32_t)nb, &L));
  MDJ_TRY(partition_side_segmented(ws, right, right_key, right_offsets, npairs, seg_base.data(), seg_nb.data(),
                                   seg_P.data(), (uint32_t)nb, &R));
  Plan plan;
  plan.P = 1;
  plan.nbuckets = (uint32_t)nb;
  plan.cap = cap;
  ItemMap map;
  const bool k64 = left->cols[left_key].dtype == MDJ_I64;
  MDJ_TRY(k64 ? run_join<int64_t>(ws, L, R, plan, out, true, &map) : run_join<int32_t>(ws, L, R, plan, out, true, &map));
  // segment boundaries in the (segment-major) output
  uint32_t *dbase = (uint32_t *)ws.get((size_t)npairs * 4);
  uint64_t *doff = (uint64_t *)ws.get((size_t)(npairs + 1) * 8);
  int rc = MDJ_OK;
  if (!dbase || !doff) rc = MDJ_ERR_OOM;
  if (rc == MDJ_OK)
    rc = cuda_status(cudaMemcpyAsync(dbase, seg_base.data(), (size_t)npairs * 4, cudaMemcpyHostToDevice, s));
  if (rc == MDJ_OK) {
    {
      TraceScope tr("pair_offsets", s);
      k_pair_offsets<<<(npairs + 1 + 255) / 256, 256, 0, s>>>(dbase, (uint32_t)npairs, (uint32_t)nb,
                                                              map.bucket_items, map.item_out, map.nitems, out->nrows,
                                                              doff);
    }
    rc = cuda_status(cudaGetLastError());
  }
  if (rc == MDJ_OK)
    rc = cuda_status(cudaMemcpyAsync(pair_offsets, doff, (size_t)(npairs + 1) * 8, cudaMemcpyDeviceToHost, s));
  if (rc == MDJ_OK) rc = cuda_status(cudaStreamSynchronize(s));
  if (rc != MDJ_OK) mdj_result_release(out, alloc, stream);
  return rc;
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

int mdj_join_batch(const mdj_table *left, int32_t left_key, const uint64_t *left_offsets, const mdj_table *right,
                   int32_t right_key, const uint64_t *right_offsets, int32_t npairs, const mdj_tuning *tuning,
                   const mdj_allocator *alloc, void *stream, mdj_result *out, uint64_t *pair_offsets) {
  return batch_impl(left, left_key, left_offsets, right, right_key, right_offsets, npairs, nullptr, tuning, alloc,
                    stream, out, pair_offsets);
}

int mdj_merge_batch(const mdj_table *left, int32_t left_key, const uint64_t *left_offsets, const mdj_table *right,
                    int32_t right_key, const uint64_t *right_offsets, int32_t nreq, const uint32_t *P,
                    const mdj_tuning *tuning, const mdj_allocator *alloc, void *stream, mdj_result *out,
                    uint64_t *req_offsets) {
  if (!P) return MDJ_ERR_INVALID_ARG;
  return batch_impl(left, left_key, left_offsets, right, right_key, right_offsets, nreq, P, tuning, alloc, stream,
                    out, req_offsets);
}

}  // extern "C"
