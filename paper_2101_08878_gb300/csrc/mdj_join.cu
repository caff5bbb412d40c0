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
// The pair count and checksum of a join (mdj_count_checksum) come from the
// streamed output's grouping instead (mdj_stream.cu), which handles key groups
// of any size without re-reading probe rows.
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "mdj_internal.cuh"
#include "mdj_join_dev.cuh"
#include "mdj_shuffle_dev.cuh"

namespace mdj {
namespace {


// ------------------------------------------------------------- work items

// Items of bucket b: ceil(nl / cap) build chunks x ceil(nr / rch) probe chunks
// (0 when either side is empty).
// The thread past the last bucket also clears the join's counters `tail`
// (total, ticket, flags, item count: five words).
__global__ void k_items(const uint32_t *__restrict__ offL, const uint32_t *__restrict__ offR, uint32_t nb, uint32_t cap,
                        uint32_t rch, uint64_t *__restrict__ items, unsigned long long *__restrict__ tail) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) {
    uint64_t nl = offL[b + 1] - offL[b], nr = offR[b + 1] - offR[b];
    items[b] = (nl && nr) ? ((nl + cap - 1) / cap) * ((nr + rch - 1) / rch) : 0ull;
  } else if (b == nb) {
    items[nb] = 0;
    for (int w = 0; w < 5; w++) tail[w] = 0;
  }
}

// One descriptor per item: its build and probe row ranges.  The item count
// is item_off[nb]; more than `ulim` items (the descriptor array's size) sets
// FLAG_ITEMS and writes nothing.
__global__ void k_expand(const uint32_t *__restrict__ offL, const uint32_t *__restrict__ offR, uint32_t nb,
                         uint32_t cap, uint32_t rch, const uint64_t *__restrict__ item_off, uint32_t ulim,
                         Item *__restrict__ desc, int *flags) {
  const uint64_t total = item_off[nb];
  if (total > ulim) {
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[FLAG_ITEMS] = 1;
    return;
  }
  const uint32_t nitems = (uint32_t)total;
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

// bulk: the build side's staged columns (key, row ids, first payload) have
// 16-byte-aligned bases, so items stage them by bulk copies.  The item count
// is read from *nitems_dev (no work when it exceeds `ulim`: k_expand has set
// FLAG_ITEMS and the host reruns the join with exact arrays).
template <typename KeyT, bool HAVE_OFFSETS, int NT, bool COUNT = false>
__global__ void __launch_bounds__(NT, 1024 / NT)
    k_join_write(JSide L, JSide R, const Item *__restrict__ desc, const uint64_t *nitems_dev, uint32_t ulim,
                 uint32_t cap, uint32_t *ticket, unsigned long long *state, uint64_t *__restrict__ item_off,
                 unsigned long long *total, uint64_t capacity, int *flags, int withhold_first, int ordered, int bulk,
                 JOut out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Item s_item;
  __shared__ uint32_t s_it;
  __shared__ __align__(8) JoinShared js;
  const uint32_t tid = threadIdx.x;
  const uint64_t nit = *nitems_dev;
  const uint32_t nitems = nit > ulim ? 0u : (uint32_t)nit;
  if (blockIdx.x == 0 && threadIdx.x == 0) total[4] = nit;  // read back with the total and the flags
  const Resv rs = {state, item_off, total, capacity, flags, withhold_first, ordered};
  uint32_t phase = 0;
  if (tid == 0) {
    if (bulk) mbar_init(&js.bar, 1);
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
    if (!join_item<KeyT, HAVE_OFFSETS, NT, COUNT>(smem, cap, L, R, d, it, rs, out, js, bulk != 0, phase)) break;
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

// The build side's staged columns all start on 16-byte boundaries (bulk copies).
int bulk_ok(const Side &s) {
  auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
  return al(s.key) && (!s.rid || al(s.rid)) && (s.ncols == 0 || al(s.cols[0])) ? 1 : 0;
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

// Work items of the whole join, with `rch` probe rows per item at most, into
// a descriptor array of `ulim` items.  No host wait: the count stays on the
// device at (*item_off)[nb] (per-bucket item prefix in *item_off), and a count
// above ulim sets FLAG_ITEMS instead of writing descriptors.
int make_items(Workspace &ws, const Side &Ls, const Side &Rs, uint32_t nb, uint32_t cap, uint32_t rch, uint32_t ulim,
               unsigned long long *tail, Item **desc, uint64_t **item_off_out) {
  int *flags = (int *)(tail + 2);
  cudaStream_t s = ws.stream();
  uint64_t *item_off = (uint64_t *)ws.get((size_t)(nb + 1) * 8);
  *desc = (Item *)ws.get((size_t)(ulim ? ulim : 1) * sizeof(Item));
  if (!item_off || !*desc) return MDJ_ERR_OOM;
  {
    TraceScope tr("join_items", s);
    k_items<<<(nb + 1 + 255) / 256, 256, 0, s>>>(Ls.off, Rs.off, nb, cap, rch, item_off, tail);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u64(ws, item_off, item_off, nb + 1));
  {
    TraceScope tr("join_expand", s);
    const uint64_t want = ((uint64_t)ulim + 255) / 256, most = (uint64_t)num_sms() * 8;
    const unsigned g = (unsigned)std::max<uint64_t>(1, want < most ? want : most);
    k_expand<<<g, 256, 0, s>>>(Ls.off, Rs.off, nb, cap, rch, item_off, ulim, *desc, flags);
  }
  MDJ_LAUNCH_CHECK();
  *item_off_out = item_off;
  return MDJ_OK;
}

// Descriptor slots for a join without reading its item count: every bucket
// one item, plus room for buckets that split into several (a count above it
// costs one rerun with exact arrays).  MDJ_TEST_ITEM_BOUND (test hook) sets it.
uint32_t item_bound(uint32_t nb, uint64_t nl, uint64_t nr, uint32_t cap, uint32_t rch) {
  const char *e = getenv("MDJ_TEST_ITEM_BOUND");
  if (e) {
    const long long v = atoll(e);
    if (v >= 1) return (uint32_t)std::min<long long>(v, (1ll << 31) - 1);
  }
  const uint64_t u = (uint64_t)nb + 2 * ((nl + cap - 1) / cap + (nr + rch - 1) / rch) + 1024;
  return (uint32_t)std::min<uint64_t>(u, (1ull << 31) - 1);
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

// The join's counters in one read: output total, flags, item count.
int read_tail(const unsigned long long *tail, cudaStream_t s, unsigned long long *total, int *flags,
              uint64_t *items) {
  unsigned long long t[5];
  MDJ_CUDA_TRY(cudaMemcpyAsync(t, tail, sizeof t, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  *total = t[0];
  memcpy(flags, &t[2], FLAG_WORDS * sizeof(int));
  *items = t[4];
  return MDJ_OK;
}

template <typename KeyT, int NT>
int run_join_t(Workspace &ws, const Side &Ls, const Side &Rs, const Plan &plan, mdj_result *res,
               bool force_ordered = false, ItemMap *map = nullptr, uint32_t exact_items = 0) {
  cudaStream_t s = ws.stream();
  const uint32_t rch = (uint32_t)kWPF * NT;
  const uint32_t ulim = exact_items ? exact_items : item_bound(plan.nbuckets, Ls.nrows, Rs.nrows, plan.cap, rch);
  const int ordered = force_ordered || ordered_output() ? 1 : 0;
  // the optimistic output buffer (none for two-pass output); nothing below
  // waits for the device until the join has run
  const uint64_t cap_rows = force_ordered ? 0 : output_capacity_hint(Ls.nrows, Rs.nrows);
  mdj_result r;
  JOut o;
  MDJ_TRY(alloc_result(ws, Ls, Rs, sizeof(KeyT), cap_rows, &r, &o));
  // state[ulim] | item_off[ulim] | total | ticket | flags (2 words) | item count
  const size_t words = 2 * (size_t)ulim + 5;
  unsigned long long *state = (unsigned long long *)ws.get(words * 8);
  int rc = state ? MDJ_OK : MDJ_ERR_OOM;
  uint64_t *item_off = state ? (uint64_t *)(state + ulim) : nullptr;
  unsigned long long *total = state ? state + 2 * (size_t)ulim : nullptr;
  uint32_t *ticket = (uint32_t *)(total + 1);
  int *flags = (int *)(total + 2);
  // the look-back slots start empty (ordered); k_items clears the counters
  if (rc == MDJ_OK && ordered) rc = cuda_status(cudaMemsetAsync(state, 0, (size_t)ulim * 8, s));
  Item *desc = nullptr;
  uint64_t *bucket_items = nullptr;
  if (rc == MDJ_OK) rc = make_items(ws, Ls, Rs, plan.nbuckets, plan.cap, rch, ulim, total, &desc, &bucket_items);
  if (rc != MDJ_OK) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    return rc;
  }
  const uint64_t *nitems_dev = bucket_items + plan.nbuckets;

  const size_t sm = WriteLayout<KeyT>(plan.cap).total;  // ~105 KB at cap 4096: two blocks per SM
  if (force_ordered) {
    // two-pass ordered output (the batched joins): a count pass records every
    // item's rows, a scan places the items in item order (item_off[ulim] is
    // `total`, which receives the sum), and the exact pass writes each item
    // at its offset; no item waits on another
    int grid;
    unsigned long long host_total = 0;
    uint64_t host_items = 0;
    int host_flags[FLAG_WORDS] = {0, 0, 0, 0};
    rc = cuda_status(cudaMemsetAsync(item_off, 0, ((size_t)ulim + 1) * 8, s));
    if (rc == MDJ_OK) rc = resident_grid(k_join_write<KeyT, false, NT, true>, sm, ulim, &grid, NT);
    if (rc == MDJ_OK) {
      TraceScope tr("join_count", s);
      k_join_write<KeyT, false, NT, true><<<grid, NT, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems_dev, ulim,
                                                            plan.cap, ticket, state, item_off, total, 0, flags, 0,
                                                            0, bulk_ok(Ls), o);
      rc = cuda_status(cudaGetLastError());
    }
    if (rc == MDJ_OK) rc = exclusive_scan_u64(ws, item_off, item_off, (size_t)ulim + 1);
    if (rc == MDJ_OK) rc = read_tail(total, s, &host_total, host_flags, &host_items);
    if (rc == MDJ_OK && host_flags[FLAG_TIMEOUT]) rc = MDJ_ERR_DEVICE_TIMEOUT;
    mdj_result_release(&r, ws.allocator(), (void *)s);
    if (rc != MDJ_OK) return rc;
    if (host_flags[FLAG_ITEMS]) {
      if (host_items >= (1ull << 31)) return MDJ_ERR_TOO_LARGE;
      ws.give_back(desc);
      ws.give_back(bucket_items);
      ws.give_back(state);
      return run_join_t<KeyT, NT>(ws, Ls, Rs, plan, res, force_ordered, map, (uint32_t)host_items);
    }
    const uint64_t m = host_total;
    MDJ_TRY(alloc_result(ws, Ls, Rs, sizeof(KeyT), m, &r, &o));
    if (m > 0) {
      rc = resident_grid(k_join_write<KeyT, true, NT>, sm, ulim, &grid, NT);
      if (rc == MDJ_OK) rc = cuda_status(cudaMemsetAsync(ticket, 0, 4, s));
      if (rc == MDJ_OK) {
        TraceScope tr("join_write_exact", s);
        k_join_write<KeyT, true, NT><<<grid, NT, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems_dev, ulim,
                                                       plan.cap, ticket, state, item_off, total, m, flags, 0, 0,
                                                       bulk_ok(Ls), o);
        rc = cuda_status(cudaGetLastError());
      }
      if (rc != MDJ_OK) {
        mdj_result_release(&r, ws.allocator(), (void *)s);
        return rc;
      }
    }
    r.nrows = m;
    *res = r;
    if (map) {
      map->bucket_items = bucket_items;
      map->item_out = item_off;
      map->nitems = (uint32_t)host_items;
    }
    return MDJ_OK;
  }
  int grid;
  rc = resident_grid(k_join_write<KeyT, false, NT>, sm, ulim, &grid, NT);
  if (rc == MDJ_OK) {
    TraceScope tr("join_write", s);
    k_join_write<KeyT, false, NT><<<grid, NT, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems_dev, ulim, plan.cap,
                                                    ticket, state, item_off, total, cap_rows, flags,
                                                    test_withhold_first(), ordered, bulk_ok(Ls), o);
    rc = cuda_status(cudaGetLastError());
  }
  unsigned long long host_total = 0;
  uint64_t host_items = 0;
  int host_flags[FLAG_WORDS] = {0, 0, 0, 0};
  if (rc == MDJ_OK) rc = read_tail(total, s, &host_total, host_flags, &host_items);
  if (rc == MDJ_OK && host_flags[FLAG_TIMEOUT]) rc = MDJ_ERR_DEVICE_TIMEOUT;
  if (rc == MDJ_OK && host_flags[FLAG_ITEMS]) {
    // more items than the bound: again, with arrays of the exact count
    mdj_result_release(&r, ws.allocator(), (void *)s);
    if (host_items >= (1ull << 31)) return MDJ_ERR_TOO_LARGE;
    ws.give_back(desc);
    ws.give_back(bucket_items);
    ws.give_back(state);
    return run_join_t<KeyT, NT>(ws, Ls, Rs, plan, res, force_ordered, map, (uint32_t)host_items);
  }
  if (rc != MDJ_OK) {
    mdj_result_release(&r, ws.allocator(), (void *)s);
    return rc;
  }
  const uint32_t nitems = (uint32_t)host_items;
  const uint64_t m = host_total;
  if (m > cap_rows || m == 0) {
    // the join outgrew the optimistic buffer (or is empty): exact buffers,
    // then one write pass at the offsets the first pass recorded
    mdj_result_release(&r, ws.allocator(), (void *)s);
    MDJ_TRY(alloc_result(ws, Ls, Rs, sizeof(KeyT), m, &r, &o));
    if (m > 0) {
      MDJ_TRY(resident_grid(k_join_write<KeyT, true, NT>, sm, nitems, &grid, NT));
      MDJ_CUDA_TRY(cudaMemsetAsync(ticket, 0, 4, s));
      {
        TraceScope tr("join_write_exact", s);
        k_join_write<KeyT, true, NT><<<grid, NT, sm, s>>>(to_jside(Ls), to_jside(Rs), desc, nitems_dev, ulim,
                                                       plan.cap, ticket, state, item_off, total, m, flags, 0, 0,
                                                       bulk_ok(Ls), o);
      }
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        mdj_result_release(&r, ws.allocator(), (void *)s);
        return cuda_status(e);
      }
    }
  }
  r.nrows = m;
  *res = r;
  if (map) {
    map->bucket_items = bucket_items;
    map->item_out = item_off;
    map->nitems = nitems;
  }
  return MDJ_OK;
}

template <typename KeyT>
int run_join(Workspace &ws, const Side &Ls, const Side &Rs, const Plan &plan, mdj_result *res,
             bool force_ordered = false, ItemMap *map = nullptr) {
  if (plan.join_threads == 256) return run_join_t<KeyT, 256>(ws, Ls, Rs, plan, res, force_ordered, map);
  return run_join_t<KeyT, kWT>(ws, Ls, Rs, plan, res, force_ordered, map);
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

}  // namespace

// The merge's steps; `after_left` (if set) runs once the left side's
// partition is queued and before the right side's is, so that a caller can
// bring the right side's columns in meanwhile.
int merge_steps(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P,
                const mdj_allocator *alloc, void *stream, mdj_result *out, int (*after_left)(void *), void *ctx) {
  MDJ_TRY(check_table(left, lk));
  MDJ_TRY(check_table(right, rk));
  if (P < 1 || P > MDJ_MAX_PARTITIONS) return MDJ_ERR_INVALID_ARG;
  if (left->cols[lk].dtype != right->cols[rk].dtype) return MDJ_ERR_INVALID_ARG;
  if (!out) return MDJ_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  Workspace ws(alloc, (cudaStream_t)stream);
  Plan plan = make_plan(left->nrows, P, cap_from_env(), P > 1);
  // ordered output is deterministic only over stable partition passes
  plan.stable = ordered_output() != 0;
  const bool k64 = left->cols[lk].dtype == MDJ_I64;
  Side L, R;
  MDJ_TRY(partition_side(ws, left, lk, plan, &L));
  if (after_left) MDJ_TRY(after_left(ctx));
  MDJ_TRY(partition_side(ws, right, rk, plan, &R));
  return k64 ? run_join<int64_t>(ws, L, R, plan, out) : run_join<int32_t>(ws, L, R, plan, out);
}

namespace {

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

  if (checksum_mode) return grouped_count_checksum(left, lk, right, rk, P, alloc, stream, count, checksum);
  return merge_steps(left, lk, right, rk, P, alloc, stream, out, nullptr, nullptr);
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
  uint32_t join_threads = kWT;
  if (tuning) {
    if (tuning->join_threads) {
      if (tuning->join_threads != 256 && tuning->join_threads != 512) return MDJ_ERR_INVALID_ARG;
      join_threads = tuning->join_threads;
    }
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
  plan.join_threads = join_threads;
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
