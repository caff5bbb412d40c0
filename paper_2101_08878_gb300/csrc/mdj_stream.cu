// Streamed output of the merge: the join of mdj_merge written in windows of
// any size, for results too large to hold at once (the many-to-many merge of
// Sec. V-B with skewed keys: Zipf(1.1) over 5e7 x 2e8 rows has ~2e14 pairs).
//
// mdj_stream_open runs the merge up to its output.  Both tables are shuffled
// into P partitions of sub-buckets exactly as mdj_merge does (the exchange of
// Sec. IV-B done on one device).  In every sub-bucket the build rows are then
// regrouped so that equal keys are contiguous ("grouped order"), and every
// probe row learns its key's group: first grouped position and size.  That
// fixes an order on the join's rows: matching probe rows in shuffled order,
// each followed through its group.  A prefix sum over the matching probe
// rows' group sizes gives each one's first output row.
//
// mdj_stream_emit writes rows [q0, q0 + n) of that order: a row finds its
// probe row by search over those prefix sums and its build row by offset into
// the group, so a window can start anywhere, can be written again, and
// nothing of the join is recomputed.  A tile of rows that lies inside one
// group (a heavy key) is a plain streaming copy of the group's build rows.
//
// Skew on either side: a group may have any size; a sub-bucket whose build
// side exceeds one shared-memory table is grouped with a hash table in global
// memory (one region per such sub-bucket, two slots per build row); probe
// sides of any size are split into chunks over many blocks (a light
// sub-bucket's table is saved once and reloaded by its other chunks, so every
// chunk sees the same table).
//
// Merge variants: a right or outer join makes every probe row an entry (an
// unmatched one a single row with no left side); a left or outer join also
// records each group's size and whether any probe row found it, and appends
// one entry per group nobody found (no right side).  A missing side is row id
// kNone (0xFFFFFFFF) with zero bits in its columns.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mdj_internal.cuh"

namespace mdj {

// Device view of one shuffled side.
struct GSide {
  const void *key;
  const uint32_t *rid;  // NULL: identity
  const uint32_t *off;  // sub-bucket offsets [nbuckets + 1]
  const void *cols[MDJ_MAX_COLS];
  int32_t width[MDJ_MAX_COLS];
  int32_t ncols;
};

// What the emit kernel reads: matching probe rows (entries) with their first
// output row, probe row and group start; the probe side; the grouped build side.
struct EmitSrc {
  const uint64_t *moff;  // [nm + 1], moff[nm] = total rows
  const uint32_t *mr;    // [nm] shuffled probe row
  const uint32_t *mg;    // [nm] first grouped build position of its group
  uint32_t nm;
  const void *rkey;
  const uint32_t *rrid;  // NULL: identity
  const void *rcols[MDJ_MAX_COLS];
  int32_t rwidth[MDJ_MAX_COLS];
  int32_t nrc;
  const uint32_t *grid;  // grouped build rows' input row ids
  const void *gkey;      // grouped build keys (joins that keep unmatched left rows), else NULL
  const void *gcols[MDJ_MAX_COLS];
  int32_t lwidth[MDJ_MAX_COLS];
  int32_t nlc;
};

struct EmitDst {
  void *key;
  uint32_t *lrow;
  uint32_t *rrow;
  void *lcols[MDJ_MAX_COLS];
  void *rcols[MDJ_MAX_COLS];
};

}  // namespace mdj

// The handle: everything a later window needs, on the open stream.
struct mdj_stream {
  mdj_allocator alloc;
  bool has_alloc;
  cudaStream_t stream;
  mdj::Workspace *ws;  // owns every device buffer of the handle
  int32_t key_dtype;
  uint64_t total;
  uint64_t cursor;
  mdj::EmitSrc src;
};

namespace mdj {
namespace {

constexpr int kGT = 512;                   // threads of a grouping block
constexpr uint32_t kGCap = 4096;           // build rows of a shared-memory group table
constexpr int kGRows = kGCap / kGT;        // build rows per thread
constexpr uint32_t kGTab = 2 * kGCap;      // slots of the largest shared-memory table
static_assert(kGTab * 4 >= kGCap * 8, "the slot table stages a sub-bucket's 8-byte keys");
constexpr uint32_t kProbeChunk = 65536;    // probe rows per grouping unit
constexpr int kHT = 256;                   // threads of a global-table block
constexpr uint32_t kHChunk = 8192;         // rows per global-table unit
constexpr int kET = 256;                   // threads of the emit block
constexpr uint32_t kETile = 2048;          // output rows per emit tile
constexpr int kERows = kETile / kET;
constexpr int kEBatch = 4;                 // loads in flight per thread and column

struct LightUnit {
  uint32_t b, r0, nr;
  int32_t dump;  // >= 0: the table is saved in (or, for later chunks, loaded from) dump slot `dump`
};
// A sub-bucket grouped in global memory: build rows [lb, lb + nl), slots
// [ts0, ts0 + tsz) (tsz = 2 nl) of the slot arrays, rows [hr0, hr0 + nl) of
// the per-row arrays; hr0 = build rows of the earlier such sub-buckets.
struct HeavyDesc {
  uint32_t b, lb, nl, tsz, ts0, hr0;
};
struct HeavyUnit {
  uint32_t h, i0, n;  // build units: local rows [i0, i0 + n); probe units: probe rows [i0, i0 + n)
};

constexpr uint32_t kNone = 0xFFFFFFFFu;  // no row on this side (outer joins)

struct GOut {
  uint32_t *grid;                  // grouped build side: input row ids
  void *gcols[MDJ_MAX_COLS];       // grouped build side: non-key columns
  uint32_t *cnt;                   // per probe row: group size (0 = no match)
  uint32_t *gbase;                 // per probe row: first grouped position of its group
  // joins that keep unmatched left rows (else NULL):
  void *gkey;                      // grouped build side: keys
  uint32_t *gsize;                 // group size at each group's first grouped position, 0 elsewhere
  uint32_t *hit;                   // 1 at the first grouped position of every group a probe row found
};

// In-table position and tag of a key: multiplicative hash of the key bits
// (the multiplier is SplitMix64's second constant); top logt bits pick the
// slot, bits 16..31 the tag.
__device__ __forceinline__ uint64_t table_hash(uint64_t kb) { return (kb ^ (kb >> 29)) * 0xBF58476D1CE4E5B9ULL; }

__device__ __forceinline__ void small_slot_tag(uint64_t kb, uint32_t logt, uint32_t &slot, uint32_t &tag) {
  const uint64_t g = table_hash(kb);
  slot = (uint32_t)(g >> (64 - logt));
  tag = (uint32_t)(g >> 16) & 0xFFFFu;
}

__device__ __forceinline__ uint32_t big_home(uint64_t kb, uint32_t tsz) {
  return __umulhi((uint32_t)(table_hash(kb) >> 32), tsz);
}

__host__ __device__ __forceinline__ uint32_t small_logt(uint32_t nl) {
  uint32_t logt = 5;
  while ((1u << logt) < 2 * nl) logt++;
  return logt;
}

// Shared-memory layout of a group table (and of its saved copy): keys[kGCap],
// slots[kGTab], base[kGCap + 1], then the block-scan scratch (33 words).
template <typename KeyT>
__host__ __device__ constexpr size_t group_slots_at() {
  return (size_t)kGCap * sizeof(KeyT);
}
constexpr size_t kGBaseWords = kGCap + 1;
template <typename KeyT>
__host__ __device__ constexpr size_t group_smem_bytes() {
  return group_slots_at<KeyT>() + (size_t)kGTab * 4 + kGBaseWords * 4 + 33 * 4;
}

template <typename KeyT>
__host__ __device__ constexpr size_t dump_stride() {
  return (group_smem_bytes<KeyT>() + 255) & ~(size_t)255;
}

__device__ __forceinline__ void copy_col(void *dst, uint64_t di, const void *src, uint64_t si, int width) {
  if (width == 8)
    ((uint64_t *)dst)[di] = ((const uint64_t *)src)[si];
  else
    ((uint32_t *)dst)[di] = ((const uint32_t *)src)[si];
}

// Probe rows [r0, r0 + nr) against a shared-memory group table: keys, slot
// words tag << 16 | representative + 1 (the build row that claimed the slot),
// and base = exclusive prefix over build rows of the group sizes, each size
// counted at its representative, so a group starts at base[rep] and has
// base[rep + 1] - base[rep] rows.  Four rows per thread are loaded before any
// is probed.
template <typename KeyT>
__device__ __forceinline__ void load_probe_batch(const KeyT *__restrict__ Rk, uint32_t r0, uint32_t nr, uint32_t i0,
                                                 KeyT (&kv)[4]) {
#pragma unroll
  for (int u = 0; u < 4; u++) {
    const uint32_t i = i0 + u * kGT + threadIdx.x;
    kv[u] = i < nr ? Rk[r0 + i] : KeyT(0);
  }
}

template <typename KeyT>
__device__ __forceinline__ void probe_small(const KeyT *keys, const uint32_t *slots, const uint32_t *base, uint32_t logt,
                                            uint32_t lb, const KeyT *__restrict__ Rk, uint32_t r0, uint32_t nr,
                                            const GOut &o) {
  const uint32_t mask = (1u << logt) - 1;
  for (uint32_t i0 = 0; i0 < nr; i0 += 4 * kGT) {
    KeyT kv[4];
    load_probe_batch(Rk, r0, nr, i0, kv);
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t i = i0 + u * kGT + threadIdx.x;
      if (i >= nr) continue;
      uint32_t s, tag;
      small_slot_tag(key_bits(kv[u]), logt, s, tag);
      uint32_t rep = 0xFFFFFFFFu;
      for (uint32_t p = 0; p <= mask; p++) {
        const uint32_t w = slots[s];
        if (w == 0) break;
        if ((w >> 16) == tag && keys[(w & 0xFFFFu) - 1] == kv[u]) {
          rep = (w & 0xFFFFu) - 1;
          break;
        }
        s = (s + 1) & mask;
      }
      const bool found = rep != 0xFFFFFFFFu;
      o.cnt[r0 + i] = found ? base[rep + 1] - base[rep] : 0u;
      o.gbase[r0 + i] = found ? lb + base[rep] : 0u;
      if (found && o.hit) o.hit[lb + base[rep]] = 1;
    }
  }
}

// One column of the build rows lb + threadIdx.x + k * kGT (k < kGRows, below
// lb + nl) to grouped order: values to their local positions pos[k] in the
// shared staging area (four loads in flight at a time), then out to
// dst[lb ..) with coalesced stores.  src NULL: the identity (row index).
// Ends with a barrier.
template <typename V>
__device__ __forceinline__ void stage_column(V *__restrict__ dst, const V *__restrict__ src, uint32_t lb, uint32_t nl,
                                             const uint32_t (&pos)[kGRows], unsigned char *stage_bytes) {
  V *stage = (V *)stage_bytes;
#pragma unroll
  for (int h = 0; h < kGRows; h += 4) {  // four loads in flight per thread
    V v[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t i = threadIdx.x + (h + k) * kGT;
      if (i < nl) v[k] = src ? src[lb + i] : (V)(lb + i);
    }
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (threadIdx.x + (h + k) * kGT < nl) stage[pos[h + k]] = v[k];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nl; i += kGT) dst[lb + i] = stage[i];
  __syncthreads();
}

// ------------------------------------------------------- light sub-buckets
//
// One unit per light sub-bucket (build side <= kGCap rows): build keys to
// shared memory; one slot per distinct key (linear probing, compare-and-swap
// on an empty slot; the row whose swap claimed the slot represents the group);
// a build row's rank in its group from an atomicAdd on the count kept at its
// representative; block scan of those counts over the build rows = group
// starts; the first probe chunk is probed; each build row's input row id and
// columns go to lb + start + rank.  Units of an empty build side only write
// zero counts.
template <typename KeyT>
__global__ void __launch_bounds__(kGT, 2)
    k_group_light(const __grid_constant__ GSide L, const __grid_constant__ GSide R,
                  const LightUnit *__restrict__ units, uint32_t nunits, uint32_t *ticket,
                  const __grid_constant__ GOut o, unsigned char *__restrict__ dumps) {
  extern __shared__ __align__(16) unsigned char smem[];
  KeyT *keys = (KeyT *)smem;
  uint32_t *slots = (uint32_t *)(smem + group_slots_at<KeyT>());
  uint32_t *base = slots + kGTab;
  uint32_t *scratch = base + kGBaseWords;
  __shared__ uint32_t s_u;
  const KeyT *Lk = (const KeyT *)L.key;
  const KeyT *Rk = (const KeyT *)R.key;
  for (;;) {
    if (threadIdx.x == 0) s_u = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t u = s_u;
    __syncthreads();
    if (u >= nunits) return;
    const LightUnit U = units[u];
    const uint32_t lb = L.off[U.b], nl = L.off[U.b + 1] - lb;
    if (nl == 0) {
      for (uint32_t r = U.r0 + threadIdx.x; r < U.r0 + U.nr; r += kGT) {
        o.cnt[r] = 0;
        o.gbase[r] = 0;
      }
      continue;
    }
    const uint32_t logt = small_logt(nl), T = 1u << logt, mask = T - 1;
    // every load of the build keys is issued before the first store
    KeyT kr[kGRows];
#pragma unroll
    for (int k = 0; k < kGRows; k++) {
      const uint32_t i = threadIdx.x + k * kGT;
      kr[k] = i < nl ? Lk[lb + i] : KeyT(0);
    }
    for (uint32_t s = threadIdx.x; s < T; s += kGT) slots[s] = 0;
    for (uint32_t i = threadIdx.x; i <= nl; i += kGT) base[i] = 0;
#pragma unroll
    for (int k = 0; k < kGRows; k++) {
      const uint32_t i = threadIdx.x + k * kGT;
      if (i < nl) keys[i] = kr[k];
    }
    __syncthreads();
    // per build row: representative << 16 | rank in its group (both < kGCap),
    // later its grouped position
    uint32_t pr[kGRows];
#pragma unroll
    for (int k = 0; k < kGRows; k++) {
      const uint32_t i = threadIdx.x + k * kGT;
      pr[k] = 0;
      if (i < nl) {
        const KeyT kk = keys[i];
        uint32_t s, tag;
        small_slot_tag(key_bits(kk), logt, s, tag);
        const uint32_t w = (tag << 16) | (i + 1);
        uint32_t rep = i;
        for (uint32_t p = 0; p <= mask; p++) {  // ends: 2 slots per row, so a free slot exists
          uint32_t cur = slots[s];
          if (cur == 0) {
            const uint32_t prev = atomicCAS(&slots[s], 0u, w);
            if (prev == 0) break;
            cur = prev;
          }
          if ((cur >> 16) == tag && keys[(cur & 0xFFFFu) - 1] == kk) {
            rep = (cur & 0xFFFFu) - 1;
            break;
          }
          s = (s + 1) & mask;
        }
        pr[k] = (rep << 16) | atomicAdd(&base[rep], 1u);
      }
    }
    __syncthreads();
    block_scan_array(base, nl + 1, scratch);
    if (U.dump >= 0) {  // later probe chunks of this sub-bucket reload this exact table
      unsigned char *d = dumps + (size_t)U.dump * dump_stride<KeyT>();
      KeyT *dk = (KeyT *)d;
      uint32_t *ds = (uint32_t *)(d + group_slots_at<KeyT>());
      uint32_t *db = ds + kGTab;
      for (uint32_t i = threadIdx.x; i < nl; i += kGT) dk[i] = keys[i];
      for (uint32_t s = threadIdx.x; s < T; s += kGT) ds[s] = slots[s];
      for (uint32_t i = threadIdx.x; i <= nl; i += kGT) db[i] = base[i];
    }
    probe_small<KeyT>(keys, slots, base, logt, lb, Rk, U.r0, U.nr, o);
    // grouped order: each build row's position in the group order of the
    // sub-bucket; keys and slots are dead after the probe, so their space
    // stages one column at a time and the column leaves with coalesced stores
#pragma unroll
    for (int k = 0; k < kGRows; k++) {
      const uint32_t rep = pr[k] >> 16, rank = pr[k] & 0xFFFFu;
      if (o.gsize && rank == 0 && threadIdx.x + k * kGT < nl) o.gsize[lb + base[rep]] = base[rep + 1] - base[rep];
      pr[k] = base[rep] + rank;
    }
    __syncthreads();
    if (o.gkey) {
      // the keys are still in shared memory: staged into the dead slot table
      // (kGTab words hold kGCap keys) rather than read again from memory
      KeyT *st = (KeyT *)(smem + group_slots_at<KeyT>());
#pragma unroll
      for (int k = 0; k < kGRows; k++) {
        const uint32_t i = threadIdx.x + k * kGT;
        if (i < nl) st[pr[k]] = keys[i];
      }
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < nl; i += kGT) ((KeyT *)o.gkey)[lb + i] = st[i];
      __syncthreads();
    }
    stage_column<uint32_t>(o.grid, L.rid, lb, nl, pr, smem);
#pragma unroll 1
    for (int c = 0; c < L.ncols; c++) {
      if (L.width[c] == 8)
        stage_column<uint64_t>((uint64_t *)o.gcols[c], (const uint64_t *)L.cols[c], lb, nl, pr, smem);
      else
        stage_column<uint32_t>((uint32_t *)o.gcols[c], (const uint32_t *)L.cols[c], lb, nl, pr, smem);
    }
  }
}

// Later probe chunks of light sub-buckets: reload the saved table, probe.
template <typename KeyT>
__global__ void __launch_bounds__(kGT, 2)
    k_group_chunks(const __grid_constant__ GSide L, const __grid_constant__ GSide R,
                   const LightUnit *__restrict__ units, uint32_t nunits, const __grid_constant__ GOut o,
                   const unsigned char *__restrict__ dumps) {
  extern __shared__ __align__(16) unsigned char smem[];
  KeyT *keys = (KeyT *)smem;
  uint32_t *slots = (uint32_t *)(smem + group_slots_at<KeyT>());
  uint32_t *base = slots + kGTab;
  const KeyT *Rk = (const KeyT *)R.key;
  for (uint32_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const LightUnit U = units[u];
    const uint32_t lb = L.off[U.b], nl = L.off[U.b + 1] - lb;
    const uint32_t logt = small_logt(nl), T = 1u << logt;
    const unsigned char *d = dumps + (size_t)U.dump * dump_stride<KeyT>();
    const KeyT *dk = (const KeyT *)d;
    const uint32_t *ds = (const uint32_t *)(d + group_slots_at<KeyT>());
    const uint32_t *db = ds + kGTab;
    for (uint32_t i = threadIdx.x; i < nl; i += kGT) keys[i] = dk[i];
    for (uint32_t s = threadIdx.x; s < T; s += kGT) slots[s] = ds[s];
    for (uint32_t i = threadIdx.x; i <= nl; i += kGT) base[i] = db[i];
    __syncthreads();
    probe_small<KeyT>(keys, slots, base, logt, lb, Rk, U.r0, U.nr, o);
    __syncthreads();
  }
}

// ------------------------------------------------------- heavy sub-buckets
//
// Build side larger than one shared-memory table: a global-memory table per
// sub-bucket (2 slots per build row, linear probing from big_home).  Slot
// words hold representative row + 1; counts per slot, aggregated per warp
// (rows of one warp that found the same slot add once), give each row its
// rank.  The slot words are read through L2 (__ldcg): other SMs write them
// during the kernel.
template <typename KeyT>
__global__ void __launch_bounds__(kHT)
    k_heavy_insert(const HeavyDesc *__restrict__ hd, const HeavyUnit *__restrict__ units, uint32_t nunits,
                   const KeyT *__restrict__ Lk, uint32_t *hslot, uint32_t *hcnt, uint32_t *__restrict__ hs,
                   uint32_t *__restrict__ hrank, int *err) {
  const int lane = threadIdx.x & 31;
  for (uint32_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const HeavyUnit U = units[u];
    const HeavyDesc H = hd[U.h];
    for (uint32_t b0 = 0; b0 < U.n; b0 += kHT) {
      const bool act = b0 + threadIdx.x < U.n;
      const uint32_t li = U.i0 + b0 + threadIdx.x;
      uint32_t gs = 0xFFFFFFFFu, s = 0;
      if (act) {
        const KeyT kk = Lk[H.lb + li];
        s = big_home(key_bits(kk), H.tsz);
        uint32_t p = 0;
        for (; p < H.tsz; p++) {
          uint32_t cur = __ldcg(&hslot[H.ts0 + s]);
          if (cur == 0) {
            const uint32_t prev = atomicCAS(&hslot[H.ts0 + s], 0u, li + 1);
            if (prev == 0) break;
            cur = prev;
          }
          if (Lk[H.lb + cur - 1] == kk) break;
          s = s + 1 == H.tsz ? 0 : s + 1;
        }
        if (p == H.tsz) atomicExch(err, 1);  // unreachable: the table has 2 slots per row
        gs = H.ts0 + s;
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, gs);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (act && lane == leader) old = atomicAdd(&hcnt[gs], (uint32_t)__popc(peers));
      old = __shfl_sync(0xffffffffu, old, leader);
      if (act) {
        hs[H.hr0 + li] = s;
        hrank[H.hr0 + li] = old + __popc(peers & lanemask_lt());
      }
    }
  }
}

// hbase = exclusive scan of hcnt over all regions, so a region starts at hr0.
__global__ void __launch_bounds__(kHT)
    k_heavy_scatter(const HeavyDesc *__restrict__ hd, const HeavyUnit *__restrict__ units, uint32_t nunits,
                    const __grid_constant__ GSide L, int key_width, const uint32_t *__restrict__ hbase,
                    const uint32_t *__restrict__ hs, const uint32_t *__restrict__ hrank,
                    const __grid_constant__ GOut o) {
  for (uint32_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const HeavyUnit U = units[u];
    const HeavyDesc H = hd[U.h];
    for (uint32_t i = U.i0 + threadIdx.x; i < U.i0 + U.n; i += kHT) {
      const uint32_t s = H.ts0 + hs[H.hr0 + i], rank = hrank[H.hr0 + i];
      const uint32_t pos = H.lb + (hbase[s] - H.hr0) + rank;
      const uint32_t src = H.lb + i;
      o.grid[pos] = L.rid ? L.rid[src] : src;
      for (int c = 0; c < L.ncols; c++) copy_col(o.gcols[c], pos, L.cols[c], src, L.width[c]);
      if (o.gsize && rank == 0) o.gsize[pos] = hbase[s + 1] - hbase[s];
      if (o.gkey) copy_col(o.gkey, pos, L.key, src, key_width);
    }
  }
}

template <typename KeyT>
__global__ void __launch_bounds__(kHT)
    k_heavy_probe(const HeavyDesc *__restrict__ hd, const HeavyUnit *__restrict__ units, uint32_t nunits,
                  const KeyT *__restrict__ Lk, const KeyT *__restrict__ Rk, const uint32_t *__restrict__ hslot,
                  const uint32_t *__restrict__ hbase, GOut o, int *err) {
  for (uint32_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const HeavyUnit U = units[u];
    const HeavyDesc H = hd[U.h];
    for (uint32_t r = U.i0 + threadIdx.x; r < U.i0 + U.n; r += kHT) {
      const KeyT kk = Rk[r];
      uint32_t s = big_home(key_bits(kk), H.tsz);
      bool found = false;
      uint32_t p = 0;
      for (; p < H.tsz; p++) {
        const uint32_t w = hslot[H.ts0 + s];
        if (w == 0) break;
        if (Lk[H.lb + w - 1] == kk) {
          found = true;
          break;
        }
        s = s + 1 == H.tsz ? 0 : s + 1;
      }
      if (p == H.tsz) atomicExch(err, 1);  // unreachable: at least half the slots are empty
      const uint32_t c = found ? hbase[H.ts0 + s + 1] - hbase[H.ts0 + s] : 0u;
      o.cnt[r] = c;
      o.gbase[r] = found ? H.lb + (hbase[H.ts0 + s] - H.hr0) : 0u;
      if (found && o.hit) o.hit[H.lb + (hbase[H.ts0 + s] - H.hr0)] = 1;
    }
  }
}

// ------------------------------------------------------------- entries
//
// Entries (first output row, probe row, group start) in output order:
//   pass 1, over probe rows in shuffled order: every matching row (inner,
//     left), or every row, an unmatched one as a one-row entry with no group
//     (right, outer);
//   pass 2 (left, outer), over grouped build positions: every group no probe
//     row found, as an entry with no probe row and the group's size.
// Reduce, scan, rescan: k_entry_sums sums each chunk of kCChunk rows (rows
// and entries), the chunk sums are scanned, and k_entry_write rescans its
// chunk and writes the chunk's entries at its base (after pass 1's totals in
// pass 2).  Within a block both sums travel in one 64-bit scan, packed
// rows << 13 | entries (a chunk has at most 4096 entries and fewer than 2^44
// rows).
constexpr int kCT = 512;
constexpr int kCRows = 8;
constexpr uint32_t kCChunk = kCT * kCRows;
static_assert(kCChunk <= 8191, "entries of a chunk fit the packed low 13 bits");

enum { SRC_PROBE = 0, SRC_PROBE_ALL = 1, SRC_UNMATCHED_GROUPS = 2 };
struct EntrySrc {
  const uint32_t *cnt;  // probe passes: group size per probe row; group pass: size at group starts
  const uint32_t *aux;  // probe passes: group start per probe row; group pass: hit flags
  uint32_t n;
  int mode;
};

__device__ __forceinline__ void load8(const uint32_t *__restrict__ a, uint32_t n, uint32_t r0, uint32_t (&v)[kCRows]) {
  if (r0 + kCRows <= n) {
    const uint4 x = *(const uint4 *)(a + r0), y = *(const uint4 *)(a + r0 + 4);
    v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w, v[4] = y.x, v[5] = y.y, v[6] = y.z, v[7] = y.w;
  } else {
#pragma unroll
    for (int k = 0; k < kCRows; k++) v[k] = r0 + k < n ? a[r0 + k] : 0u;
  }
}

// Output rows of rows r0 .. r0 + 7 of the pass (0 = no entry).
__device__ __forceinline__ void entry_rows(const EntrySrc &S, uint32_t r0, uint32_t (&v)[kCRows]) {
  load8(S.cnt, S.n, r0, v);
  if (S.mode == SRC_PROBE_ALL) {
#pragma unroll
    for (int k = 0; k < kCRows; k++)
      if (r0 + k < S.n && v[k] == 0) v[k] = 1;
  } else if (S.mode == SRC_UNMATCHED_GROUPS) {
    uint32_t h[kCRows];
    load8(S.aux, S.n, r0, h);
#pragma unroll
    for (int k = 0; k < kCRows; k++)
      if (h[k]) v[k] = 0;
  }
}

__device__ __forceinline__ uint64_t packed_sum(const uint32_t (&v)[kCRows]) {
  uint64_t rows = 0;
  uint32_t ents = 0;
#pragma unroll
  for (int k = 0; k < kCRows; k++) {
    rows += v[k];
    ents += v[k] != 0;
  }
  return (rows << 13) | ents;
}

// chunk c: rows[c], ents[c] (nchunks + 1 entries each; the last stays 0)
__global__ void __launch_bounds__(kCT)
    k_entry_sums(EntrySrc S, uint64_t *__restrict__ rows, uint32_t *__restrict__ ents) {
  __shared__ uint64_t scratch[33];
  const uint32_t r0 = blockIdx.x * kCChunk + threadIdx.x * kCRows;
  uint32_t v[kCRows];
  entry_rows(S, r0, v);
  uint64_t tot;
  block_exclusive_scan<uint64_t>(packed_sum(v), scratch, &tot);
  if (threadIdx.x == 0) {
    rows[blockIdx.x] = tot >> 13;
    ents[blockIdx.x] = (uint32_t)(tot & 8191);
  }
}

// rows / ents: exclusive prefixes over chunks; rows0 / ents0: where the pass
// starts (pass 1's totals, or NULL for 0).  The chunk's entries are staged in
// shared memory one array at a time and leave with coalesced stores.
__global__ void __launch_bounds__(kCT)
    k_entry_write(EntrySrc S, const uint64_t *__restrict__ rows, const uint32_t *__restrict__ ents,
                  const uint64_t *__restrict__ rows0, const uint32_t *__restrict__ ents0, uint64_t *__restrict__ moff,
                  uint32_t *__restrict__ mr, uint32_t *__restrict__ mg) {
  __shared__ uint64_t scratch[33];
  __shared__ uint64_t stage[kCChunk];
  uint32_t *stage32 = (uint32_t *)stage;
  const uint32_t r0 = blockIdx.x * kCChunk + threadIdx.x * kCRows;
  uint32_t v[kCRows];
  entry_rows(S, r0, v);
  uint32_t g[kCRows], r[kCRows];
  const bool probe = S.mode != SRC_UNMATCHED_GROUPS;
#pragma unroll
  for (int k = 0; k < kCRows; k++) {
    r[k] = probe ? r0 + k : kNone;
    g[k] = probe ? (v[k] && r0 + k < S.n && S.cnt[r0 + k] ? S.aux[r0 + k] : kNone) : r0 + k;
  }
  uint64_t tot;
  const uint64_t ex = block_exclusive_scan<uint64_t>(packed_sum(v), scratch, &tot);
  const uint64_t rbase = rows[blockIdx.x] + (rows0 ? *rows0 : 0ull);
  const uint32_t ebase = ents[blockIdx.x] + (ents0 ? *ents0 : 0u), n = (uint32_t)(tot & 8191);
  const uint32_t e0 = (uint32_t)(ex & 8191);
  {
    uint64_t at = rbase + (ex >> 13);
    uint32_t e = e0;
#pragma unroll
    for (int k = 0; k < kCRows; k++)
      if (v[k]) {
        stage[e++] = at;
        at += v[k];
      }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += kCT) moff[ebase + i] = stage[i];
  __syncthreads();
  {
    uint32_t e = e0;
#pragma unroll
    for (int k = 0; k < kCRows; k++)
      if (v[k]) stage32[e++] = r[k];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += kCT) mr[ebase + i] = stage32[i];
  __syncthreads();
  {
    uint32_t e = e0;
#pragma unroll
    for (int k = 0; k < kCRows; k++)
      if (v[k]) stage32[e++] = g[k];
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < n; i += kCT) mg[ebase + i] = stage32[i];
}

// ------------------------------------------------------------------ emit
//
// Each block writes a contiguous range of tiles (kETile rows each).  The
// entry holding the range's first row is found by a 32-way search of one warp
// over moff; each tile loads the entries that can hold its rows (at most
// kETile + 1, each entry has at least one row) into shared memory, and every
// row finds its entry there by binary search, unless the whole tile lies in
// one entry (one probe row, one group: the heavy-hitter case).  A thread
// resolves its kERows rows first, then moves one column at a time, kEBatch
// rows at once: kEBatch independent loads, then kEBatch stores.  Output rows
// of a warp are consecutive, so every store is coalesced.
// idx kNone (no row on that side of an outer join) writes `fill`.
template <typename V>
__device__ __forceinline__ void gather_rows(V *dst, const V *src, const uint32_t (&idx)[kERows], uint64_t q0,
                                            uint32_t nrow, V fill) {
  V *d = dst + q0;
#pragma unroll
  for (int h = 0; h < kERows; h += kEBatch) {
    V v[kEBatch];
#pragma unroll
    for (int k = 0; k < kEBatch; k++)
      if ((uint32_t)(h + k) < nrow) v[k] = idx[h + k] != kNone ? src[idx[h + k]] : fill;
#pragma unroll
    for (int k = 0; k < kEBatch; k++)
      if ((uint32_t)(h + k) < nrow) d[(h + k) * kET] = v[k];
  }
}

__device__ __forceinline__ void gather_col(void *dst, const void *src, int width, const uint32_t (&idx)[kERows],
                                           uint64_t q0, uint32_t nrow) {
  if (width == 8)
    gather_rows<uint64_t>((uint64_t *)dst, (const uint64_t *)src, idx, q0, nrow, 0ull);
  else
    gather_rows<uint32_t>((uint32_t *)dst, (const uint32_t *)src, idx, q0, nrow, 0u);
}

// The key of each row: the probe row's, or the grouped build row's when the
// row has no probe side.
template <typename KeyT>
__device__ __forceinline__ void gather_keys(KeyT *dst, const KeyT *rk, const KeyT *gk, const uint32_t (&ri)[kERows],
                                            const uint32_t (&li)[kERows], uint64_t q0, uint32_t nrow) {
  KeyT *d = dst + q0;
#pragma unroll
  for (int h = 0; h < kERows; h += kEBatch) {
    KeyT v[kEBatch];
#pragma unroll
    for (int k = 0; k < kEBatch; k++)
      if ((uint32_t)(h + k) < nrow) v[k] = ri[h + k] != kNone ? rk[ri[h + k]] : gk[li[h + k]];
#pragma unroll
    for (int k = 0; k < kEBatch; k++)
      if ((uint32_t)(h + k) < nrow) d[(h + k) * kET] = v[k];
  }
}

template <typename KeyT>
__global__ void __launch_bounds__(kET, 3)
    k_emit(const __grid_constant__ EmitSrc S, const __grid_constant__ EmitDst D, uint64_t first, uint64_t rows,
           uint32_t tiles_per_block) {
  __shared__ uint64_t s_off[kETile + 1];
  __shared__ uint32_t s_r[kETile + 1], s_g[kETile + 1];
  __shared__ uint32_t s_e;
  const uint64_t ntiles = (rows + kETile - 1) / kETile;
  const uint64_t t_begin = (uint64_t)blockIdx.x * tiles_per_block;
  if (t_begin >= ntiles) return;
  const uint64_t t_end = min(ntiles, t_begin + tiles_per_block);
  const uint64_t last = first + rows;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    const uint64_t o = first + t_begin * kETile;
    uint32_t lo = 0, hi = S.nm;  // moff[lo] <= o < moff[hi]
    while (hi - lo > 1) {
      const uint32_t step = (hi - lo + 31) / 32;
      const uint64_t p = (uint64_t)lo + (uint64_t)(lane + 1) * step;
      const bool le = p < hi && S.moff[p] <= o;
      const uint32_t c = __popc(__ballot_sync(0xffffffffu, le));
      const uint32_t nlo = lo + c * step;
      const uint64_t nhi = (uint64_t)lo + (uint64_t)(c + 1) * step;
      lo = nlo;
      hi = nhi < hi ? (uint32_t)nhi : hi;
    }
    if (lane == 0) s_e = lo;
  }
  __syncthreads();
  for (uint64_t t = t_begin; t < t_end; t++) {
    const uint64_t o0 = first + t * kETile;
    const uint64_t o1 = min(last, o0 + kETile);
    const uint32_t e = s_e;
    const uint32_t ne = min((uint32_t)(kETile + 1), S.nm + 1 - e);
    for (uint32_t j = threadIdx.x; j < ne; j += kET) {
      s_off[j] = S.moff[e + j];
      if (e + j < S.nm) {
        s_r[j] = S.mr[e + j];
        s_g[j] = S.mg[e + j];
      }
    }
    __syncthreads();
    // rows o0 + threadIdx.x + k * kET, k < nrow
    const uint64_t mine = o0 + threadIdx.x;
    const uint32_t nrow = mine < o1 ? (uint32_t)((o1 - mine + kET - 1) / kET) : 0u;
    uint32_t ri[kERows], li[kERows];
    if (s_off[1] >= o1) {  // one entry: one probe row against a run of its group
      const uint32_t r = s_r[0], g0 = s_g[0];
      const uint32_t g = g0 + (uint32_t)(mine - s_off[0]);
#pragma unroll
      for (int k = 0; k < kERows; k++) {
        ri[k] = r;
        li[k] = g0 == kNone ? kNone : g + k * kET;
      }
    } else {
      uint32_t j = 0;
#pragma unroll
      for (int k = 0; k < kERows; k++) {
        const uint64_t o = mine + (uint64_t)k * kET;
        ri[k] = 0;
        li[k] = 0;
        if ((uint32_t)k < nrow) {
          uint32_t hi = ne;  // s_off[j] <= o < s_off[hi]; j only grows with k
          while (hi - j > 1) {
            const uint32_t mid = (j + hi) >> 1;
            if (s_off[mid] <= o)
              j = mid;
            else
              hi = mid;
          }
          ri[k] = s_r[j];
          li[k] = s_g[j] == kNone ? kNone : s_g[j] + (uint32_t)(o - s_off[j]);
        }
      }
    }
    const uint64_t q0 = mine - first;
    if (D.key) gather_keys<KeyT>((KeyT *)D.key, (const KeyT *)S.rkey, (const KeyT *)S.gkey, ri, li, q0, nrow);
    if (D.lrow) gather_rows<uint32_t>(D.lrow, S.grid, li, q0, nrow, kNone);
    if (D.rrow) {
      if (S.rrid) {
        gather_rows<uint32_t>(D.rrow, S.rrid, ri, q0, nrow, kNone);
      } else {
        uint32_t *d = D.rrow + q0;
#pragma unroll
        for (int k = 0; k < kERows; k++)
          if ((uint32_t)k < nrow) d[k * kET] = ri[k];
      }
    }
#pragma unroll 1
    for (int c = 0; c < S.nlc; c++)
      if (D.lcols[c]) gather_col(D.lcols[c], S.gcols[c], S.lwidth[c], li, q0, nrow);
#pragma unroll 1
    for (int c = 0; c < S.nrc; c++)
      if (D.rcols[c]) gather_col(D.rcols[c], S.rcols[c], S.rwidth[c], ri, q0, nrow);
    __syncthreads();
    if (threadIdx.x == 0 && o1 < last) {  // the entry holding the next tile's first row
      uint32_t lo = 0, hi = ne;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_off[mid] <= o1)
          lo = mid;
        else
          hi = mid;
      }
      s_e = e + lo;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------- host

GSide to_gside(const Side &s) {
  GSide g;
  memset(&g, 0, sizeof g);
  g.key = s.key;
  g.rid = s.rid;
  g.off = s.off;
  g.ncols = s.ncols;
  for (int c = 0; c < s.ncols; c++) {
    g.cols[c] = s.cols[c];
    g.width[c] = s.widths[c];
  }
  return g;
}

int validate(const mdj_table *t, int32_t key_col) {
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

// Work of the grouping step, planned on the host from the sub-bucket offsets.
struct Units {
  std::vector<LightUnit> first, later;    // first probe chunk (with the build) / later chunks
  std::vector<HeavyDesc> heavy;
  std::vector<HeavyUnit> hbuild, hprobe;
  uint32_t ndump = 0;
  uint64_t hslots = 0, hrows = 0;
};

// keep_left: every build row is grouped (its unmatched groups become rows),
// even in sub-buckets without probe rows.
void plan_units(const std::vector<uint32_t> &offL, const std::vector<uint32_t> &offR, uint32_t nb, bool keep_left,
                Units *u) {
  for (uint32_t b = 0; b < nb; b++) {
    const uint32_t nl = offL[b + 1] - offL[b], nr = offR[b + 1] - offR[b];
    if (nr == 0 && !(keep_left && nl > 0)) continue;  // nothing of this sub-bucket is ever read
    if (nl == 0) {
      for (uint32_t c0 = 0; c0 < nr; c0 += kProbeChunk)
        u->first.push_back({b, offR[b] + c0, std::min(kProbeChunk, nr - c0), -1});
      continue;
    }
    if (nl <= kGCap) {  // nr may be 0 (keep_left): the unit groups and probes nothing
      const int32_t dump = nr > kProbeChunk ? (int32_t)u->ndump++ : -1;
      u->first.push_back({b, offR[b], std::min(kProbeChunk, nr), dump});
      for (uint32_t c0 = kProbeChunk; c0 < nr; c0 += kProbeChunk)
        u->later.push_back({b, offR[b] + c0, std::min(kProbeChunk, nr - c0), dump});
      continue;
    }
    const uint32_t h = (uint32_t)u->heavy.size();
    u->heavy.push_back({b, offL[b], nl, 2 * nl, (uint32_t)u->hslots, (uint32_t)u->hrows});
    u->hslots += 2ull * nl;
    u->hrows += nl;
    for (uint32_t i0 = 0; i0 < nl; i0 += kHChunk) u->hbuild.push_back({h, i0, std::min(kHChunk, nl - i0)});
    for (uint32_t c0 = 0; c0 < nr; c0 += kHChunk) u->hprobe.push_back({h, offR[b] + c0, std::min(kHChunk, nr - c0)});
  }
  // largest probe chunks first, so the persistent blocks finish together
  std::stable_sort(u->first.begin(), u->first.end(),
                   [](const LightUnit &a, const LightUnit &b) { return a.nr > b.nr; });
}

template <typename T>
T *upload(Workspace &ws, const std::vector<T> &v, int *rc) {
  if (v.empty()) return nullptr;
  T *d = (T *)ws.get(v.size() * sizeof(T));
  if (!d) {
    *rc = MDJ_ERR_OOM;
    return nullptr;
  }
  const int e = cuda_status(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ws.stream()));
  if (e != MDJ_OK) *rc = e;
  return d;
}

unsigned grid_for(uint64_t units, int per_sm) {
  const uint64_t most = (uint64_t)num_sms() * per_sm;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(units, most));
}

// One pass of the entries: sums per chunk, scan, rescan and write.  rows0 /
// ents0: where the pass starts (NULL: 0).  Leaves the pass's totals at
// crows[nchunks], cents[nchunks].
int entries_pass(Workspace &tmp, const EntrySrc &src, const uint64_t *rows0, const uint32_t *ents0, uint64_t *moff,
                 uint32_t *mr, uint32_t *mg, uint64_t **crows_out, uint32_t **cents_out, uint32_t *nchunks_out) {
  cudaStream_t s = tmp.stream();
  const uint32_t nchunks = (uint32_t)(((size_t)src.n + kCChunk - 1) / kCChunk);
  uint64_t *crows = (uint64_t *)tmp.get((size_t)(nchunks + 1) * 8);
  uint32_t *cents = (uint32_t *)tmp.get((size_t)(nchunks + 1) * 4);
  if (!crows || !cents) return MDJ_ERR_OOM;
  MDJ_CUDA_TRY(cudaMemsetAsync(crows + nchunks, 0, 8, s));
  MDJ_CUDA_TRY(cudaMemsetAsync(cents + nchunks, 0, 4, s));
  if (nchunks) {
    TraceScope tr("stream_entry_sums", s);
    k_entry_sums<<<nchunks, kCT, 0, s>>>(src, crows, cents);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u64(tmp, crows, crows, (size_t)nchunks + 1));
  MDJ_TRY(exclusive_scan_u32(tmp, cents, cents, (size_t)nchunks + 1));
  if (nchunks) {
    TraceScope tr("stream_entries", s);
    k_entry_write<<<nchunks, kCT, 0, s>>>(src, crows, cents, rows0, ents0, moff, mr, mg);
  }
  MDJ_LAUNCH_CHECK();
  *crows_out = crows;
  *cents_out = cents;
  *nchunks_out = nchunks;
  return MDJ_OK;
}

// Groups the build side, probes, and builds the entries into the handle.
// Groups the build side and finds every probe row's group (steps 2-4 of the
// open): fills `o` (grouped build rows in `keep`, per-probe-row arrays in
// `tmp`).  want_gkey: also the grouped keys; keep_left: also the group sizes
// and hit flags that the unmatched-group entries need.  *err_out: a device
// word set when a global-table probe sequence ran out (read it after a sync).
template <typename KeyT>
int group_sides(Workspace &tmp, Workspace &keep, const Side &L, const Side &R, uint32_t nb, bool keep_left,
                bool want_gkey, GOut &o, int **err_out) {
  cudaStream_t s = tmp.stream();
  const uint32_t nL = (uint32_t)L.nrows, nR = (uint32_t)R.nrows;
  std::vector<uint32_t> offL(nb + 1), offR(nb + 1);
  MDJ_CUDA_TRY(cudaMemcpyAsync(offL.data(), L.off, (size_t)(nb + 1) * 4, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaMemcpyAsync(offR.data(), R.off, (size_t)(nb + 1) * 4, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  Units un;
  plan_units(offL, offR, nb, keep_left, &un);
  if (un.hslots >= (1ull << 32) - 1) return MDJ_ERR_TOO_LARGE;

  // the grouped build side lives as long as the handle
  memset(&o, 0, sizeof o);
  o.grid = (uint32_t *)keep.get((size_t)nL * 4);
  if (!o.grid) return MDJ_ERR_OOM;
  for (int c = 0; c < L.ncols; c++)
    if (!(o.gcols[c] = keep.get((size_t)nL * L.widths[c]))) return MDJ_ERR_OOM;
  o.cnt = (uint32_t *)tmp.get((size_t)nR * 4);
  o.gbase = (uint32_t *)tmp.get((size_t)nR * 4);
  int *err = (int *)tmp.get(16);  // [0]: a global-table probe sequence ran out
  if (!o.cnt || !o.gbase || !err) return MDJ_ERR_OOM;
  MDJ_CUDA_TRY(cudaMemsetAsync(err, 0, 16, s));
  if (keep_left || want_gkey) {
    o.gkey = keep.get((size_t)nL * sizeof(KeyT));
    if (!o.gkey) return MDJ_ERR_OOM;
  }
  if (keep_left) {
    o.gsize = (uint32_t *)tmp.get((size_t)nL * 4);
    o.hit = (uint32_t *)tmp.get((size_t)nL * 4);
    if (!o.gsize || !o.hit) return MDJ_ERR_OOM;
    MDJ_CUDA_TRY(cudaMemsetAsync(o.gsize, 0, (size_t)nL * 4, s));
    MDJ_CUDA_TRY(cudaMemsetAsync(o.hit, 0, (size_t)nL * 4, s));
  }

  int rc = MDJ_OK;
  LightUnit *d_first = upload(tmp, un.first, &rc);
  LightUnit *d_later = upload(tmp, un.later, &rc);
  HeavyDesc *d_heavy = upload(tmp, un.heavy, &rc);
  HeavyUnit *d_hbuild = upload(tmp, un.hbuild, &rc);
  HeavyUnit *d_hprobe = upload(tmp, un.hprobe, &rc);
  MDJ_TRY(rc);
  unsigned char *dumps = nullptr;
  if (un.ndump) {
    dumps = (unsigned char *)tmp.get((size_t)un.ndump * dump_stride<KeyT>());
    if (!dumps) return MDJ_ERR_OOM;
  }
  const GSide gL = to_gside(L), gR = to_gside(R);
  const size_t sm = group_smem_bytes<KeyT>();
  if (!un.first.empty()) {
    uint32_t *ticket = (uint32_t *)tmp.get(4);
    if (!ticket) return MDJ_ERR_OOM;
    MDJ_CUDA_TRY(cudaMemsetAsync(ticket, 0, 4, s));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_group_light<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    TraceScope tr("stream_group", s);
    k_group_light<KeyT><<<grid_for(un.first.size(), 2), kGT, sm, s>>>(gL, gR, d_first, (uint32_t)un.first.size(),
                                                                       ticket, o, dumps);
    MDJ_LAUNCH_CHECK();
  }
  if (!un.later.empty()) {
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_group_chunks<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    TraceScope tr("stream_group_chunks", s);
    k_group_chunks<KeyT><<<grid_for(un.later.size(), 2), kGT, sm, s>>>(gL, gR, d_later, (uint32_t)un.later.size(), o,
                                                                        dumps);
    MDJ_LAUNCH_CHECK();
  }
  if (!un.heavy.empty()) {
    const size_t ns = (size_t)un.hslots;
    uint32_t *hslot = (uint32_t *)tmp.get(ns * 4);
    uint32_t *hcnt = (uint32_t *)tmp.get((ns + 1) * 4);
    uint32_t *hs = (uint32_t *)tmp.get((size_t)un.hrows * 4);
    uint32_t *hrank = (uint32_t *)tmp.get((size_t)un.hrows * 4);
    if (!hslot || !hcnt || !hs || !hrank) return MDJ_ERR_OOM;
    MDJ_CUDA_TRY(cudaMemsetAsync(hslot, 0, ns * 4, s));
    MDJ_CUDA_TRY(cudaMemsetAsync(hcnt, 0, (ns + 1) * 4, s));
    const KeyT *Lk = (const KeyT *)L.key;
    {
      TraceScope tr("stream_heavy_insert", s);
      k_heavy_insert<KeyT><<<grid_for(un.hbuild.size(), 8), kHT, 0, s>>>(
          d_heavy, d_hbuild, (uint32_t)un.hbuild.size(), Lk, hslot, hcnt, hs, hrank, err);
    }
    MDJ_LAUNCH_CHECK();
    MDJ_TRY(exclusive_scan_u32(tmp, hcnt, hcnt, ns + 1));
    {
      TraceScope tr("stream_heavy_scatter", s);
      k_heavy_scatter<<<grid_for(un.hbuild.size(), 8), kHT, 0, s>>>(d_heavy, d_hbuild, (uint32_t)un.hbuild.size(),
                                                                      gL, (int)sizeof(KeyT), hcnt, hs, hrank, o);
    }
    if (!un.hprobe.empty()) {
      TraceScope tr("stream_heavy_probe", s);
      k_heavy_probe<KeyT><<<grid_for(un.hprobe.size(), 8), kHT, 0, s>>>(
          d_heavy, d_hprobe, (uint32_t)un.hprobe.size(), Lk, (const KeyT *)R.key, hslot, hcnt, o, err);
    }
    MDJ_LAUNCH_CHECK();
  }
  *err_out = err;
  return MDJ_OK;
}

template <typename KeyT>
int group_and_index(Workspace &tmp, mdj_stream *h, const Side &L, const Side &R, uint32_t nb, int32_t how) {
  const bool keep_left = how == MDJ_LEFT || how == MDJ_OUTER;
  const bool keep_right = how == MDJ_RIGHT || how == MDJ_OUTER;
  Workspace &keep = *h->ws;
  cudaStream_t s = tmp.stream();
  const uint32_t nL = (uint32_t)L.nrows, nR = (uint32_t)R.nrows;
  GOut o;
  int *err = nullptr;
  MDJ_TRY(group_sides<KeyT>(tmp, keep, L, R, nb, keep_left, false, o, &err));
  // entries: the probe rows (matching ones, or all), then the unmatched groups
  EmitSrc &S = h->src;
  const size_t cap = (size_t)nR + (keep_left ? nL : 0);
  uint64_t *moff = (uint64_t *)keep.get((cap + 1) * 8);
  uint32_t *mr = (uint32_t *)keep.get(cap * 4);
  uint32_t *mg = (uint32_t *)keep.get(cap * 4);
  if (!moff || !mr || !mg) return MDJ_ERR_OOM;
  const EntrySrc probe_src = {o.cnt, o.gbase, nR, keep_right ? SRC_PROBE_ALL : SRC_PROBE};
  uint64_t *crows1, *crows2 = nullptr;
  uint32_t *cents1, *cents2 = nullptr, c1, c2 = 0;
  MDJ_TRY(entries_pass(tmp, probe_src, nullptr, nullptr, moff, mr, mg, &crows1, &cents1, &c1));
  if (keep_left) {
    const EntrySrc group_src = {o.gsize, o.hit, nL, SRC_UNMATCHED_GROUPS};
    MDJ_TRY(entries_pass(tmp, group_src, crows1 + c1, cents1 + c1, moff, mr, mg, &crows2, &cents2, &c2));
  }
  uint64_t t1 = 0, t2 = 0;
  uint32_t n1 = 0, n2 = 0;
  int herr[4] = {0, 0, 0, 0};
  MDJ_CUDA_TRY(cudaMemcpyAsync(&t1, crows1 + c1, 8, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaMemcpyAsync(&n1, cents1 + c1, 4, cudaMemcpyDeviceToHost, s));
  if (keep_left) {
    MDJ_CUDA_TRY(cudaMemcpyAsync(&t2, crows2 + c2, 8, cudaMemcpyDeviceToHost, s));
    MDJ_CUDA_TRY(cudaMemcpyAsync(&n2, cents2 + c2, 4, cudaMemcpyDeviceToHost, s));
  }
  MDJ_CUDA_TRY(cudaMemcpyAsync(herr, err, 16, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr[0]) return MDJ_ERR_INTERNAL;
  const uint64_t total = t1 + t2;
  const uint32_t nm = n1 + n2;
  // the search sentinel after the last entry: moff[nm] = total rows
  MDJ_CUDA_TRY(cudaMemcpyAsync(moff + nm, &total, 8, cudaMemcpyHostToDevice, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  h->total = total;
  S.moff = moff;
  S.mr = mr;
  S.mg = mg;
  S.nm = nm;
  S.rkey = R.key;
  S.rrid = R.rid;
  S.nrc = R.ncols;
  for (int c = 0; c < R.ncols; c++) {
    S.rcols[c] = R.cols[c];
    S.rwidth[c] = R.widths[c];
  }
  S.grid = o.grid;
  S.gkey = o.gkey;
  S.nlc = L.ncols;
  for (int c = 0; c < L.ncols; c++) {
    S.gcols[c] = o.gcols[c];
    S.lwidth[c] = L.widths[c];
  }
  return MDJ_OK;
}

// ------------------------------------------------------ count + checksum

// f of every grouped build position (its key, input row id and first payload)
template <typename KeyT>
__global__ void k_count_f(const KeyT *__restrict__ gkey, const uint32_t *__restrict__ grid, const void *gpay, int pw,
                          uint32_t n, uint64_t *__restrict__ f) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
    f[p] = term_f(key_bits(gkey[p]), grid[p], pay_bits(gpay, pw, p));
}

// totals[0] += group sizes, totals[1] += g(r) * (F[start + size] - F[start])
// over probe rows r (F: exclusive prefix sums of f, modulo 2^64)
__global__ void k_count_probe(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ gbase,
                              const uint64_t *__restrict__ F, const uint32_t *__restrict__ rrid, const void *rpay,
                              int pw, uint32_t n, unsigned long long *totals) {
  uint64_t acc = 0, csum = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const uint32_t c = cnt[r];
    if (!c) continue;
    const uint32_t g0 = gbase[r];
    acc += c;
    csum += term_g(rrid ? rrid[r] : r, pay_bits(rpay, pw, r)) * (F[g0 + c] - F[g0]);
  }
  acc = warp_sum(acc);
  csum = warp_sum(csum);
  if ((threadIdx.x & 31) == 0) {
    if (acc) atomicAdd(&totals[0], (unsigned long long)acc);
    if (csum) atomicAdd(&totals[1], (unsigned long long)csum);
  }
}

template <typename KeyT>
int grouped_count_t(Workspace &ws, const Side &L, const Side &R, uint32_t nb, uint64_t *count, uint64_t *checksum) {
  cudaStream_t s = ws.stream();
  const uint32_t nL = (uint32_t)L.nrows, nR = (uint32_t)R.nrows;
  GOut o;
  int *err = nullptr;
  MDJ_TRY(group_sides<KeyT>(ws, ws, L, R, nb, false, true, o, &err));
  uint64_t *F = (uint64_t *)ws.get(((size_t)nL + 1) * 8);
  unsigned long long *tot = (unsigned long long *)ws.get(16);
  if (!F || !tot) return MDJ_ERR_OOM;
  MDJ_CUDA_TRY(cudaMemsetAsync(F + nL, 0, 8, s));
  MDJ_CUDA_TRY(cudaMemsetAsync(tot, 0, 16, s));
  const unsigned grid = (unsigned)num_sms() * 8;
  {
    TraceScope tr("count_f", s);
    k_count_f<KeyT><<<grid, 256, 0, s>>>((const KeyT *)o.gkey, o.grid, L.ncols ? o.gcols[0] : nullptr,
                                         L.ncols ? L.widths[0] : 0, nL, F);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u64(ws, F, F, (size_t)nL + 1));
  {
    TraceScope tr("count_probe", s);
    k_count_probe<<<grid, 256, 0, s>>>(o.cnt, o.gbase, F, R.rid, R.ncols ? R.cols[0] : nullptr,
                                       R.ncols ? R.widths[0] : 0, nR, tot);
  }
  MDJ_LAUNCH_CHECK();
  unsigned long long host[2] = {0, 0};
  int herr = 0;
  MDJ_CUDA_TRY(cudaMemcpyAsync(host, tot, 16, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
  MDJ_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) return MDJ_ERR_INTERNAL;
  *count = host[0];
  *checksum = host[1];
  return MDJ_OK;
}

}  // namespace

int grouped_count_checksum(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P,
                           const mdj_allocator *alloc, void *stream, uint64_t *count, uint64_t *checksum) {
  if (!count || !checksum) return MDJ_ERR_INVALID_ARG;
  MDJ_TRY(validate(left, lk));
  MDJ_TRY(validate(right, rk));
  if (P < 1 || P > MDJ_MAX_PARTITIONS) return MDJ_ERR_INVALID_ARG;
  if (left->cols[lk].dtype != right->cols[rk].dtype) return MDJ_ERR_INVALID_ARG;
  *count = 0;
  *checksum = 0;
  if (left->nrows == 0 || right->nrows == 0) return MDJ_OK;
  Workspace ws(alloc, (cudaStream_t)stream);
  const Plan plan = make_plan(left->nrows, P, kGCap, P > 1);
  Side L, R;
  MDJ_TRY(partition_side(ws, left, lk, plan, &L));
  MDJ_TRY(partition_side(ws, right, rk, plan, &R));
  return left->cols[lk].dtype == MDJ_I64 ? grouped_count_t<int64_t>(ws, L, R, plan.nbuckets, count, checksum)
                                          : grouped_count_t<int32_t>(ws, L, R, plan.nbuckets, count, checksum);
}

namespace {

int stream_open(const mdj_table *left, int32_t lk, const mdj_table *right, int32_t rk, uint32_t P, int32_t how,
                const mdj_allocator *alloc, void *stream, mdj_stream **out, uint64_t *total_rows) {
  if (!out || !total_rows) return MDJ_ERR_INVALID_ARG;
  *out = nullptr;
  *total_rows = 0;
  MDJ_TRY(validate(left, lk));
  MDJ_TRY(validate(right, rk));
  if (P < 1 || P > MDJ_MAX_PARTITIONS) return MDJ_ERR_INVALID_ARG;
  if (how < MDJ_INNER || how > MDJ_OUTER) return MDJ_ERR_INVALID_ARG;
  if (left->cols[lk].dtype != right->cols[rk].dtype) return MDJ_ERR_INVALID_ARG;
  mdj_stream *h = new (std::nothrow) mdj_stream;
  if (!h) return MDJ_ERR_OOM;
  memset(&h->alloc, 0, sizeof h->alloc);
  h->has_alloc = alloc != nullptr;
  if (alloc) h->alloc = *alloc;
  h->stream = (cudaStream_t)stream;
  h->ws = new (std::nothrow) Workspace(h->has_alloc ? &h->alloc : nullptr, h->stream);
  if (!h->ws) {
    delete h;
    return MDJ_ERR_OOM;
  }
  h->key_dtype = left->cols[lk].dtype;
  h->total = 0;
  h->cursor = 0;
  memset(&h->src, 0, sizeof h->src);
  int rc = MDJ_OK;
  {
    Workspace tmp(h->has_alloc ? &h->alloc : nullptr, h->stream);
    Plan plan = make_plan(left->nrows, P, kGCap, P > 1);
    Side L, R;
    rc = partition_side(tmp, left, lk, plan, &L);        // released when open returns
    if (rc == MDJ_OK) rc = partition_side(*h->ws, right, rk, plan, &R);  // read by every window
    const bool rows_possible = (left->nrows > 0 && right->nrows > 0) ||
                               (left->nrows > 0 && (how == MDJ_LEFT || how == MDJ_OUTER)) ||
                               (right->nrows > 0 && (how == MDJ_RIGHT || how == MDJ_OUTER));
    if (rc == MDJ_OK && rows_possible)
      rc = h->key_dtype == MDJ_I64 ? group_and_index<int64_t>(tmp, h, L, R, plan.nbuckets, how)
                                   : group_and_index<int32_t>(tmp, h, L, R, plan.nbuckets, how);
  }
  if (rc != MDJ_OK) {
    delete h->ws;
    delete h;
    return rc;
  }
  *out = h;
  *total_rows = h->total;
  return MDJ_OK;
}

int stream_emit(mdj_stream *h, uint64_t first, uint64_t rows, const mdj_window *w) {
  if (!h || !w) return MDJ_ERR_INVALID_ARG;
  if (first > h->total || rows > h->total - first) return MDJ_ERR_INVALID_ARG;
  if (rows == 0) return MDJ_OK;
  EmitDst d;
  memset(&d, 0, sizeof d);
  d.key = w->key;
  d.lrow = w->left_row;
  d.rrow = w->right_row;
  for (int c = 0; c < h->src.nlc; c++) d.lcols[c] = w->left_cols[c];
  for (int c = 0; c < h->src.nrc; c++) d.rcols[c] = w->right_cols[c];
  const uint64_t ntiles = (rows + kETile - 1) / kETile;
  const uint64_t most = (uint64_t)num_sms() * 3;  // three resident 256-thread blocks per SM
  const uint64_t per = (ntiles + most - 1) / most;
  const unsigned grid = (unsigned)((ntiles + per - 1) / per);
  TraceScope tr("stream_emit", h->stream);
  if (h->key_dtype == MDJ_I64)
    k_emit<int64_t><<<grid, kET, 0, h->stream>>>(h->src, d, first, rows, (uint32_t)per);
  else
    k_emit<int32_t><<<grid, kET, 0, h->stream>>>(h->src, d, first, rows, (uint32_t)per);
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

}  // namespace
}  // namespace mdj

extern "C" {

int mdj_stream_open(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key, uint32_t P,
                    int32_t how, const mdj_allocator *alloc, void *stream, mdj_stream **out, uint64_t *total_rows) {
  return mdj::stream_open(left, left_key, right, right_key, P, how, alloc, stream, out, total_rows);
}

int mdj_stream_emit(mdj_stream *s, uint64_t first_row, uint64_t nrows, const mdj_window *out) {
  return mdj::stream_emit(s, first_row, nrows, out);
}

int mdj_stream_next(mdj_stream *s, uint64_t max_rows, const mdj_window *out, uint64_t *first_row, uint64_t *nrows) {
  if (!s || !first_row || !nrows) return MDJ_ERR_INVALID_ARG;
  const uint64_t n = std::min(max_rows, s->total - s->cursor);
  const int rc = mdj::stream_emit(s, s->cursor, n, out);
  if (rc != MDJ_OK) return rc;
  *first_row = s->cursor;
  *nrows = n;
  s->cursor += n;
  return MDJ_OK;
}

uint64_t mdj_stream_rows(const mdj_stream *s) { return s ? s->total : 0; }

void mdj_stream_close(mdj_stream *s) {
  if (!s) return;
  delete s->ws;  // releases every buffer in stream order
  delete s;
}

}  // extern "C"
