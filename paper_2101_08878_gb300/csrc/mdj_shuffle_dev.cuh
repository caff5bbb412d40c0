// Device code of the merge's shuffle passes: the column set of a pass, the
// direct (unstaged) path of a tile, the register load of a tile and one
// staged tile (shuffle_tile).
#pragma once

#include <string.h>

#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr int kNW = 16;                     // warps per scatter block
constexpr int kRPL = 8;                     // rows per lane per tile
constexpr uint32_t kTile = kNW * 32 * kRPL; // 4096 rows per tile

struct ColMove {
  const void *src[MDJ_MAX_COLS];
  void *dst[MDJ_MAX_COLS];
  int32_t width[MDJ_MAX_COLS];
  int32_t n;
  int32_t key_index;
};

// Direct path of a pass-2 tile whose rows span too many buckets for shared
// memory (tiny or very skewed pass-1 buckets): warp-aggregated reservation,
// each row written straight to its slot.
template <typename KeyT>
__device__ void scatter_direct(const KeyT (&kv)[kRPL], uint32_t wrow0, uint32_t rend, const BucketSpec &bs,
                               uint32_t *__restrict__ cursors, const ColMove &cm,
                               const uint32_t *__restrict__ rid_in, uint32_t *__restrict__ rid_out) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int c = 0; c < kRPL; c++) {
    uint32_t r = wrow0 + c * 32 + lane;
    bool valid = r < rend;
    uint32_t fb = valid ? sub_bucket_of(fmix64(key_bits(kv[c])), bs) : 0xFFFFFFFFu;
    uint32_t peers = __match_any_sync(0xffffffffu, fb);
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&cursors[fb], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!valid) continue;
    uint32_t pos = base + __popc(peers & lanemask_lt());
    for (int j = 0; j < cm.n; j++) {
      if (cm.width[j] == 8) {
        uint64_t v = j == cm.key_index ? (uint64_t)kv[c] : ((const uint64_t *)cm.src[j])[r];
        ((uint64_t *)cm.dst[j])[pos] = v;
      } else {
        uint32_t v = j == cm.key_index ? (uint32_t)kv[c] : ((const uint32_t *)cm.src[j])[r];
        ((uint32_t *)cm.dst[j])[pos] = v;
      }
    }
    if (rid_out) rid_out[pos] = rid_in ? rid_in[r] : r;
  }
}

// ---------------------------------------------------------------- k_shuffle
//
// One block of kShNT threads per SM, tiles of kShTile rows (kRPL per thread),
// at most kShSpan local buckets per tile.  Shared memory per block:
//   rec    [kShTile]  16 bytes: key bits, first non-key column (bucket order)
//   meta   [kShTile]   4 bytes: pass 1: (row in tile << 10) | local bucket;
//                               pass 2: the row id (the local bucket is
//                               recomputed from the key at write-out: cheaper
//                               than staging it, measured)
//   cnt    [2][kShSpan] rank counters (two buffers, alternating tiles)
//   lst    [kShSpan]   local start of each bucket in the staged tile
//   gdelta [kShSpan]   destination - staged position, per bucket
//   wsum   [32]        warp sums of the count scan
constexpr int kShNT = 1024;
constexpr uint32_t kShTile = (uint32_t)kShNT * kRPL;  // 8192 rows
constexpr uint32_t kShSpan = kShNT;                   // one local bucket per thread
static_assert(kShSpan <= 1024, "pass-1 metadata keeps the local bucket in 10 bits");
static_assert(kShTile <= (1u << 22), "pass-1 metadata keeps the row in tile in 22 bits");

struct ShLayout {
  static constexpr size_t rec = 0;
  static constexpr size_t meta = rec + (size_t)kShTile * 16;
  static constexpr size_t cnt = meta + (size_t)kShTile * 4;
  static constexpr size_t lst = cnt + (size_t)2 * kShSpan * 4;
  static constexpr size_t gdelta = lst + (size_t)kShSpan * 4;
  static constexpr size_t wsum = gdelta + (size_t)kShSpan * 4;
  static constexpr size_t total = wsum + 32 * 4;
};

// scatter_direct for k_shuffle, reading the keys again from memory so that
// the caller's key registers need no addressable copy.
template <typename KeyT>
__device__ __noinline__ void shuffle_direct(const KeyT *__restrict__ keys, uint32_t wrow0, uint32_t rend,
                                            const BucketSpec &bs, uint32_t *__restrict__ cursors, const ColMove &cm,
                                            const uint32_t *__restrict__ rid_in, uint32_t *__restrict__ rid_out) {
  KeyT kv[kRPL];
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    const uint32_t r = wrow0 + c * 32 + (threadIdx.x & 31);
    kv[c] = r < rend ? keys[r] : KeyT(0);
  }
  scatter_direct<KeyT>(kv, wrow0, rend, bs, cursors, cm, rid_in, rid_out);
}

// Loads the carried columns of the tile of rows [row0, rend) into registers:
// warp w holds rows row0 + w*256 + c*32 + lane (c < kRPL), the layout
// scatter_direct uses.  PASS2 also loads the row ids and the tile's first
// and last key (its pass-1 bucket span).
template <typename KeyT, bool PASS2>
__device__ __forceinline__ void shuffle_load(const KeyT *__restrict__ keys, uint32_t row0, uint32_t rend,
                                             const ColMove &cm, int reg_col, int pw,
                                             const uint32_t *__restrict__ rid_in, KeyT (&kv)[kRPL],
                                             uint64_t (&pv)[kRPL], uint32_t (&rv)[kRPL], KeyT &kfirst,
                                             KeyT &klast) {
  const uint32_t wrow0 = row0 + (threadIdx.x >> 5) * 32 * kRPL;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    const uint32_t r = wrow0 + c * 32 + lane;
    const bool ok = r < rend;
    kv[c] = ok ? keys[r] : KeyT(0);
    pv[c] = 0;
    if (ok && pw == 8) pv[c] = ((const uint64_t *)cm.src[reg_col])[r];
    if (ok && pw == 4) pv[c] = ((const uint32_t *)cm.src[reg_col])[r];
    if (PASS2) rv[c] = ok ? rid_in[r] : 0u;
  }
  if (PASS2) {
    kfirst = keys[row0];
    klast = keys[rend - 1];
  }
}

// One staged tile: rows [row0, rend) (at most kShTile) whose columns are in
// registers, local buckets [lb0, lb0 + Floc) (Floc <= kShSpan).
//   1. rank: a row's rank in its bucket is a shared-memory atomicAdd;
//   2. counts: thread b scans bucket b's count into its local start and
//      reserves the run's destination with one atomicAdd on
//      cursors[lb0 + b], whose result is needed only at write-out (its
//      latency overlaps the scan and the staging);
//   3. stage: each row goes to its bucket-ordered slot (16-byte record and
//      4-byte meta); the other counter buffer is cleared for the next tile;
//   4. the next tile's columns load into the freed registers (unless EXTRA);
//   5. write-out: consecutive threads store consecutive rows of one run;
//   6. EXTRA: every further column, one at a time through the record's
//      payload half.
// Four block barriers per tile.
template <typename KeyT, bool PASS2, bool EXTRA>
__device__ __forceinline__ void shuffle_tile(unsigned char *smem, const KeyT *__restrict__ keys, uint32_t row0,
                                             uint32_t rend, uint32_t lb0, uint32_t Floc, const BucketSpec &bs,
                                             uint32_t *__restrict__ cursors, const ColMove &cm, int reg_col, int pw,
                                             const uint32_t *__restrict__ rid_in, uint32_t *__restrict__ rid_out,
                                             KeyT (&kv)[kRPL], uint64_t (&pv)[kRPL], uint32_t (&rv)[kRPL],
                                             uint32_t next_row0, uint32_t next_rend, KeyT &kfirst, KeyT &klast,
                                             int parity) {
  ulonglong2 *rec = (ulonglong2 *)(smem + ShLayout::rec);
  uint32_t *meta = (uint32_t *)(smem + ShLayout::meta);
  uint32_t *cnt = (uint32_t *)(smem + ShLayout::cnt) + (size_t)parity * kShSpan;
  uint32_t *cnt_next = (uint32_t *)(smem + ShLayout::cnt) + (size_t)(1 - parity) * kShSpan;
  uint32_t *lst = (uint32_t *)(smem + ShLayout::lst);
  uint32_t *gdelta = (uint32_t *)(smem + ShLayout::gdelta);  // modulo 2^32
  uint32_t *wsum = (uint32_t *)(smem + ShLayout::wsum);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rows = rend - row0;
  const uint32_t wl0 = (uint32_t)warp * 32 * kRPL;  // this warp's first row in the tile
  const uint32_t b = threadIdx.x;                    // the local bucket this thread scans


  // 1. rank
  uint32_t pk[kRPL];
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    pk[c] = 0xFFFFFFFFu;
    if (row0 + wl0 + c * 32 + lane < rend) {
      const uint64_t h = fmix64(key_bits(kv[c]));
      const uint32_t lb = (PASS2 ? sub_bucket_of(h, bs) : bucket_of(h, bs)) - lb0;
      pk[c] = (lb << 16) | atomicAdd(&cnt[lb], 1u);
    }
  }
  __syncthreads();

  // 2. counts: local starts by a block scan; the run's destination
  const uint32_t cb = b < Floc ? cnt[b] : 0u;
  const uint32_t gb = cb ? atomicAdd(&cursors[lb0 + b], cb) : 0u;
  const uint32_t inc = warp_inclusive_scan(cb);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int w = 0; w < kShNT / 32; w++)
    if (w < warp) before += wsum[w];
  const uint32_t ex = before + inc - cb;
  if (b < Floc) lst[b] = ex;
  __syncthreads();

  // 3. stage
  cnt_next[threadIdx.x] = 0;
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    if (pk[c] != 0xFFFFFFFFu) {
      const uint32_t lb = pk[c] >> 16, rank = pk[c] & 0xFFFFu;
      const uint32_t lp = lst[lb] + rank;
      uint64_t kb = 0;
      memcpy(&kb, &kv[c], sizeof(KeyT));
      rec[lp] = make_ulonglong2(kb, pv[c]);
      meta[lp] = PASS2 ? rv[c] : (((wl0 + c * 32 + lane) << 10) | lb);
    }
  }
  if (b < Floc) gdelta[b] = gb - ex;
  __syncthreads();
  if (!EXTRA && next_row0 < next_rend)
    shuffle_load<KeyT, PASS2>(keys, next_row0, next_rend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);

  // 5. write-out
  KeyT *kdst = (KeyT *)cm.dst[cm.key_index];
  for (uint32_t i = threadIdx.x; i < rows; i += kShNT) {
    const ulonglong2 r = rec[i];
    const uint32_t m = meta[i];
    KeyT k;
    memcpy(&k, &r.x, sizeof(KeyT));
    const uint32_t lb = PASS2 ? sub_bucket_of(fmix64(key_bits(k)), bs) - lb0 : (m & 0x3FFu);
    const uint32_t d = i + gdelta[lb];
    kdst[d] = k;
    if (pw == 8) ((uint64_t *)cm.dst[reg_col])[d] = r.y;
    if (pw == 4) ((uint32_t *)cm.dst[reg_col])[d] = (uint32_t)r.y;
    if (rid_out) rid_out[d] = PASS2 ? m : row0 + (m >> 10);
  }

  // 6. further columns, one at a time through the payload half of the stage
  if (EXTRA) {
    for (int j = 0; j < cm.n; j++) {
      if (j == cm.key_index || j == reg_col) continue;
      const int w = cm.width[j];
      uint64_t val[kRPL];
#pragma unroll
      for (int c = 0; c < kRPL; c++) {
        const uint32_t r = row0 + wl0 + c * 32 + lane;
        val[c] = 0;
        if (r < rend) val[c] = w == 8 ? ((const uint64_t *)cm.src[j])[r] : ((const uint32_t *)cm.src[j])[r];
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < kRPL; c++)
        if (pk[c] != 0xFFFFFFFFu) rec[lst[pk[c] >> 16] + (pk[c] & 0xFFFFu)].y = val[c];
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < rows; i += kShNT) {
        const ulonglong2 r = rec[i];
        KeyT k;
        memcpy(&k, &r.x, sizeof(KeyT));
        const uint32_t lb = PASS2 ? sub_bucket_of(fmix64(key_bits(k)), bs) - lb0 : (meta[i] & 0x3FFu);
        const uint32_t d = i + gdelta[lb];
        if (w == 8)
          ((uint64_t *)cm.dst[j])[d] = r.y;
        else
          ((uint32_t *)cm.dst[j])[d] = (uint32_t)r.y;
      }
    }
    if (next_row0 < next_rend)
      shuffle_load<KeyT, PASS2>(keys, next_row0, next_rend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);
  }
}

// Clears both counter buffers of shuffle_tile (block-wide, no barrier).
__device__ __forceinline__ void shuffle_clear_counters(unsigned char *smem) {
  uint32_t *cnt = (uint32_t *)(smem + ShLayout::cnt);
  for (uint32_t i = threadIdx.x; i < 2 * kShSpan; i += kShNT) cnt[i] = 0;
}

}  // namespace
}  // namespace mdj
