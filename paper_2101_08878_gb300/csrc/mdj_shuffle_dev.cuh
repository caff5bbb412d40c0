// Device code of a shuffle pass shared by the partition and the fused
// join kernels of this library: the column set of a pass, the direct
// (unstaged) path of a tile, the register load of a tile and one staged tile
// (shuffle_one_tile).
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

// k_shuffle: NT threads, tiles of NT * kRPL rows, at most 2 * NT local
// buckets per tile, 1024 / NT blocks per SM.
constexpr int kShuffleNT = 512;
template <int NT>
__host__ __device__ constexpr uint32_t shuffle_tile() { return (uint32_t)NT * kRPL; }
template <int NT>
__host__ __device__ constexpr uint32_t shuffle_span() { return 2u * NT; }
template <int NT>
constexpr size_t shuffle_smem_bytes() {
  // stage (16-byte key/payload record, 8-byte row id/destination) per row;
  // two counter buffers and the packed (local start, destination base) per
  // local bucket; warp sums
  return (size_t)shuffle_tile<NT>() * (16 + 8) + (size_t)shuffle_span<NT>() * (4 + 4 + 8) + 32 * 4;
}

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
// scatter_direct uses.  PASS2 also fetches the tile's first and last key
// (its pass-1 bucket span).
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
    rv[c] = rid_in ? (ok ? rid_in[r] : 0u) : r;
  }
  if (PASS2) {
    kfirst = keys[row0];
    klast = keys[rend - 1];
  }
}

// One staged tile of a shuffle pass: rows [row0, rend) (at most NT * kRPL)
// whose columns are already in registers, local buckets [lb0, lb0 + Floc)
// (Floc <= 2 * NT).  Each (tile, bucket) run is reserved on cursors[lb0 + b];
// a row reserved at cursor value g lands at index g - dst_base of the
// destination columns.  With next_row0 < next_rend the registers receive the
// rows [next_row0, next_rend) once this tile is staged (before its write-out).
//
// Counters: buffer `parity` (all 2 * NT entries) must be zero on entry; the
// tile zeroes buffer 1 - parity while it stages, so consecutive tiles of one
// block alternate buffers and need no barrier between them: a warp may rank
// the next tile while others still write this one out.  Four block barriers
// per tile (after ranking, inside the scan, after the scan, after staging).
template <int NT, typename KeyT, bool PASS2, bool EXTRA>
__device__ __forceinline__ void shuffle_one_tile(unsigned char *smem, const KeyT *__restrict__ keys, uint32_t row0,
                                                 uint32_t rend, uint32_t lb0, uint32_t Floc, const BucketSpec &bs,
                                                 uint32_t *__restrict__ cursors, uint32_t dst_base, const ColMove &cm,
                                                 int reg_col, int pw, const uint32_t *__restrict__ rid_in,
                                                 uint32_t *__restrict__ rid_out, KeyT (&kv)[kRPL],
                                                 uint64_t (&pv)[kRPL], uint32_t (&rv)[kRPL], uint32_t next_row0,
                                                 uint32_t next_rend, KeyT &kfirst, KeyT &klast, int parity) {
  constexpr uint32_t kFTile = shuffle_tile<NT>(), kFSpan = shuffle_span<NT>();
  constexpr int kFT = NT, kNWarps = NT / 32;
  // stage: per row a 16-byte (key, payload) record and an 8-byte (row id,
  // destination) pair, so a row is scattered with two stores, not four
  ulonglong2 *rec = (ulonglong2 *)smem;
  uint2 *meta = (uint2 *)(smem + (size_t)kFTile * 16);
  uint32_t *cnt = (uint32_t *)(meta + kFTile) + (size_t)parity * kFSpan;
  uint32_t *cnt_next = (uint32_t *)(meta + kFTile) + (size_t)(1 - parity) * kFSpan;
  uint2 *lg = (uint2 *)((uint32_t *)(meta + kFTile) + 2 * kFSpan);  // (local start, destination base)
  uint32_t *wsum = (uint32_t *)(lg + kFSpan);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rows = rend - row0;
  const uint32_t wrow0 = row0 + warp * 32 * kRPL;

  // 1. rank of each row in its bucket (order among equal buckets: arbitrary)
  uint32_t pk[kRPL];
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    pk[c] = 0xFFFFFFFFu;
    if (wrow0 + c * 32 + lane < rend) {
      const uint64_t h = fmix64(key_bits(kv[c]));
      const uint32_t b = (PASS2 ? sub_bucket_of(h, bs) : bucket_of(h, bs)) - lb0;
      pk[c] = (b << 16) | atomicAdd(&cnt[b], 1u);
    }
  }
  __syncthreads();

  // 2. reserve every non-empty run (two buckets per thread), scan the counts:
  //    warp sums published once, each warp adds up the sums before it
  const uint32_t b0 = 2 * threadIdx.x, b1 = b0 + 1;
  const uint32_t c0 = b0 < Floc ? cnt[b0] : 0u, c1 = b1 < Floc ? cnt[b1] : 0u;
  const uint32_t g0 = c0 ? atomicAdd(&cursors[lb0 + b0], c0) : 0u;
  const uint32_t g1 = c1 ? atomicAdd(&cursors[lb0 + b1], c1) : 0u;
  const uint32_t v = c0 + c1;
  const uint32_t inc = warp_inclusive_scan(v);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int w = 0; w < kNWarps; w++)
    if (w < warp) before += wsum[w];
  const uint32_t ex = before + inc - v;
  if (b0 < Floc) lg[b0] = make_uint2(ex, g0 - dst_base);
  if (b1 < Floc) lg[b1] = make_uint2(ex + c0, g1 - dst_base);
  __syncthreads();

  // 3. stage the carried columns in bucket order, with each row's destination;
  //    clear the other counter buffer for the next tile
  for (uint32_t i = threadIdx.x; i < kFSpan; i += kFT) cnt_next[i] = 0;
  uint32_t lp[kRPL];
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    lp[c] = 0xFFFFFFFFu;
    if (pk[c] != 0xFFFFFFFFu) {
      const uint32_t b = pk[c] >> 16, rank = pk[c] & 0xFFFFu;
      const uint2 e = lg[b];
      lp[c] = e.x + rank;
      uint64_t kb = 0;
      memcpy(&kb, &kv[c], sizeof(KeyT));
      rec[lp[c]] = make_ulonglong2(kb, pv[c]);
      meta[lp[c]] = make_uint2(rv[c], e.y + rank);
    }
  }
  __syncthreads();
  if (!EXTRA && next_row0 < next_rend)
    shuffle_load<KeyT, PASS2>(keys, next_row0, next_rend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);

  // 4. write-out: consecutive threads store consecutive rows of one run
  KeyT *kdst = (KeyT *)cm.dst[cm.key_index];
  for (uint32_t i = threadIdx.x; i < rows; i += kFT) {
    const ulonglong2 r = rec[i];
    const uint2 m = meta[i];
    const uint32_t d = m.y;
    KeyT k;
    memcpy(&k, &r.x, sizeof(KeyT));
    kdst[d] = k;
    if (pw == 8) ((uint64_t *)cm.dst[reg_col])[d] = r.y;
    if (pw == 4) ((uint32_t *)cm.dst[reg_col])[d] = (uint32_t)r.y;
    if (rid_out) rid_out[d] = m.x;
  }

  // 5. any further column, one at a time through the payload half of the stage
  if (EXTRA) {
    for (int j = 0; j < cm.n; j++) {
      if (j == cm.key_index || j == reg_col) continue;
      const int w = cm.width[j];
      uint64_t val[kRPL];
#pragma unroll
      for (int c = 0; c < kRPL; c++) {
        const uint32_t r = wrow0 + c * 32 + lane;
        val[c] = 0;
        if (r < rend) val[c] = w == 8 ? ((const uint64_t *)cm.src[j])[r] : ((const uint32_t *)cm.src[j])[r];
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < kRPL; c++)
        if (lp[c] != 0xFFFFFFFFu) rec[lp[c]].y = val[c];
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < rows; i += kFT) {
        const uint32_t d = meta[i].y;
        if (w == 8)
          ((uint64_t *)cm.dst[j])[d] = rec[i].y;
        else
          ((uint32_t *)cm.dst[j])[d] = (uint32_t)rec[i].y;
      }
    }
    if (next_row0 < next_rend)
      shuffle_load<KeyT, PASS2>(keys, next_row0, next_rend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);
  }
}

// Clears both counter buffers of shuffle_one_tile (block-wide, no barrier).
template <int NT>
__device__ __forceinline__ void shuffle_clear_counters(unsigned char *smem) {
  uint32_t *cnt = (uint32_t *)(smem + (size_t)shuffle_tile<NT>() * 24);
  for (uint32_t i = threadIdx.x; i < 2 * shuffle_span<NT>(); i += NT) cnt[i] = 0;
}

}  // namespace
}  // namespace mdj
