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
  return (size_t)shuffle_tile<NT>() * (8 + 8 + 4 + 4) + (size_t)shuffle_span<NT>() * 8 + 40 * 4;
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
template <int NT, typename KeyT, bool PASS2, bool EXTRA>
__device__ __forceinline__ void shuffle_one_tile(unsigned char *smem, const KeyT *__restrict__ keys, uint32_t row0,
                                                 uint32_t rend, uint32_t lb0, uint32_t Floc, const BucketSpec &bs,
                                                 uint32_t *__restrict__ cursors, uint32_t dst_base, const ColMove &cm,
                                                 int reg_col, int pw, const uint32_t *__restrict__ rid_in,
                                                 uint32_t *__restrict__ rid_out, KeyT (&kv)[kRPL],
                                                 uint64_t (&pv)[kRPL], uint32_t (&rv)[kRPL], uint32_t next_row0,
                                                 uint32_t next_rend, KeyT &kfirst, KeyT &klast) {
  constexpr uint32_t kFTile = shuffle_tile<NT>(), kFSpan = shuffle_span<NT>();
  constexpr int kFT = NT;
  KeyT *sk = (KeyT *)smem;
  uint64_t *sp = (uint64_t *)(smem + (size_t)kFTile * 8);
  uint32_t *sr = (uint32_t *)(smem + (size_t)kFTile * 16);
  uint32_t *dstmap = sr + kFTile;
  uint32_t *lstart = dstmap + kFTile;
  uint32_t *gbase = lstart + kFSpan;
  uint32_t *scratch = gbase + kFSpan;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rows = rend - row0;
  const uint32_t wrow0 = row0 + warp * 32 * kRPL;

    // 1. rank of each row in its bucket (order among equal buckets: arbitrary)
    uint32_t *cnt = lstart;
    for (uint32_t i = threadIdx.x; i < Floc; i += kFT) cnt[i] = 0;
    __syncthreads();
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

    // 2. reserve every non-empty run (two buckets per thread), scan the counts
    const uint32_t b0 = 2 * threadIdx.x, b1 = b0 + 1;
    const uint32_t c0 = b0 < Floc ? cnt[b0] : 0u, c1 = b1 < Floc ? cnt[b1] : 0u;
    const uint32_t g0 = c0 ? atomicAdd(&cursors[lb0 + b0], c0) : 0u;
    const uint32_t g1 = c1 ? atomicAdd(&cursors[lb0 + b1], c1) : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<uint32_t>(c0 + c1, scratch, &total);
    if (b0 < Floc) {
      lstart[b0] = ex;
      gbase[b0] = g0;
    }
    if (b1 < Floc) {
      lstart[b1] = ex + c0;
      gbase[b1] = g1;
    }
    __syncthreads();

    // 3. stage the carried columns in bucket order, with each row's destination
    uint32_t lp[kRPL];
#pragma unroll
    for (int c = 0; c < kRPL; c++) {
      lp[c] = 0xFFFFFFFFu;
      if (pk[c] != 0xFFFFFFFFu) {
        const uint32_t b = pk[c] >> 16, rank = pk[c] & 0xFFFFu;
        lp[c] = lstart[b] + rank;
        dstmap[lp[c]] = gbase[b] + rank - dst_base;
        sk[lp[c]] = kv[c];
        sp[lp[c]] = pv[c];
        sr[lp[c]] = rv[c];
      }
    }
    __syncthreads();
    if (!EXTRA && next_row0 < next_rend)
      shuffle_load<KeyT, PASS2>(keys, next_row0, next_rend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);

    // 4. write-out: consecutive threads store consecutive rows of one run
    KeyT *kdst = (KeyT *)cm.dst[cm.key_index];
    for (uint32_t i = threadIdx.x; i < rows; i += kFT) {
      const uint32_t d = dstmap[i];
      kdst[d] = sk[i];
      if (pw == 8) ((uint64_t *)cm.dst[reg_col])[d] = sp[i];
      if (pw == 4) ((uint32_t *)cm.dst[reg_col])[d] = (uint32_t)sp[i];
      if (rid_out) rid_out[d] = sr[i];
    }

    // 5. any further column, one at a time through the payload stage
    if (EXTRA) {
      for (int j = 0; j < cm.n; j++) {
        if (j == cm.key_index || j == reg_col) continue;
        const int w = cm.width[j];
        uint64_t v[kRPL];
#pragma unroll
        for (int c = 0; c < kRPL; c++) {
          const uint32_t r = wrow0 + c * 32 + lane;
          v[c] = 0;
          if (r < rend) v[c] = w == 8 ? ((const uint64_t *)cm.src[j])[r] : ((const uint32_t *)cm.src[j])[r];
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kRPL; c++)
          if (lp[c] != 0xFFFFFFFFu) sp[lp[c]] = v[c];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < rows; i += kFT) {
          const uint32_t d = dstmap[i];
          if (w == 8)
            ((uint64_t *)cm.dst[j])[d] = sp[i];
          else
            ((uint32_t *)cm.dst[j])[d] = (uint32_t)sp[i];
        }
      }
      if (next_row0 < next_rend)
        shuffle_load<KeyT, PASS2>(keys, next_row0, next_rend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);
    }
}

}  // namespace
}  // namespace mdj
