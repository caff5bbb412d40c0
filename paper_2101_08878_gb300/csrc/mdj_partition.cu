// The shuffle: hash partitioning of a table on the device.
//
// In the paper the shuffle moves partition p of every worker's table to worker
// p over MPI (Sec. IV-B, the Isend/Irecv coroutines; Sec. V-B "Shuffle: True").
// On one GPU that exchange is a scatter: partition p's region of the output
// plays worker p's receive buffer.  Kernels:
//
//   k_hist       per-tile bucket histogram (warp match_any + shared counters);
//                optionally also the per-sub-bucket totals of a two-level plan
//   (scan)       exclusive scan of the bucket-major (bucket, tile) histogram
//                matrix = the global base of every (bucket, tile) run
//   k_scatter    stable local counting sort of a tile in shared memory, then
//                every column leaves as coalesced runs (one per bucket)
//                RESERVE variant (pass 2): rows already grouped by pass-1
//                bucket are split further; each tile reserves its runs with
//                one atomicAdd per (tile, bucket) - not stable, coalesced
//
// Every kernel is bandwidth-bound: no tensor cores, integer hashing only.
#include <string.h>

#include "mdj_internal.cuh"
#include "mdj_shuffle_dev.cuh"

namespace mdj {
namespace {

constexpr int kHistThreads = 512;


__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

size_t scatter_smem_bytes(uint32_t FL) {
  return (size_t)kTile * 8 + (size_t)kTile * 4 + align16((size_t)kNW * FL * 2) + (size_t)FL * 8 + 40 * 4;
}

// ------------------------------------------------------------------ k_hist

template <typename KeyT>
__global__ void __launch_bounds__(kHistThreads) k_hist(const KeyT *__restrict__ keys, uint32_t n, BucketSpec bs,
                                                       uint32_t F, uint32_t tile, uint32_t ntiles,
                                                       uint32_t *__restrict__ hist, uint32_t *__restrict__ total2,
                                                       uint32_t nsub) {
  extern __shared__ uint32_t sh[];
  uint32_t *cnt = sh;
  uint32_t *cnt2 = sh + F;
  if (total2)
    for (uint32_t i = threadIdx.x; i < nsub; i += blockDim.x) cnt2[i] = 0;
  constexpr int U = 8;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (uint32_t b = threadIdx.x; b < F; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const uint32_t row0 = t * tile;
    const uint32_t end = min(row0 + tile, n);
    for (uint32_t base = row0; base < end; base += blockDim.x * U) {
      KeyT kv[U];
#pragma unroll
      for (int u = 0; u < U; u++) {
        uint32_t r = base + u * blockDim.x + threadIdx.x;
        kv[u] = r < end ? keys[r] : KeyT(0);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        uint32_t r = base + u * blockDim.x + threadIdx.x;
        if (r < end) {
          const uint64_t h = fmix64(key_bits(kv[u]));
          if (total2) {
            const uint32_t p = mod_p(h, bs), x = (uint32_t)(h >> 32);
            atomicAdd(&cnt[p * bs.S1 + __umulhi(x, bs.S1)], 1u);
            atomicAdd(&cnt2[p * bs.S + __umulhi(x, bs.S)], 1u);
          } else {
            atomicAdd(&cnt[bucket_of(h, bs)], 1u);
          }
        }
      }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < F; b += blockDim.x) hist[(size_t)b * ntiles + t] = cnt[b];
    __syncthreads();
  }
  if (total2) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nsub; i += blockDim.x)
      if (cnt2[i]) atomicAdd(&total2[i], cnt2[i]);
  }
}

// --------------------------------------------------------------- k_scatter

// SEG (with RESERVE): tiles come from `seg_tiles` and never cross a segment;
// a segment with P_seg partitions of S_seg sub-buckets each puts a row in its
// local bucket p * S_seg + floor(hi32(h) * S_seg / 2^32), p = h mod P_seg,
// among the segment's buckets starting at seg_base[seg] (a batch of
// independent merges; P_seg = 1 for a batch of joins).  seg_nb holds
// P_seg * S_seg, seg_P holds P_seg and seg_S holds S_seg.
template <typename KeyT, bool RESERVE, bool SEG>
__global__ void __launch_bounds__(kNW * 32, 2)
    k_scatter(const KeyT *__restrict__ keys, uint32_t n, BucketSpec bs, uint32_t F, uint32_t ntiles,
              const uint32_t *__restrict__ tile_base, uint32_t *__restrict__ cursors, uint32_t F2, ColMove cm,
              const uint32_t *__restrict__ rid_in, uint32_t *__restrict__ rid_out, const SegTile *__restrict__ seg_tiles,
              const uint32_t *__restrict__ seg_base, const uint32_t *__restrict__ seg_nb,
              const uint32_t *__restrict__ seg_P, const uint32_t *__restrict__ seg_S) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t FL = RESERVE ? kPass2SpanMax : F;
  uint64_t *stage64 = (uint64_t *)smem;
  uint32_t *stage32 = (uint32_t *)smem;
  uint32_t *dstmap = (uint32_t *)(smem + (size_t)kTile * 8);
  uint16_t *whist = (uint16_t *)(smem + (size_t)kTile * 12);
  uint32_t *lstart = (uint32_t *)(smem + (size_t)kTile * 12 + align16((size_t)kNW * FL * 2));
  uint32_t *gbase = lstart + FL;
  uint32_t *scratch = gbase + FL;

  const uint32_t t = blockIdx.x;
  SegTile td = {0, 0, 0};
  if (SEG) td = seg_tiles[t];
  const uint32_t row0 = SEG ? td.row0 : t * kTile;
  const uint32_t rows = SEG ? td.rows : min(kTile, n - row0);
  const uint32_t rend = row0 + rows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t wrow0 = row0 + warp * 32 * kRPL;

  KeyT kv[kRPL];
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    uint32_t r = wrow0 + c * 32 + lane;
    kv[c] = r < rend ? keys[r] : KeyT(0);
  }

  uint32_t Floc = F, lb0 = 0, Sseg = 0;
  BucketSpec sp = bs;
  if (SEG) {
    lb0 = seg_base[td.seg];
    Floc = seg_nb[td.seg];
    Sseg = seg_S[td.seg];
    sp = make_spec_dev(seg_P[td.seg]);
  } else if (RESERVE) {
    uint32_t b1f = sub_bucket_of(fmix64(key_bits(keys[row0])), bs) / F2;
    uint32_t b1l = sub_bucket_of(fmix64(key_bits(keys[rend - 1])), bs) / F2;
    lb0 = b1f * F2;
    Floc = (b1l - b1f + 1) * F2;
    if (Floc > kPass2SpanMax) {
      scatter_direct<KeyT>(kv, wrow0, rend, bs, cursors, cm, rid_in, rid_out);
      return;
    }
  }

  // 1. per-warp stable ranks: warp w owns rows [wrow0, wrow0 + 32*kRPL) and
  //    walks them in order, so (warp, rank) order is input order.
  for (uint32_t i = threadIdx.x; i < (kNW * Floc + 1) / 2; i += blockDim.x) ((uint32_t *)whist)[i] = 0;
  __syncthreads();
  uint32_t pk[kRPL];
  uint16_t *wh = whist + warp * Floc;
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    uint32_t r = wrow0 + c * 32 + lane;
    bool valid = r < rend;
    uint32_t b = 0xFFFFFFFFu;
    if (valid) {
      const uint64_t h = fmix64(key_bits(kv[c]));
      b = SEG ? mod_p(h, sp) * Sseg + __umulhi((uint32_t)(h >> 32), Sseg) : bucket_of(h, bs) - lb0;
    }
    uint32_t peers = __match_any_sync(0xffffffffu, b);
    uint32_t rank = __popc(peers & lanemask_lt());
    uint32_t old = valid ? wh[b] : 0u;
    __syncwarp();
    if (valid && rank == 0) wh[b] = (uint16_t)(old + __popc(peers));
    __syncwarp();
    pk[c] = (b << 16) | (old + rank);
  }
  __syncthreads();

  // 2. per bucket: warp offsets (exclusive over warps) and the tile count
  for (uint32_t b = threadIdx.x; b < Floc; b += blockDim.x) {
    uint32_t run = 0;
    for (int w = 0; w < kNW; w++) {
      uint32_t c = whist[w * Floc + b];
      whist[w * Floc + b] = (uint16_t)run;
      run += c;
    }
    lstart[b] = run;
  }
  __syncthreads();
  block_scan_array(lstart, Floc, scratch);

  // 3. global base of each bucket's run
  for (uint32_t b = threadIdx.x; b < Floc; b += blockDim.x) {
    if (!RESERVE) {
      gbase[b] = tile_base[(size_t)b * ntiles + t];
    } else {
      uint32_t e = b + 1 < Floc ? lstart[b + 1] : rows;
      uint32_t cnt = e - lstart[b];
      gbase[b] = cnt ? atomicAdd(&cursors[lb0 + b], cnt) : 0u;
    }
  }
  __syncthreads();

  // 4. sorted position of each row and its destination
  uint32_t lp[kRPL];
#pragma unroll
  for (int c = 0; c < kRPL; c++) {
    uint32_t r = wrow0 + c * 32 + lane;
    lp[c] = 0;
    if (r < rend) {
      uint32_t b = pk[c] >> 16, lr = pk[c] & 0xFFFFu;
      uint32_t wo = whist[warp * Floc + b];
      lp[c] = lstart[b] + wo + lr;
      dstmap[lp[c]] = gbase[b] + wo + lr;
    }
  }
  __syncthreads();

  // 5. every column: stage in sorted order, leave as runs
  for (int j = 0; j < cm.n; j++) {
    if (cm.width[j] == 8) {
      const uint64_t *src = (const uint64_t *)cm.src[j];
      uint64_t v[kRPL];
#pragma unroll
      for (int c = 0; c < kRPL; c++) {
        uint32_t r = wrow0 + c * 32 + lane;
        v[c] = j == cm.key_index ? (uint64_t)kv[c] : (r < rend ? src[r] : 0ull);
      }
#pragma unroll
      for (int c = 0; c < kRPL; c++)
        if (wrow0 + c * 32 + lane < rend) stage64[lp[c]] = v[c];
      __syncthreads();
      uint64_t *dst = (uint64_t *)cm.dst[j];
      for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) dst[dstmap[i]] = stage64[i];
      __syncthreads();
    } else {
      const uint32_t *src = (const uint32_t *)cm.src[j];
      uint32_t v[kRPL];
#pragma unroll
      for (int c = 0; c < kRPL; c++) {
        uint32_t r = wrow0 + c * 32 + lane;
        v[c] = j == cm.key_index ? (uint32_t)kv[c] : (r < rend ? src[r] : 0u);
      }
#pragma unroll
      for (int c = 0; c < kRPL; c++)
        if (wrow0 + c * 32 + lane < rend) stage32[lp[c]] = v[c];
      __syncthreads();
      uint32_t *dst = (uint32_t *)cm.dst[j];
      for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) dst[dstmap[i]] = stage32[i];
      __syncthreads();
    }
  }
  if (rid_out) {
    uint32_t v[kRPL];
#pragma unroll
    for (int c = 0; c < kRPL; c++) {
      uint32_t r = wrow0 + c * 32 + lane;
      v[c] = rid_in ? (r < rend ? rid_in[r] : 0u) : r;
    }
#pragma unroll
    for (int c = 0; c < kRPL; c++)
      if (wrow0 + c * 32 + lane < rend) stage32[lp[c]] = v[c];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < rows; i += blockDim.x) rid_out[dstmap[i]] = stage32[i];
  }
}

// ------------------------------------------------- unstable shuffle (merge)
//
// The merge needs every row in its sub-bucket, not the input order inside a
// bucket, so its shuffle drops stability (the public partition keeps it):
//
//   k_tot      rows per final sub-bucket (shared counters, flushed with one
//              global add per counter); the next chunk's keys load while the
//              current chunk is counted
//   k_shuffle  persistent blocks over tiles of 4096 rows: every column of a
//              row is loaded before the tile is processed (the next tile's
//              while the current one is written out), a row's rank in its
//              bucket is a shared-memory atomic, each (tile, bucket) run is
//              reserved with one global atomicAdd on the bucket's cursor, and
//              the columns are staged in bucket order and leave as runs;
//              three block barriers per tile.
//              PASS2: rows already grouped by pass-1 bucket (sub-bucket / F2)
//              are split into their sub-buckets, as in k_scatter's RESERVE.
// A pass-1 bucket holds the rows of sub-buckets [b * F2, (b + 1) * F2)
// (pass-1 bucket = sub-bucket / F2, see BucketSpec), so the scanned counts
// of the final sub-buckets also place the pass-1 buckets.

constexpr int kTotThreads = 1024;
constexpr int kTotU = 8;                        // keys per thread per chunk
template <typename KeyT>
__device__ __forceinline__ void tot_load(const KeyT *__restrict__ keys, uint64_t base, uint32_t n, KeyT (&v)[kTotU]) {
#pragma unroll
  for (int u = 0; u < kTotU; u++) {
    const uint64_t r = base + (uint64_t)u * kTotThreads + threadIdx.x;
    v[u] = r < n ? keys[r] : KeyT(0);
  }
}

// tot[sb] += rows of sub-bucket sb (spec bs, nsub = P * S).
template <typename KeyT>
__global__ void __launch_bounds__(kTotThreads) k_tot(const KeyT *__restrict__ keys, uint32_t n, BucketSpec bs,
                                                     uint32_t nsub, uint32_t *__restrict__ tot) {
  extern __shared__ uint32_t cnt[];
  for (uint32_t i = threadIdx.x; i < nsub; i += kTotThreads) cnt[i] = 0;
  __syncthreads();
  const uint64_t chunk = (uint64_t)kTotThreads * kTotU, stride = chunk * gridDim.x;
  uint64_t base = chunk * blockIdx.x;
  KeyT cur[kTotU], nxt[kTotU];
  tot_load<KeyT>(keys, base, n, cur);
  for (; base < n; base += stride) {
    tot_load<KeyT>(keys, base + stride, n, nxt);
#pragma unroll
    for (int u = 0; u < kTotU; u++) {
      const uint64_t r = base + (uint64_t)u * kTotThreads + threadIdx.x;
      if (r < n) atomicAdd(&cnt[sub_bucket_of(fmix64(key_bits(cur[u])), bs)], 1u);
      cur[u] = nxt[u];
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nsub; i += kTotThreads)
    if (cnt[i]) atomicAdd(&tot[i], cnt[i]);
}

// cur[b] = off[b * F2]: the first row of pass-1 bucket b
// Pass-1 cursors (the first row of every pass-1 bucket) and, for two-level
// plans, pass 2's: the first row of every sub-bucket (cur2 may be NULL).
__global__ void k_pass1_cursors(const uint32_t *__restrict__ off, uint32_t F1, uint32_t F2,
                                uint32_t *__restrict__ cur, uint32_t *__restrict__ cur2, uint32_t nsub) {
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < F1) cur[b] = off[(size_t)b * F2];
  if (cur2 && b < nsub) cur2[b] = off[b];
}

// Persistent: block b takes tiles b, b + gridDim.x, ...  Once a tile is
// staged its registers are free, so the next tile's columns are loaded into
// them before the staged tile is written out; the DRAM latency of the load
// overlaps the write-out.  `reg_col` is the non-key column carried in
// registers (-1: none); with EXTRA, the other non-key columns are loaded and
// staged one at a time after the first write-out (and the next tile's load
// waits until they are done).  Run destinations are reserved on `cursors`.
template <typename KeyT, bool PASS2, bool EXTRA>
__global__ void __launch_bounds__(kShNT, 1)
    k_shuffle(const KeyT *__restrict__ keys, uint32_t n, uint32_t ntiles, BucketSpec bs, uint32_t F, uint32_t F2,
              uint32_t *__restrict__ cursors, ColMove cm, int reg_col,
              const uint32_t *__restrict__ rid_in, uint32_t *__restrict__ rid_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int pw = reg_col >= 0 ? cm.width[reg_col] : 0;
  KeyT kv[kRPL];
  uint64_t pv[kRPL];
  uint32_t rv[kRPL];
  KeyT kfirst = KeyT(0), klast = KeyT(0);
  uint32_t t = blockIdx.x;
  const uint32_t tend = ntiles, tstep = gridDim.x;
  if (t >= tend) return;
  shuffle_load<KeyT, PASS2>(keys, t * kShTile, min(t * kShTile + kShTile, n), cm, reg_col, pw, rid_in, kv, pv, rv,
                            kfirst, klast);
  shuffle_clear_counters(smem);
  __syncthreads();
  int parity = 0;  // counter buffer of the next staged tile

  while (t < tend) {
    const uint32_t tn = t + tstep;
    const uint32_t row0 = t * kShTile, rend = min(row0 + kShTile, n);
    const uint32_t nrow0 = tn < tend ? tn * kShTile : 0u, nrend = tn < tend ? min(nrow0 + kShTile, n) : 0u;
    uint32_t lb0 = 0, Floc = F;
    if (PASS2) {
      const uint32_t b1f = sub_bucket_of(fmix64(key_bits(kfirst)), bs) / F2;
      const uint32_t b1l = sub_bucket_of(fmix64(key_bits(klast)), bs) / F2;
      lb0 = b1f * F2;
      Floc = (b1l - b1f + 1) * F2;
      if (Floc > kShSpan) {  // uniform over the block: no barrier inside
        shuffle_direct<KeyT>(keys, row0 + warp * 32 * kRPL, rend, bs, cursors, cm, rid_in, rid_out);
        if (nrow0 < nrend)
          shuffle_load<KeyT, PASS2>(keys, nrow0, nrend, cm, reg_col, pw, rid_in, kv, pv, rv, kfirst, klast);
        t = tn;
        continue;
      }
    }
    shuffle_tile<KeyT, PASS2, EXTRA>(smem, keys, row0, rend, lb0, Floc, bs, cursors, cm, reg_col, pw, rid_in,
                                     rid_out, kv, pv, rv, nrow0, nrend, kfirst, klast, parity);
    parity ^= 1;
    t = tn;
  }
}

// ------------------------------------------------------------ small kernels

__global__ void k_bucket_starts(const uint32_t *__restrict__ hist, uint32_t F, uint32_t ntiles, uint32_t n,
                                uint32_t *__restrict__ start) {
  uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < F) start[b] = ntiles ? hist[(size_t)b * ntiles] : 0u;
  if (b == F) start[F] = n;
}

// offsets of partition p in rows already sorted by p: first row with p' >= p
template <typename KeyT>
__global__ void k_offsets_bsearch(const KeyT *__restrict__ keys, uint32_t n, BucketSpec bs, uint32_t P,
                                  uint32_t *__restrict__ off) {
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > P) return;
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (mod_p(fmix64(key_bits(keys[mid])), bs) < p)
      lo = mid + 1;
    else
      hi = mid;
  }
  off[p] = lo;
}

__global__ void k_two(uint32_t *p, uint32_t a, uint32_t b) {
  p[0] = a;
  p[1] = b;
}

__global__ void k_u32_to_i64(const uint32_t *__restrict__ a, int64_t *__restrict__ b, uint32_t n) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (int64_t)a[i];
}

// ------------------------------------------------------------- host passes

int hist_grid(size_t smem) {
  int per_sm = 1;
  if (smem <= 48 * 1024) per_sm = 4;
  else if (smem <= 100 * 1024) per_sm = 2;
  return num_sms() * per_sm;
}

template <typename KeyT>
int set_smem_attrs() {
  static PerDeviceOnce once;
  return once_per_device(once, [] {
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_scatter<KeyT, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)scatter_smem_bytes(kMaxFanout)));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_scatter<KeyT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)scatter_smem_bytes(kPass2SpanMax)));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_scatter<KeyT, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)scatter_smem_bytes(kPass2SpanMax)));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_hist<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((kMaxFanout + kMaxSubBuckets) * 4)));
    return (int)MDJ_OK;
  });
}

// One stable scatter pass over n rows into F <= kMaxFanout buckets.  If
// `start` is given it receives the F+1 bucket start positions.  If `total2` is
// given, the pass also counts rows per sub-bucket (nsub entries, zeroed by the
// caller) for a following RESERVE pass.
template <typename KeyT>
int stable_pass(Workspace &ws, const KeyT *keys, uint32_t n, const BucketSpec &bs, uint32_t F, const ColMove &cm,
                const uint32_t *rid_in, uint32_t *rid_out, uint32_t *start, uint32_t *total2, uint32_t nsub) {
  cudaStream_t s = ws.stream();
  MDJ_TRY(set_smem_attrs<KeyT>());
  const uint32_t tile = kTile;
  const uint32_t ntiles = (n + tile - 1) / tile;
  if (ntiles == 0) {
    if (start) MDJ_CUDA_TRY(cudaMemsetAsync(start, 0, (size_t)(F + 1) * 4, s));
    return MDJ_OK;
  }
  uint32_t *hist = (uint32_t *)ws.get((size_t)F * ntiles * 4);
  if (!hist) return MDJ_ERR_OOM;
  const size_t hsmem = (size_t)(F + (total2 ? nsub : 0)) * 4;
  {
    TraceScope tr("hist", s);
    const unsigned hgrid = (unsigned)(ntiles < (uint32_t)hist_grid(hsmem) ? ntiles : (uint32_t)hist_grid(hsmem));
    k_hist<KeyT><<<hgrid, kHistThreads, hsmem, s>>>(keys, n, bs, F, tile, ntiles, hist, total2, nsub);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u32(ws, hist, hist, (size_t)F * ntiles));
  if (start) {
    TraceScope tr("bucket_starts", s);
    k_bucket_starts<<<(F + 1 + 255) / 256, 256, 0, s>>>(hist, F, ntiles, n, start);
  }
  MDJ_LAUNCH_CHECK();
  {
    TraceScope tr("scatter_stable", s);
    k_scatter<KeyT, false, false><<<ntiles, kNW * 32, scatter_smem_bytes(F), s>>>(
        keys, n, bs, F, ntiles, hist, nullptr, 1, cm, rid_in, rid_out, nullptr, nullptr, nullptr, nullptr, nullptr);
  }
  MDJ_LAUNCH_CHECK();
  ws.give_back(hist);
  return MDJ_OK;
}

// Pass 2 of a two-level plan: rows grouped by pass-1 bucket (sb / F2) are
// split into final sub-buckets sb with atomic run reservation.
template <typename KeyT>
int reserve_pass(Workspace &ws, const KeyT *keys, uint32_t n, const BucketSpec &bs_sub, uint32_t F2,
                 uint32_t *cursors, const ColMove &cm, const uint32_t *rid_in, uint32_t *rid_out) {
  cudaStream_t s = ws.stream();
  MDJ_TRY(set_smem_attrs<KeyT>());
  const uint32_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles == 0) return MDJ_OK;
  {
    TraceScope tr("scatter_reserve", s);
    k_scatter<KeyT, true, false><<<ntiles, kNW * 32, scatter_smem_bytes(kPass2SpanMax), s>>>(
        keys, n, bs_sub, 0, ntiles, nullptr, cursors, F2, cm, rid_in, rid_out, nullptr, nullptr, nullptr, nullptr,
        nullptr);
  }
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

// Buffers of one partitioned copy of a table: every column and the row ids
// carved from one allocation (each part 256-byte aligned).
struct TableBufs {
  void *cols[MDJ_MAX_COLS];
  uint32_t *rid;
  void *block;
};

int alloc_table_bufs(Workspace &ws, const mdj_table *t, TableBufs *b, bool with_rid) {
  const size_t n = t->nrows;
  auto part = [](size_t bytes) { return (bytes + 255) & ~(size_t)255; };
  size_t total = with_rid ? part(n * 4) : 0;
  for (int j = 0; j < t->ncols; j++) total += part(n * dtype_width(t->cols[j].dtype));
  b->block = ws.get(total ? total : 256);
  if (!b->block) return MDJ_ERR_OOM;
  unsigned char *p = (unsigned char *)b->block;
  for (int j = 0; j < t->ncols; j++) {
    b->cols[j] = p;
    p += part(n * dtype_width(t->cols[j].dtype));
  }
  b->rid = with_rid ? (uint32_t *)p : nullptr;
  return MDJ_OK;
}

void release_table_bufs(Workspace &ws, const mdj_table *, TableBufs *b) { ws.give_back(b->block); }

ColMove make_move(const mdj_table *t, int32_t key_col, const void *const *src, void *const *dst) {
  ColMove cm;
  memset(&cm, 0, sizeof cm);
  cm.n = t->ncols;
  cm.key_index = key_col;
  for (int j = 0; j < t->ncols; j++) {
    cm.src[j] = src[j];
    cm.dst[j] = dst[j];
    cm.width[j] = dtype_width(t->cols[j].dtype);
  }
  return cm;
}

// ------------------------------------------------ unstable shuffle (host)

// MDJ_STABLE_SHUFFLE=1 makes the merge use the stable passes (for comparison).
bool fast_shuffle_enabled() {
  const char *e = getenv("MDJ_STABLE_SHUFFLE");
  return !(e && e[0] == '1');
}

template <typename KeyT>
int set_shuffle_attrs() {
  static PerDeviceOnce once;
  return once_per_device(once, [] {
    const int sm = (int)ShLayout::total;
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_shuffle<KeyT, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_shuffle<KeyT, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_shuffle<KeyT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_shuffle<KeyT, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    MDJ_CUDA_TRY(cudaFuncSetAttribute(k_tot<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(kMaxSubBuckets * 4)));
    return (int)MDJ_OK;
  });
}

template <typename KeyT>
auto shuffle_kernel(bool pass2, bool extra) {
  if (pass2) return extra ? k_shuffle<KeyT, true, true> : k_shuffle<KeyT, true, false>;
  return extra ? k_shuffle<KeyT, false, true> : k_shuffle<KeyT, false, false>;
}

// One unstable shuffle pass (see k_shuffle) of n rows, one block per SM, with
// run cursors `cur` (pass 1: one per pass-1 bucket; pass 2: one per sub-bucket).
template <typename KeyT, bool PASS2>
int shuffle_pass(Workspace &ws, const KeyT *keys, uint32_t n, const BucketSpec &bs, uint32_t F, uint32_t F2,
                 uint32_t *cur, const ColMove &cm, const uint32_t *rid_in, uint32_t *rid_out) {
  const uint32_t ntiles = (n + kShTile - 1) / kShTile;
  if (ntiles == 0) return MDJ_OK;
  int reg_col = -1;
  for (int j = 0; j < cm.n && reg_col < 0; j++)
    if (j != cm.key_index) reg_col = j;
  const uint32_t sms = (uint32_t)num_sms();
  const uint32_t grid = ntiles < sms ? ntiles : sms;
  TraceScope tr(PASS2 ? "shuffle_pass2" : "shuffle_pass1", ws.stream());
  shuffle_kernel<KeyT>(PASS2, cm.n > 2)<<<grid, kShNT, ShLayout::total, ws.stream()>>>(keys, n, ntiles, bs, F, F2, cur,
                                                                                       cm, reg_col, rid_in, rid_out);
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

// The merge's partition of one side with the unstable passes, first half:
// count the final sub-buckets, scan them into `off`, then the only pass
// (F2 == 1) or pass 1 (two-level plans) into freshly allocated `out`.
// cur2 (two-level plans): pass 2's cursors, allocated here and filled from
// the offsets by the same kernel as pass 1's.
template <typename KeyT>
int shuffle_count_pass1_t(Workspace &ws, const mdj_table *t, int32_t key_col, const Plan &plan, uint32_t *off,
                          TableBufs *out, uint32_t **cur2 = nullptr) {
  cudaStream_t s = ws.stream();
  MDJ_TRY(set_shuffle_attrs<KeyT>());
  const uint32_t n = (uint32_t)t->nrows;
  const uint32_t nsub = plan.nbuckets;
  const uint32_t F1 = plan.F2 == 1 ? nsub : plan.F1;
  const void *src[MDJ_MAX_COLS];
  for (int j = 0; j < t->ncols; j++) src[j] = t->cols[j].data;
  const KeyT *keys = (const KeyT *)src[key_col];
  const BucketSpec sub = make_spec(plan.P, plan.S, 1);

  MDJ_CUDA_TRY(cudaMemsetAsync(off, 0, (size_t)(nsub + 1) * 4, s));
  MDJ_TRY(alloc_table_bufs(ws, t, out, true));
  if (n == 0) return MDJ_OK;
  uint32_t *cur = (uint32_t *)ws.get((size_t)(nsub + 1) * 4);
  if (!cur) return MDJ_ERR_OOM;
  if (cur2 && !(*cur2 = (uint32_t *)ws.get((size_t)(nsub + 1) * 4))) return MDJ_ERR_OOM;
  {
    const size_t smem = (size_t)nsub * 4;
    int per_sm = 0;
    MDJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tot<KeyT>, kTotThreads, smem));
    if (per_sm < 1) per_sm = 1;
    const uint64_t chunks = ((uint64_t)n + (uint64_t)kTotThreads * kTotU - 1) / ((uint64_t)kTotThreads * kTotU);
    const uint64_t full = (uint64_t)num_sms() * per_sm;
    const unsigned grid = (unsigned)(chunks < full ? chunks : full);
    TraceScope tr("hist", s);
    k_tot<KeyT><<<grid, kTotThreads, smem, s>>>(keys, n, sub, nsub, off);
  }
  MDJ_LAUNCH_CHECK();
  MDJ_TRY(exclusive_scan_u32(ws, off, off, (size_t)nsub + 1));
  {
    // pass-1 cursors: the first row of every pass-1 bucket
    TraceScope tr("pass1_cursors", s);
    const uint32_t nk = cur2 ? (F1 > nsub ? F1 : nsub) : F1;
    k_pass1_cursors<<<(nk + 255) / 256, 256, 0, s>>>(off, F1, plan.F2, cur, cur2 ? *cur2 : nullptr, nsub);
  }
  MDJ_LAUNCH_CHECK();
  ColMove cm = make_move(t, key_col, src, out->cols);
  const BucketSpec spec1 = plan.F2 == 1 ? sub : make_spec(plan.P, plan.S, plan.F2);
  MDJ_TRY((shuffle_pass<KeyT, false>(ws, keys, n, spec1, F1, plan.F2, cur, cm, nullptr, out->rid)));
  ws.give_back(cur);
  return MDJ_OK;
}

// Second half of a two-level plan: pass 2 from the pass-1 copy `p1` into
// freshly allocated `fin` (sub-bucket offsets `off` from the first half).
template <typename KeyT>
int shuffle_pass2_t(Workspace &ws, const mdj_table *t, int32_t key_col, const Plan &plan, uint32_t *cur,
                    const TableBufs &p1, TableBufs *fin) {
  const uint32_t n = (uint32_t)t->nrows;
  MDJ_TRY(alloc_table_bufs(ws, t, fin, true));
  if (n == 0) return MDJ_OK;
  ColMove cm2 = make_move(t, key_col, p1.cols, fin->cols);
  MDJ_TRY((shuffle_pass<KeyT, true>(ws, (const KeyT *)p1.cols[key_col], n, make_spec(plan.P, plan.S, 1), 0, plan.F2,
                                    cur, cm2, p1.rid, fin->rid)));
  ws.give_back(cur);
  return MDJ_OK;
}

template <typename KeyT>
int shuffle_side_t(Workspace &ws, const mdj_table *t, int32_t key_col, const Plan &plan, uint32_t *off,
                   TableBufs *fin) {
  if (plan.F2 == 1) return shuffle_count_pass1_t<KeyT>(ws, t, key_col, plan, off, fin);
  TableBufs p1;
  uint32_t *cur2 = nullptr;
  MDJ_TRY(shuffle_count_pass1_t<KeyT>(ws, t, key_col, plan, off, &p1, &cur2));
  MDJ_TRY(shuffle_pass2_t<KeyT>(ws, t, key_col, plan, cur2, p1, fin));
  release_table_bufs(ws, t, &p1);
  return MDJ_OK;
}

// Stable partition by p with P > kMaxFanout: two stable LSD digit passes
// (p mod 1024, then p / 1024), which sort stably by p.  Writes into `dst`
// buffers; `off` (device u32[P+1]) receives the partition offsets.
template <typename KeyT>
int lsd_partition(Workspace &ws, const mdj_table *t, int32_t key_col, uint32_t P, void *const *dst_cols,
                  uint32_t *dst_rid, uint32_t *off) {
  const uint32_t n = (uint32_t)t->nrows;
  const void *src[MDJ_MAX_COLS];
  for (int j = 0; j < t->ncols; j++) src[j] = t->cols[j].data;
  TableBufs mid;
  MDJ_TRY(alloc_table_bufs(ws, t, &mid, true));
  const uint32_t d0 = kMaxFanout, d1 = (P + kMaxFanout - 1) / kMaxFanout;
  ColMove cm0 = make_move(t, key_col, src, mid.cols);
  MDJ_TRY(stable_pass<KeyT>(ws, (const KeyT *)src[key_col], n, make_digit_spec(P, 1, d0), d0, cm0, nullptr, mid.rid,
                            nullptr, nullptr, 0));
  ColMove cm1 = make_move(t, key_col, mid.cols, dst_cols);
  MDJ_TRY(stable_pass<KeyT>(ws, (const KeyT *)mid.cols[key_col], n, make_digit_spec(P, d0, d1), d1, cm1, mid.rid,
                            dst_rid, nullptr, nullptr, 0));
  release_table_bufs(ws, t, &mid);
  {
    TraceScope tr("offsets_bsearch", ws.stream());
    k_offsets_bsearch<KeyT><<<(P + 1 + 255) / 256, 256, 0, ws.stream()>>>((const KeyT *)dst_cols[key_col], n,
                                                                         make_spec(P, 1, 1), P, off);
  }
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

template <typename KeyT>
int stable_partition_t(Workspace &ws, const mdj_table *t, int32_t key_col, uint32_t P, void *const *out_cols,
                       uint32_t *out_rid, int64_t *out_offsets) {
  cudaStream_t s = ws.stream();
  const uint32_t n = (uint32_t)t->nrows;
  uint32_t *off = (uint32_t *)ws.get((size_t)(P + 1) * 4);
  if (!off) return MDJ_ERR_OOM;
  uint32_t *rid = out_rid;
  if (!rid && n > 0) {
    // row ids are needed by the second LSD pass only; a single pass can skip them
    if (P > kMaxFanout) {
      rid = (uint32_t *)ws.get((size_t)n * 4);
      if (!rid) return MDJ_ERR_OOM;
    }
  }
  if (P <= kMaxFanout) {
    const void *src[MDJ_MAX_COLS];
    for (int j = 0; j < t->ncols; j++) src[j] = t->cols[j].data;
    ColMove cm = make_move(t, key_col, src, out_cols);
    MDJ_TRY(stable_pass<KeyT>(ws, (const KeyT *)src[key_col], n, make_spec(P, 1, 1), P, cm, nullptr, out_rid, off,
                              nullptr, 0));
  } else {
    if (n == 0) {
      MDJ_CUDA_TRY(cudaMemsetAsync(off, 0, (size_t)(P + 1) * 4, s));
    } else {
      MDJ_TRY(lsd_partition<KeyT>(ws, t, key_col, P, out_cols, rid, off));
    }
  }
  {
    TraceScope tr("offsets_i64", s);
    k_u32_to_i64<<<(P + 1 + 255) / 256, 256, 0, s>>>(off, out_offsets, P + 1);
  }
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

template <typename KeyT>
int partition_side_t(Workspace &ws, const mdj_table *t, int32_t key_col, const Plan &plan, Side *out) {
  cudaStream_t s = ws.stream();
  const uint32_t n = (uint32_t)t->nrows;
  const void *src[MDJ_MAX_COLS];
  for (int j = 0; j < t->ncols; j++) src[j] = t->cols[j].data;

  uint32_t *off = (uint32_t *)ws.get((size_t)(plan.nbuckets + 1) * 4);
  if (!off) return MDJ_ERR_OOM;
  TableBufs fin;
  fin.rid = nullptr;
  const void *key = src[key_col];
  const void *const *cols = src;
  const uint32_t *rid = nullptr;

  if (!plan.partition) {
    TraceScope tr("offsets_whole", s);
    k_two<<<1, 1, 0, s>>>(off, 0u, n);
    MDJ_LAUNCH_CHECK();
  } else if (!plan.lsd && !plan.stable && fast_shuffle_enabled()) {
    MDJ_TRY(shuffle_side_t<KeyT>(ws, t, key_col, plan, off, &fin));
    key = fin.cols[key_col];
    cols = fin.cols;
    rid = fin.rid;
  } else if (plan.lsd) {
    MDJ_TRY(alloc_table_bufs(ws, t, &fin, true));
    MDJ_TRY(lsd_partition<KeyT>(ws, t, key_col, plan.P, fin.cols, fin.rid, off));
    key = fin.cols[key_col];
    cols = fin.cols;
    rid = fin.rid;
  } else if (plan.F2 == 1) {
    MDJ_TRY(alloc_table_bufs(ws, t, &fin, true));
    ColMove cm = make_move(t, key_col, src, fin.cols);
    MDJ_TRY(stable_pass<KeyT>(ws, (const KeyT *)key, n, make_spec(plan.P, plan.S, 1), plan.nbuckets, cm, nullptr,
                              fin.rid, off, nullptr, 0));
    key = fin.cols[key_col];
    cols = fin.cols;
    rid = fin.rid;
  } else {
    // pass 1: F1 = P*S/F2 stable buckets, counting the final sub-buckets too
    uint32_t *cur = (uint32_t *)ws.get((size_t)(plan.nbuckets + 1) * 4);
    if (!cur) return MDJ_ERR_OOM;
    MDJ_CUDA_TRY(cudaMemsetAsync(off, 0, (size_t)(plan.nbuckets + 1) * 4, s));
    TableBufs p1;
    MDJ_TRY(alloc_table_bufs(ws, t, &p1, true));
    ColMove cm1 = make_move(t, key_col, src, p1.cols);
    MDJ_TRY(stable_pass<KeyT>(ws, (const KeyT *)key, n, make_spec(plan.P, plan.S, plan.F2), plan.F1, cm1, nullptr,
                              p1.rid, nullptr, off, plan.nbuckets));
    MDJ_TRY(exclusive_scan_u32(ws, off, off, plan.nbuckets + 1));
    MDJ_CUDA_TRY(cudaMemcpyAsync(cur, off, (size_t)plan.nbuckets * 4, cudaMemcpyDeviceToDevice, s));
    // pass 2
    MDJ_TRY(alloc_table_bufs(ws, t, &fin, true));
    ColMove cm2 = make_move(t, key_col, p1.cols, fin.cols);
    MDJ_TRY(reserve_pass<KeyT>(ws, (const KeyT *)p1.cols[key_col], n, make_spec(plan.P, plan.S, 1), plan.F2, cur,
                               cm2, p1.rid, fin.rid));
    release_table_bufs(ws, t, &p1);
    ws.give_back(cur);
    key = fin.cols[key_col];
    cols = fin.cols;
    rid = fin.rid;
  }

  out->key = key;
  out->key_dtype = t->cols[key_col].dtype;
  out->ncols = 0;
  for (int j = 0; j < t->ncols; j++) {
    if (j == key_col) continue;
    out->cols[out->ncols] = cols[j];
    out->widths[out->ncols] = dtype_width(t->cols[j].dtype);
    out->dtypes[out->ncols] = t->cols[j].dtype;
    out->ncols++;
  }
  out->rid = rid;
  out->off = off;
  out->nrows = n;
  return MDJ_OK;
}

}  // namespace

Plan make_plan(uint64_t n_build, uint32_t P, uint32_t cap, bool force_partition) {
  Plan pl;
  pl.P = P;
  pl.cap = cap;
  // target mean build rows per sub-bucket: ~85% of a table, so that hash
  // variance rarely overflows one table
  const uint64_t target = (uint64_t)cap * 85 / 100;
  uint64_t need = (n_build + target - 1) / target;
  if (need < 1) need = 1;
  if (P > kMaxFanout) {
    pl.lsd = true;
    pl.S = 1;
    pl.nbuckets = P;
    pl.F1 = P;
    pl.F2 = 1;
    return pl;
  }
  if (P == 1 && need == 1 && !force_partition) {
    pl.partition = false;
    pl.S = 1;
    pl.nbuckets = 1;
    return pl;
  }
  uint64_t S = (need + P - 1) / P;
  if (S < 1) S = 1;
  if ((uint64_t)P * S <= kMaxFanout) {
    pl.S = (uint32_t)S;
    pl.F1 = P * pl.S;
    pl.F2 = 1;
    pl.nbuckets = pl.F1;
    return pl;
  }
  const uint32_t fan = kMergeFanout;
  uint32_t S1 = fan / P;
  if (S1 < 1) S1 = 1;
  uint64_t F2 = (S + S1 - 1) / S1;
  uint64_t max_f2 = kMaxSubBuckets / ((uint64_t)P * S1);
  if (F2 > max_f2) F2 = max_f2;  // larger inputs: sub-buckets split into several tables
  if (F2 > kPass2SpanMax / 2) F2 = kPass2SpanMax / 2;
  if (F2 < 1) F2 = 1;
  pl.F2 = (uint32_t)F2;
  pl.S = S1 * pl.F2;
  pl.F1 = P * S1;
  pl.nbuckets = P * pl.S;
  return pl;
}

int partition_side(Workspace &ws, const mdj_table *t, int32_t key_col, const Plan &plan, Side *out) {
  if (t->cols[key_col].dtype == MDJ_I64) return partition_side_t<int64_t>(ws, t, key_col, plan, out);
  return partition_side_t<int32_t>(ws, t, key_col, plan, out);
}

namespace {
void fill_side(const mdj_table *t, int32_t key_col, const TableBufs &b, uint32_t *off, Side *out) {
  out->key = b.cols[key_col];
  out->key_dtype = t->cols[key_col].dtype;
  out->ncols = 0;
  for (int j = 0; j < t->ncols; j++) {
    if (j == key_col) continue;
    out->cols[out->ncols] = b.cols[j];
    out->widths[out->ncols] = dtype_width(t->cols[j].dtype);
    out->dtypes[out->ncols] = t->cols[j].dtype;
    out->ncols++;
  }
  out->rid = b.rid;
  out->off = off;
  out->nrows = t->nrows;
}
}  // namespace

int stable_partition(Workspace &ws, const mdj_table *t, int32_t key_col, uint32_t P, void *const *out_cols,
                     uint32_t *out_rid, int64_t *out_offsets) {
  if (t->cols[key_col].dtype == MDJ_I64)
    return stable_partition_t<int64_t>(ws, t, key_col, P, out_cols, out_rid, out_offsets);
  return stable_partition_t<int32_t>(ws, t, key_col, P, out_cols, out_rid, out_offsets);
}

}  // namespace mdj

namespace mdj {
namespace {

template <typename KeyT>
int stable_partition_scratch_t(const mdj_table *t, int32_t key_col, uint32_t P, void *const *out_cols,
                               uint32_t *out_rid, int64_t *out_offsets, uint32_t *scratch, size_t scratch_words,
                               cudaStream_t s) {
  const uint32_t n = (uint32_t)t->nrows, F = P;
  const uint32_t ntiles = (n + kTile - 1) / kTile;
  const size_t nhist = (size_t)F * ntiles;
  if (stable_partition_scratch_words(n, P) > scratch_words) return MDJ_ERR_TOO_LARGE;
  MDJ_TRY(set_smem_attrs<KeyT>());
  uint32_t *hist = scratch;
  uint32_t *sums = hist + nhist;
  uint32_t *start = sums + scan_scratch_words(nhist);
  if (ntiles == 0) {
    MDJ_CUDA_TRY(cudaMemsetAsync(start, 0, (size_t)(F + 1) * 4, s));
  } else {
    const BucketSpec bs = make_spec(P, 1, 1);
    const size_t hsmem = (size_t)F * 4;
    const unsigned hgrid = (unsigned)(ntiles < (uint32_t)hist_grid(hsmem) ? ntiles : (uint32_t)hist_grid(hsmem));
    k_hist<KeyT><<<hgrid, kHistThreads, hsmem, s>>>((const KeyT *)t->cols[key_col].data, n, bs, F, kTile, ntiles,
                                                   hist, nullptr, 0);
    MDJ_LAUNCH_CHECK();
    MDJ_TRY(exclusive_scan_u32_scratch(hist, hist, nhist, sums, s));
    k_bucket_starts<<<(F + 1 + 255) / 256, 256, 0, s>>>(hist, F, ntiles, n, start);
    MDJ_LAUNCH_CHECK();
    const void *src[MDJ_MAX_COLS];
    for (int j = 0; j < t->ncols; j++) src[j] = t->cols[j].data;
    ColMove cm = make_move(t, key_col, src, out_cols);
    k_scatter<KeyT, false, false><<<ntiles, kNW * 32, scatter_smem_bytes(F), s>>>(
        (const KeyT *)src[key_col], n, bs, F, ntiles, hist, nullptr, 1, cm, nullptr, out_rid, nullptr, nullptr,
        nullptr, nullptr, nullptr);
    MDJ_LAUNCH_CHECK();
  }
  k_u32_to_i64<<<(P + 1 + 255) / 256, 256, 0, s>>>(start, out_offsets, P + 1);
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

}  // namespace

size_t stable_partition_scratch_words(uint64_t n, uint32_t P) {
  const uint64_t nhist = (uint64_t)P * ((n + kTile - 1) / kTile);
  return (size_t)(nhist + scan_scratch_words(nhist) + P + 1);
}

int stable_partition_scratch(const mdj_table *t, int32_t key_col, uint32_t P, void *const *out_cols,
                             uint32_t *out_rid, int64_t *out_offsets, uint32_t *scratch, size_t scratch_words,
                             cudaStream_t s) {
  if (t->cols[key_col].dtype == MDJ_I64)
    return stable_partition_scratch_t<int64_t>(t, key_col, P, out_cols, out_rid, out_offsets, scratch,
                                               scratch_words, s);
  return stable_partition_scratch_t<int32_t>(t, key_col, P, out_cols, out_rid, out_offsets, scratch, scratch_words,
                                             s);
}

}  // namespace mdj

// ------------------------------------------------- segmented (batched) form
namespace mdj {
namespace {

// Per tile: counts of its segment's buckets, added into totals[seg_base + b].
template <typename KeyT>
__global__ void __launch_bounds__(kHistThreads) k_seg_hist(const KeyT *__restrict__ keys,
                                                           const SegTile *__restrict__ tiles,
                                                           const uint32_t *__restrict__ seg_base,
                                                           const uint32_t *__restrict__ seg_nb,
                                                           const uint32_t *__restrict__ seg_P,
                                                           const uint32_t *__restrict__ seg_S,
                                                           uint32_t *__restrict__ totals) {
  extern __shared__ uint32_t cnt[];
  const SegTile td = tiles[blockIdx.x];
  const uint32_t NB = seg_nb[td.seg], B = seg_base[td.seg], S = seg_S[td.seg];
  const BucketSpec sp = make_spec_dev(seg_P[td.seg]);
  for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < td.rows; i += blockDim.x) {
    const uint64_t h = fmix64(key_bits(keys[td.row0 + i]));
    atomicAdd(&cnt[mod_p(h, sp) * S + __umulhi((uint32_t)(h >> 32), S)], 1u);
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < NB; b += blockDim.x)
    if (cnt[b]) atomicAdd(&totals[B + b], cnt[b]);
}

template <typename T>
T *upload(Workspace &ws, const std::vector<T> &v) {
  T *d = (T *)ws.get(v.size() * sizeof(T) + 16);
  if (!d) return nullptr;
  if (!v.empty() && cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ws.stream()) !=
                        cudaSuccess)
    return nullptr;
  return d;
}

template <typename KeyT>
int seg_partition_t(Workspace &ws, const mdj_table *t, int32_t key_col, const uint64_t *seg_off, uint32_t nseg,
                    const uint32_t *seg_base, const uint32_t *seg_nb, const uint32_t *seg_P, uint32_t nb,
                    Side *out) {
  cudaStream_t s = ws.stream();
  const uint32_t n = (uint32_t)t->nrows;
  const void *src[MDJ_MAX_COLS];
  for (int j = 0; j < t->ncols; j++) src[j] = t->cols[j].data;
  bool all_single = true;
  for (uint32_t i = 0; i < nseg; i++) all_single = all_single && seg_nb[i] == 1;

  const void *key = src[key_col];
  const void *const *cols = src;
  const uint32_t *rid = nullptr;
  uint32_t *off = nullptr;
  TableBufs fin;
  fin.rid = nullptr;
  if (all_single) {
    // every segment is one bucket: bucket offsets are the segment offsets
    std::vector<uint32_t> h(nseg + 1);
    for (uint32_t i = 0; i <= nseg; i++) h[i] = (uint32_t)seg_off[i];
    off = upload(ws, h);
    if (!off) return MDJ_ERR_OOM;
  } else {
    MDJ_TRY(set_smem_attrs<KeyT>());
    std::vector<SegTile> tiles;
    for (uint32_t i = 0; i < nseg; i++)
      for (uint64_t r = seg_off[i]; r < seg_off[i + 1]; r += kTile)
        tiles.push_back(SegTile{(uint32_t)r, (uint32_t)std::min<uint64_t>(kTile, seg_off[i + 1] - r), i});
    std::vector<uint32_t> hb(seg_base, seg_base + nseg), hs(seg_nb, seg_nb + nseg), hp(seg_P, seg_P + nseg),
        hS(nseg);
    for (uint32_t i = 0; i < nseg; i++) hS[i] = seg_nb[i] / seg_P[i];
    SegTile *dt = upload(ws, tiles);
    uint32_t *db = upload(ws, hb), *ds = upload(ws, hs), *dp = upload(ws, hp), *dS = upload(ws, hS);
    off = (uint32_t *)ws.get((size_t)(nb + 1) * 4);
    uint32_t *cur = (uint32_t *)ws.get((size_t)(nb + 1) * 4);
    if (!dt || !db || !ds || !dp || !dS || !off || !cur) return MDJ_ERR_OOM;
    MDJ_CUDA_TRY(cudaMemsetAsync(off, 0, (size_t)(nb + 1) * 4, s));
    uint32_t smax = 1;
    for (uint32_t i = 0; i < nseg; i++) smax = std::max(smax, seg_nb[i]);
    if (!tiles.empty()) {
      TraceScope tr("seg_hist", s);
      k_seg_hist<KeyT><<<(unsigned)tiles.size(), kHistThreads, smax * 4, s>>>((const KeyT *)key, dt, db, ds, dp, dS,
                                                                            off);
    }
    MDJ_LAUNCH_CHECK();
    MDJ_TRY(exclusive_scan_u32(ws, off, off, nb + 1));
    MDJ_CUDA_TRY(cudaMemcpyAsync(cur, off, (size_t)nb * 4, cudaMemcpyDeviceToDevice, s));
    MDJ_TRY(alloc_table_bufs(ws, t, &fin, true));
    ColMove cm = make_move(t, key_col, src, fin.cols);
    if (!tiles.empty()) {
      TraceScope tr("seg_scatter", s);
      k_scatter<KeyT, true, true><<<(unsigned)tiles.size(), kNW * 32, scatter_smem_bytes(kPass2SpanMax), s>>>(
          (const KeyT *)key, n, make_spec(1, 1, 1), 0, (uint32_t)tiles.size(), nullptr, cur, 1, cm, nullptr,
          fin.rid, dt, db, ds, dp, dS);
    }
    MDJ_LAUNCH_CHECK();
    key = fin.cols[key_col];
    cols = fin.cols;
    rid = fin.rid;
  }
  out->key = key;
  out->key_dtype = t->cols[key_col].dtype;
  out->ncols = 0;
  for (int j = 0; j < t->ncols; j++) {
    if (j == key_col) continue;
    out->cols[out->ncols] = cols[j];
    out->widths[out->ncols] = dtype_width(t->cols[j].dtype);
    out->dtypes[out->ncols] = t->cols[j].dtype;
    out->ncols++;
  }
  out->rid = rid;
  out->off = off;
  out->nrows = n;
  return MDJ_OK;
}

}  // namespace

int partition_side_segmented(Workspace &ws, const mdj_table *t, int32_t key_col, const uint64_t *seg_off,
                             uint32_t nseg, const uint32_t *seg_base, const uint32_t *seg_nb, const uint32_t *seg_P,
                             uint32_t nbuckets, Side *out) {
  if (t->cols[key_col].dtype == MDJ_I64)
    return seg_partition_t<int64_t>(ws, t, key_col, seg_off, nseg, seg_base, seg_nb, seg_P, nbuckets, out);
  return seg_partition_t<int32_t>(ws, t, key_col, seg_off, nseg, seg_base, seg_nb, seg_P, nbuckets, out);
}

}  // namespace mdj
