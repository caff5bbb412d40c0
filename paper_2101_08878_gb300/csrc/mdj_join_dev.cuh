// Device code of the fused join item, shared by the join kernels of this
// library: descriptors, the shared-memory layout of a write item, the
// bounded look-back, and join_item (one item by one block).
#pragma once

#include <string.h>

#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr int kJoinThreads = 512;
constexpr int kPF = 8;                                   // probe rows per thread per round
constexpr uint32_t kWriteChunk = kPF * kJoinThreads;     // probe rows per write item (one round)
constexpr uint32_t kDefaultCap = 4096;
constexpr uint32_t kMaxCap = 8192;      // write-pass table: 8-byte keys fit 227 KB of shared memory
constexpr uint64_t kWaitLimitNs = 1000000000ull;         // look-back wait bound: 1 s of device time
constexpr uint32_t kPollLimit = 1u << 26;                // and a poll-count bound as a backstop
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagInc = 2ull << 62, kValMask = (1ull << 62) - 1;

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

struct Item {
  uint32_t lbeg, nl, rbeg, nr;
};

// flags[] words shared by the join kernels and the host
// (FLAG_ITEMS: the join has more work items than the arrays sized for it)
enum { FLAG_OVERFLOW = 0, FLAG_TIMEOUT = 1, FLAG_ABORT = 2, FLAG_ITEMS = 3, FLAG_WORDS = 4 };

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// ------------------------------------------------------------ fused write

// Exclusive output offset of item `it` whose own count is `total`: publish the
// count, then walk back over predecessors until one whose inclusive prefix is
// known.  Bounded: after kWaitLimitNs (or kPollLimit polls) the wait is
// abandoned, FLAG_TIMEOUT and FLAG_ABORT are set (other waiters then stop
// too) and ~0 is returned.  `withhold_first` (test hook) keeps item 0 from
// publishing, so that every later wait runs out.
__device__ uint64_t look_back(unsigned long long *state, uint32_t it, uint64_t total, int *flags,
                              int withhold_first) {
  volatile unsigned long long *vs = state;
  if (it == 0) {
    if (withhold_first) return ~0ull;
    __threadfence();
    atomicExch(&state[0], kFlagInc | total);
    return 0;
  }
  __threadfence();
  atomicExch(&state[it], kFlagAgg | total);
  uint64_t excl = 0;
  uint32_t j = it - 1;
  uint32_t polls = 0;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    const unsigned long long v = vs[j];
    const uint64_t flag = v & ~kValMask;
    if (flag == 0) {
      if (++polls > kPollLimit || globaltimer_ns() - t0 > kWaitLimitNs || ((volatile int *)flags)[FLAG_ABORT]) {
        atomicExch(&flags[FLAG_TIMEOUT], 1);
        atomicExch(&flags[FLAG_ABORT], 1);
        return ~0ull;
      }
      __nanosleep(64);
      continue;
    }
    excl += v & kValMask;
    if (flag == kFlagInc || j == 0) break;
    j--;
  }
  __threadfence();
  atomicExch(&state[it], kFlagInc | (excl + total));
  return excl;
}

// ------------------------------------------------------------ fused write
//
// Two 512-thread blocks per SM.  Per item:
//   1. the build chunk's keys, row ids and first payload column go to shared
//      memory: its 16-byte-aligned interior by bulk asynchronous copies (TMA,
//      completing on an mbarrier), the ragged ends by ordinary loads; the
//      probe keys load into registers and the table heads are cleared
//      meanwhile;
//   2. build: a chained table, heads[slot] -> row, nxt[row] -> row, one
//      atomicExch per build row (no probing loop, no compare-and-swap);
//   3. probe: walk the key's chain; first match and match count per row;
//   4. the row ids and first payload of matching probe rows are loaded, so
//      their latency overlaps the offset computation;
//   5. offsets: every warp counts its single-match rows (ballot + popc per
//      round) and its multi-match rows' matches; one warp scans the warps'
//      counts and reserves the item's range (atomicAdd) or looks it back
//      (ordered): two block barriers;
//   6. write: a warp's single-match rows land consecutively (warp, round,
//      lane order), then each multi-match row expands its chain; build-side
//      values from shared memory, probe-side from registers.
// The next item's ticket and descriptor are fetched while the current one runs.

constexpr int kWT = 512;                        // threads of the write block (default; 256 also built)
constexpr int kWPF = 8;                         // probe rows per thread
constexpr int kWW = kWT / 32;                   // warps of the largest write block
static_assert(kWPF * kWT == (int)kWriteChunk, "probe chunk = one round");
constexpr uint64_t kStageWaitNs = 1000000000ull;  // bulk-copy wait bound: 1 s of device time

// Shared memory of a write block: each staged column has 16 bytes of slack in
// front (its first element sits at the chunk start's offset within a 16-byte
// line, so the bulk-copied interior lands on a 16-byte boundary).
template <typename KeyT>
struct WriteLayout {
  size_t keys, rid, pay, heads, nxt, total;
  uint32_t tsz;  // chain heads of the largest table (>= cap: mean chain length <= 1)
  __host__ __device__ WriteLayout(uint32_t cap) {
    tsz = 32;
    while (tsz < cap) tsz *= 2;
    keys = 0;
    rid = align16((size_t)cap * sizeof(KeyT) + 16);
    pay = align16(rid + (size_t)cap * 4 + 16);
    heads = align16(pay + (size_t)cap * 8 + 16);
    nxt = heads + (size_t)tsz * 4;
    total = align16(nxt + (size_t)cap * 2);
  }
};

// Chain-head slot of a key: 32-bit fold, one multiply, top logt bits.
__device__ __forceinline__ uint32_t chain_slot(uint64_t kb, uint32_t logt) {
  const uint32_t f = (uint32_t)kb ^ (uint32_t)(kb >> 32);
  return (f * 0x9E3779B1u) >> (32 - logt);
}

__device__ __forceinline__ void cp_async_4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(__cvta_generic_to_global(src))
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- bulk copies (TMA, cp.async.bulk) completing on an mbarrier

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once, announcing `bytes` of transaction count still to land.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar`, for at most `limit_ns` of device time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t polls = 0; polls < (1u << 26); polls++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Elements [beg, beg + n) of a column of `es`-byte elements whose base is
// 16-byte aligned: the 16-byte-aligned interior [a, b) goes by one bulk copy,
// the head [beg, a) and tail [b, beg + n) by ordinary loads.  In shared
// memory element beg + i sits at index sh + i of the staging buffer, sh =
// beg mod (16 / es), so the interior starts on a 16-byte boundary.
struct BulkPart {
  uint32_t sh, a, b;
};
__device__ __forceinline__ BulkPart bulk_part(uint32_t beg, uint32_t n, uint32_t es) {
  const uint32_t per = 16 / es;
  BulkPart p;
  p.sh = beg % per;
  p.a = (beg + per - 1) / per * per;
  p.b = (beg + n) / per * per;
  if (p.b <= p.a) p.a = p.b = beg + n;  // no aligned interior: all by ordinary loads
  return p;
}

// Non-key columns after the first of each side (gathered from global memory).
__device__ __forceinline__ void copy_extra_cols(const JSide &L, const JSide &R, const JOut &out, uint64_t pos,
                                                uint32_t lrow, uint32_t r) {
  for (int cc = 1; cc < L.ncols; cc++) {
    if (L.width[cc] == 8)
      ((uint64_t *)out.lcols[cc])[pos] = ((const uint64_t *)L.cols[cc])[lrow];
    else
      ((uint32_t *)out.lcols[cc])[pos] = ((const uint32_t *)L.cols[cc])[lrow];
  }
  for (int cc = 1; cc < R.ncols; cc++) {
    if (R.width[cc] == 8)
      ((uint64_t *)out.rcols[cc])[pos] = ((const uint64_t *)R.cols[cc])[r];
    else
      ((uint32_t *)out.rcols[cc])[pos] = ((const uint32_t *)R.cols[cc])[r];
  }
}

// One output row: build row li of the staged chunk, probe row r with row id
// rr and first payload rp.
template <typename KeyT>
__device__ __forceinline__ void write_row(const JSide &L, const JSide &R, const JOut &out, uint64_t pos,
                                          const KeyT *bkey, const uint32_t *brid, const unsigned char *bpay, int lpw,
                                          uint32_t li, uint32_t lbeg, uint32_t r, uint32_t rr, uint64_t rp) {
  ((KeyT *)out.key)[pos] = bkey[li];
  out.lrow[pos] = brid[li];
  out.rrow[pos] = rr;
  if (lpw == 8) ((uint64_t *)out.lcols[0])[pos] = ((const uint64_t *)bpay)[li];
  if (lpw == 4) ((uint32_t *)out.lcols[0])[pos] = ((const uint32_t *)bpay)[li];
  if (R.ncols > 0) {
    if (R.width[0] == 8)
      ((uint64_t *)out.rcols[0])[pos] = rp;
    else
      ((uint32_t *)out.rcols[0])[pos] = (uint32_t)rp;
  }
  if (L.ncols > 1 || R.ncols > 1) copy_extra_cols(L, R, out, pos, lbeg + li, r);
}

struct JoinShared {
  uint64_t base;
  uint64_t item_total;
  uint32_t wsingle[kWW];   // per warp: exclusive prefix of single-match rows
  uint64_t wmulti[kWW];    // per warp: exclusive prefix of multi-match output rows
  uint32_t single_total;
  int stage_ok;            // the build chunk's bulk copies landed in time
  uint64_t bar;            // mbarrier of the build chunk's bulk copies (initialised by the kernel)
};

struct Resv {
  unsigned long long *state;
  uint64_t *item_off;
  unsigned long long *total;
  uint64_t capacity;
  int *flags;
  int withhold_first;
  int ordered;
};

// One join item (steps 1-6 above) by the whole block; `it` is the item's
// index (its look-back slot and item_off entry).  `bulk`: the build side's
// columns may be staged by bulk copies (their bases are 16-byte aligned);
// `phase` is the mbarrier's phase, kept by every thread.  Leaves every thread
// past the write, with no barrier after it; returns false if a bulk-copy
// wait ran out (FLAG_TIMEOUT and FLAG_ABORT are then set).
// COUNT: build and probe only; the item's output row count goes to
// item_off[it] (the count pass of two-pass ordered output).
template <typename KeyT, bool HAVE_OFFSETS, int NT, bool COUNT = false>
__device__ __forceinline__ bool join_item(unsigned char *smem, uint32_t cap, const JSide &L, const JSide &R,
                                          const Item &d, uint32_t it, const Resv &rs, const JOut &out,
                                          JoinShared &js, bool bulk, uint32_t &phase) {
  constexpr int kWT = NT, kWW = NT / 32;  // this block's threads and warps
  const WriteLayout<KeyT> lay(cap);
  const KeyT *__restrict__ Lkey = (const KeyT *)L.key;
  const KeyT *__restrict__ Rkey = (const KeyT *)R.key;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lpw = L.ncols > 0 ? L.width[0] : 0;
  const int rpw = R.ncols > 0 ? R.width[0] : 0;
  const uint32_t ek = sizeof(KeyT);

  // 1. stage the build chunk; probe keys to registers; clear the heads
  const BulkPart pk = bulk_part(d.lbeg, d.nl, ek);
  const BulkPart pr = bulk_part(d.lbeg, d.nl, 4);
  const BulkPart pp = bulk_part(d.lbeg, d.nl, lpw ? (uint32_t)lpw : 8u);
  KeyT *bkey = (KeyT *)(smem + lay.keys) + (bulk ? pk.sh : 0u);
  uint32_t *brid = (uint32_t *)(smem + lay.rid) + (bulk ? pr.sh : 0u);
  unsigned char *bpay = smem + lay.pay + (bulk ? (size_t)pp.sh * (lpw ? lpw : 8) : 0u);
  uint32_t *heads = (uint32_t *)(smem + lay.heads);
  uint16_t *nxt = (uint16_t *)(smem + lay.nxt);
  if (bulk) {
    if (tid == 0) {
      const uint32_t bk = (pk.b - pk.a) * ek, br = L.rid ? (pr.b - pr.a) * 4 : 0u,
                     bp = lpw ? (pp.b - pp.a) * (uint32_t)lpw : 0u;
      fence_proxy_async_shared();  // the previous item's reads of these buffers come first
      mbar_arrive_expect_tx(&js.bar, bk + br + bp);
      if (bk) bulk_g2s(bkey + (pk.a - d.lbeg), Lkey + pk.a, bk, &js.bar);
      if (br) bulk_g2s(brid + (pr.a - d.lbeg), L.rid + pr.a, br, &js.bar);
      if (bp) bulk_g2s(bpay + (size_t)(pp.a - d.lbeg) * lpw, (const unsigned char *)L.cols[0] + (size_t)pp.a * lpw,
                       bp, &js.bar);
    }
    // the ragged ends by ordinary loads: at most 6 elements before the
    // aligned interior (all of a range too short to have one) and 3 after
    if (tid < 8) {
      const uint32_t i = tid;
      if (i < pk.a - d.lbeg) bkey[i] = Lkey[d.lbeg + i];
      if (L.rid && i < pr.a - d.lbeg) brid[i] = L.rid[d.lbeg + i];
      if (lpw == 8 && i < pp.a - d.lbeg) ((uint64_t *)bpay)[i] = ((const uint64_t *)L.cols[0])[d.lbeg + i];
      if (lpw == 4 && i < pp.a - d.lbeg) ((uint32_t *)bpay)[i] = ((const uint32_t *)L.cols[0])[d.lbeg + i];
    } else if (tid < 16) {
      const uint32_t q = tid - 8;
      if (pk.b + q < d.lbeg + d.nl) bkey[pk.b + q - d.lbeg] = Lkey[pk.b + q];
      if (L.rid && pr.b + q < d.lbeg + d.nl) brid[pr.b + q - d.lbeg] = L.rid[pr.b + q];
      if (lpw == 8 && pp.b + q < d.lbeg + d.nl)
        ((uint64_t *)bpay)[pp.b + q - d.lbeg] = ((const uint64_t *)L.cols[0])[pp.b + q];
      if (lpw == 4 && pp.b + q < d.lbeg + d.nl)
        ((uint32_t *)bpay)[pp.b + q - d.lbeg] = ((const uint32_t *)L.cols[0])[pp.b + q];
    }
    if (!L.rid)
      for (uint32_t i = tid; i < d.nl; i += kWT) brid[i] = d.lbeg + i;
  } else {
    for (uint32_t i = tid; i < d.nl; i += kWT) {
      const uint32_t g = d.lbeg + i;
      if (sizeof(KeyT) == 8)
        cp_async_8(&bkey[i], &Lkey[g]);
      else
        cp_async_4(&bkey[i], &Lkey[g]);
      if (L.rid)
        cp_async_4(&brid[i], &L.rid[g]);
      else
        brid[i] = g;
      if (lpw == 8) cp_async_8(&((uint64_t *)bpay)[i], &((const uint64_t *)L.cols[0])[g]);
      if (lpw == 4) cp_async_4(&((uint32_t *)bpay)[i], &((const uint32_t *)L.cols[0])[g]);
    }
  }
  KeyT rk[kWPF];
#pragma unroll
  for (int j = 0; j < kWPF; j++) {
    const uint32_t rl = j * kWT + tid;
    rk[j] = rl < d.nr ? Rkey[d.rbeg + rl] : KeyT(0);
  }
  uint32_t logt = 5;
  while ((1u << logt) < d.nl) logt++;
  const uint32_t tsz = 1u << logt;
  {
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (uint32_t s = tid * 4; s < tsz; s += kWT * 4) *(uint4 *)(heads + s) = z;
  }
  if (bulk) {
    // thread 0 waits (bounded) and tells the block; the others then see the
    // completed phase at once (each thread's own wait orders the copied data)
    if (tid == 0) {
      js.stage_ok = mbar_wait_bounded(&js.bar, phase, kStageWaitNs) ? 1 : 0;
      if (!js.stage_ok) {
        atomicExch(&rs.flags[FLAG_TIMEOUT], 1);
        atomicExch(&rs.flags[FLAG_ABORT], 1);
        mbar_wait_bounded(&js.bar, phase, kStageWaitNs);  // let copies in flight land before leaving
      }
    }
    __syncthreads();
    if (!js.stage_ok) return false;
    if (tid != 0) mbar_wait_bounded(&js.bar, phase, kStageWaitNs);
    phase ^= 1;
  } else {
    cp_async_wait_all();
  }
  __syncthreads();

  // 2. build: push every row onto its slot's chain
  for (uint32_t i = tid; i < d.nl; i += kWT) {
    const uint32_t s = chain_slot(key_bits(bkey[i]), logt);
    nxt[i] = (uint16_t)atomicExch(&heads[s], i + 1);
  }
  __syncthreads();

  // 3. probe: ch[j] = (matches << 16) | (first matching row + 1)
  uint32_t ch[kWPF];
  uint32_t nm = 0;
#pragma unroll
  for (int j = 0; j < kWPF; j++) {
    ch[j] = 0;
    if (j * kWT + tid < d.nr) {
      const KeyT k = rk[j];
      uint32_t li = heads[chain_slot(key_bits(k), logt)], first = 0, c = 0;
      while (li) {
        if (bkey[li - 1] == k) {
          if (!c) first = li;
          c++;
        }
        li = nxt[li - 1];
      }
      ch[j] = (c << 16) | first;
      if (c >= 2) nm += c;
    }
  }

  // 4. probe-side row id and first payload of every matching row
  uint32_t rr[kWPF];
  uint64_t rp[kWPF];
#pragma unroll
  for (int j = 0; j < kWPF; j++) {
    rr[j] = 0;
    rp[j] = 0;
    if (!COUNT && ch[j]) {
      const uint32_t r = d.rbeg + j * kWT + tid;
      rr[j] = R.rid ? R.rid[r] : r;
      if (rpw == 8) rp[j] = ((const uint64_t *)R.cols[0])[r];
      if (rpw == 4) rp[j] = ((const uint32_t *)R.cols[0])[r];
    }
  }

  // 5. offsets: per-warp counts, one scanning warp, the item's range
  uint32_t wsingle = 0;
#pragma unroll
  for (int j = 0; j < kWPF; j++) wsingle += __popc(__ballot_sync(0xffffffffu, (ch[j] >> 16) == 1));
  const uint32_t nm_inc = warp_inclusive_scan(nm);
  if (lane == 31) {
    js.wsingle[warp] = wsingle;
    js.wmulti[warp] = nm_inc;
  }
  __syncthreads();
  if (warp == 0) {
    const uint32_t sv = lane < kWW ? js.wsingle[lane] : 0u;
    const uint64_t mv = lane < kWW ? js.wmulti[lane] : 0ull;
    const uint32_t si = warp_inclusive_scan(sv);
    const uint64_t mi = warp_inclusive_scan(mv);
    const uint32_t S = __shfl_sync(0xffffffffu, si, 31);
    const uint64_t M = __shfl_sync(0xffffffffu, mi, 31);
    if (lane < kWW) {
      js.wsingle[lane] = si - sv;
      js.wmulti[lane] = mi - mv;
    }
    if (lane == 0) {
      const uint64_t item_total = S + M;
      uint64_t base;
      if (COUNT) {
        rs.item_off[it] = item_total;
        base = ~0ull;
      } else if (HAVE_OFFSETS) {
        base = rs.item_off[it];
      } else {
        if (rs.ordered) {
          base = look_back(rs.state, it, item_total, rs.flags, rs.withhold_first);
          if (base != ~0ull && item_total) atomicAdd(rs.total, (unsigned long long)item_total);
        } else {
          base = item_total ? atomicAdd(rs.total, (unsigned long long)item_total) : 0ull;
        }
        if (base != ~0ull) {
          rs.item_off[it] = base;
          if (base + item_total > rs.capacity) atomicExch(&rs.flags[FLAG_OVERFLOW], 1);
        }
      }
      js.base = base;
      js.single_total = S;
      js.item_total = item_total;
    }
  }
  __syncthreads();
  if (COUNT) return true;

  // 6. write (an item that overflows the optimistic buffer writes nothing:
  // the exact second pass places it)
  const uint64_t base = js.base;
  if (base != ~0ull && base + js.item_total <= rs.capacity) {
    const uint32_t S = js.single_total;
    uint64_t spos = base + js.wsingle[warp];
#pragma unroll
    for (int j = 0; j < kWPF; j++) {
      const bool one = (ch[j] >> 16) == 1;
      const uint32_t bal = __ballot_sync(0xffffffffu, one);
      if (one) {
        const uint64_t pos = spos + __popc(bal & lanemask_lt());
        write_row<KeyT>(L, R, out, pos, bkey, brid, bpay, lpw, (ch[j] & 0xFFFFu) - 1, d.lbeg,
                        d.rbeg + j * kWT + tid, rr[j], rp[j]);
      }
      spos += __popc(bal);
    }
    if (nm) {
      uint64_t pos = base + S + js.wmulti[warp] + (nm_inc - nm);
#pragma unroll
      for (int j = 0; j < kWPF; j++) {
        if ((ch[j] >> 16) < 2) continue;
        uint32_t li = ch[j] & 0xFFFFu;
        const KeyT k = bkey[li - 1];
        while (li) {
          if (bkey[li - 1] == k)
            write_row<KeyT>(L, R, out, pos++, bkey, brid, bpay, lpw, li - 1, d.lbeg, d.rbeg + j * kWT + tid,
                            rr[j], rp[j]);
          li = nxt[li - 1];
        }
      }
    }
  }
  return true;
}

}  // namespace
}  // namespace mdj
