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
constexpr uint32_t kCountChunk = 65536;                  // probe rows per count item
constexpr uint32_t kDefaultCap = 4096;
constexpr uint32_t kMaxCap = 8192;      // write-pass table: 8-byte keys fit 227 KB of shared memory
constexpr uint32_t kCountCapMax = 4096;  // count/checksum table (per-slot counts and sums)
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
enum { FLAG_OVERFLOW = 0, FLAG_TIMEOUT = 1, FLAG_ABORT = 2, FLAG_WORDS = 4 };

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
//      memory by asynchronous copies (cp.async) while the probe keys load
//      into registers and the table heads are cleared;
//   2. build: a chained table, heads[slot] -> row, nxt[row] -> row, one
//      atomicExch per build row (no probing loop, no compare-and-swap);
//   3. probe: walk the key's chain; first match and match count per row;
//   4. the row ids and first payload of matching probe rows are loaded, so
//      their latency overlaps the offset computation;
//   5. offsets: rows with one match are ordered by (round j, warp, lane), so
//      the matching lanes of one warp store consecutive output rows (ballot +
//      popc); rows with several matches follow, each expanded by its thread;
//      the item's range is reserved (atomicAdd) or looked back (ordered);
//   6. write: build-side values from shared memory, probe-side from registers.
// The next item's ticket and descriptor are fetched while the current one runs.

constexpr int kWT = 512;                        // threads of the write block
constexpr int kWPF = 8;                         // probe rows per thread
constexpr int kWW = kWT / 32;                   // warps of the write block
static_assert(kWPF * kWT == (int)kWriteChunk, "probe chunk = one round");

template <typename KeyT>
struct WriteLayout {
  size_t keys, rid, pay, heads, nxt, cnt1, total;
  uint32_t tsz;  // chain heads of the largest table (>= cap: mean chain length <= 1)
  __host__ __device__ WriteLayout(uint32_t cap) {
    tsz = 32;
    while (tsz < cap) tsz *= 2;
    keys = 0;
    rid = align16((size_t)cap * sizeof(KeyT));
    pay = align16(rid + (size_t)cap * 4);
    heads = align16(pay + (size_t)cap * 8);
    nxt = heads + (size_t)tsz * 4;
    cnt1 = align16(nxt + (size_t)cap * 2);
    total = cnt1 + (size_t)kWPF * kWW * 4;
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
                                          const KeyT *bkey, const uint32_t *brid, const uint64_t *bpay, uint32_t li,
                                          uint32_t lbeg, uint32_t r, uint32_t rr, uint64_t rp) {
  ((KeyT *)out.key)[pos] = bkey[li];
  out.lrow[pos] = brid[li];
  out.rrow[pos] = rr;
  if (L.ncols > 0) {
    if (L.width[0] == 8)
      ((uint64_t *)out.lcols[0])[pos] = bpay[li];
    else
      ((uint32_t *)out.lcols[0])[pos] = (uint32_t)bpay[li];
  }
  if (R.ncols > 0) {
    if (R.width[0] == 8)
      ((uint64_t *)out.rcols[0])[pos] = rp;
    else
      ((uint32_t *)out.rcols[0])[pos] = (uint32_t)rp;
  }
  if (L.ncols > 1 || R.ncols > 1) copy_extra_cols(L, R, out, pos, lbeg + li, r);
}

// One join item (steps 1-6 above) by the whole block; `it` is the item's
// index (its look-back slot and item_off entry).  Leaves every thread past
// the write, with no barrier after it.
struct JoinShared {
  uint32_t single;
  uint64_t base;
  uint64_t scratch64[33];
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

template <typename KeyT, bool HAVE_OFFSETS>
__device__ __forceinline__ void join_item(unsigned char *smem, uint32_t cap, const JSide &L, const JSide &R,
                                          const Item &d, uint32_t it, const Resv &rs, const JOut &out,
                                          JoinShared &js) {
  const WriteLayout<KeyT> lay(cap);
  KeyT *bkey = (KeyT *)(smem + lay.keys);
  uint32_t *brid = (uint32_t *)(smem + lay.rid);
  uint64_t *bpay = (uint64_t *)(smem + lay.pay);
  uint32_t *heads = (uint32_t *)(smem + lay.heads);
  uint16_t *nxt = (uint16_t *)(smem + lay.nxt);
  uint32_t *cnt1 = (uint32_t *)(smem + lay.cnt1);
  const KeyT *__restrict__ Lkey = (const KeyT *)L.key;
  const KeyT *__restrict__ Rkey = (const KeyT *)R.key;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lpw = L.ncols > 0 ? L.width[0] : 0;
  const int rpw = R.ncols > 0 ? R.width[0] : 0;

    // 1. stage the build chunk; probe keys to registers; clear the heads
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
      if (lpw == 8) cp_async_8(&bpay[i], &((const uint64_t *)L.cols[0])[g]);
      if (lpw == 4) cp_async_4(&bpay[i], &((const uint32_t *)L.cols[0])[g]);
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
    cp_async_wait_all();
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
      if (ch[j]) {
        const uint32_t r = d.rbeg + j * kWT + tid;
        rr[j] = R.rid ? R.rid[r] : r;
        if (rpw == 8) rp[j] = ((const uint64_t *)R.cols[0])[r];
        if (rpw == 4) rp[j] = ((const uint32_t *)R.cols[0])[r];
      }
    }

    // 5. offsets: single-match rows by (j, warp, lane), then the rest
#pragma unroll
    for (int j = 0; j < kWPF; j++) {
      const uint32_t bal = __ballot_sync(0xffffffffu, (ch[j] >> 16) == 1);
      if (lane == 0) cnt1[j * kWW + warp] = __popc(bal);
    }
    uint64_t mtot;
    const uint64_t mex = block_exclusive_scan<uint64_t>(nm, js.scratch64, &mtot);  // barriers inside
    if (warp == 0) {
      constexpr int per = kWPF * kWW / 32;
      uint32_t v[per], sum = 0;
#pragma unroll
      for (int q = 0; q < per; q++) {
        v[q] = cnt1[lane * per + q];
        sum += v[q];
      }
      const uint32_t inc = warp_inclusive_scan(sum);
      uint32_t run = inc - sum;
#pragma unroll
      for (int q = 0; q < per; q++) {
        cnt1[lane * per + q] = run;
        run += v[q];
      }
      if (lane == 31) js.single = inc;
    }
    __syncthreads();
    const uint32_t S = js.single;
    const uint64_t item_total = S + mtot;
    if (tid == 0) {
      uint64_t base;
      if (HAVE_OFFSETS) {
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
    }
    __syncthreads();

    // 6. write
    const uint64_t base = js.base;
    if (base != ~0ull && base + item_total <= rs.capacity) {
#pragma unroll
      for (int j = 0; j < kWPF; j++) {
        const bool one = (ch[j] >> 16) == 1;
        const uint32_t bal = __ballot_sync(0xffffffffu, one);
        if (one) {
          const uint64_t pos = base + cnt1[j * kWW + warp] + __popc(bal & lanemask_lt());
          write_row<KeyT>(L, R, out, pos, bkey, brid, bpay, (ch[j] & 0xFFFFu) - 1, d.lbeg, d.rbeg + j * kWT + tid,
                          rr[j], rp[j]);
        }
      }
      if (nm) {
        uint64_t pos = base + S + mex;
#pragma unroll
        for (int j = 0; j < kWPF; j++) {
          if ((ch[j] >> 16) < 2) continue;
          uint32_t li = ch[j] & 0xFFFFu;
          const KeyT k = bkey[li - 1];
          while (li) {
            if (bkey[li - 1] == k)
              write_row<KeyT>(L, R, out, pos++, bkey, brid, bpay, li - 1, d.lbeg, d.rbeg + j * kWT + tid, rr[j],
                              rp[j]);
            li = nxt[li - 1];
          }
        }
      }
    }
}

}  // namespace
}  // namespace mdj
