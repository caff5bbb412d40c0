// The paper's second workload: the sum of an array and its transpose,
// y = x + x^T (Sec. V-B "Sum of cuPy Array and its Transpose", Fig. 7:
// 16K x 16K in 4K chunks; Sec. V-C, Fig. 9(a): 20E3 x 20E3 in 5E2 chunks).
// With the chunks spread over Dask workers, chunk (i, j) of y needs chunk
// (j, i) of x from another worker: that exchange is what the benchmark times.
// On one GPU the chunk exchange is the read of the mirrored tile.
//
// One block handles a pair of mirrored 64 x 64 tiles, (I, J) and (J, I) with
// I <= J: it loads both into padded shared memory (row stride 65, so reading
// a tile column hits distinct banks), then writes y(I, J) = x(I, J) +
// x(J, I)^T and y(J, I) = x(J, I) + x(I, J)^T.  Every element of x is read
// once and every element of y written once (16 bytes per float64 element),
// with coalesced rows both ways.  A block reads both tiles before it writes
// either, and no other block touches them, so y may be x (in place).
// Integer types add with wraparound; float types with one IEEE addition, so
// the result is exact and symmetric.
#include <math.h>
#include <string.h>

#include "mdj_internal.cuh"

namespace mdj {
namespace {

constexpr int kTW = 8;  // warps per block

template <typename V>
__device__ __forceinline__ V add(V a, V b) {
  return a + b;
}

// Pair p of the upper triangle of nt x nt tiles, row-major: (I, J), I <= J.
// Row I holds nt - I pairs and starts at S(I) = I * (2 nt - I + 1) / 2.
__device__ __forceinline__ void pair_of(uint64_t p, uint32_t nt, uint32_t &I, uint32_t &J) {
  const double b = 2.0 * nt + 1.0;
  double g = floor((b - sqrt(b * b - 8.0 * (double)p)) / 2.0);
  uint64_t i = g < 0 ? 0 : (uint64_t)g;
  auto S = [nt](uint64_t r) { return r * (2ull * nt - r + 1) / 2; };
  while (i > 0 && S(i) > p) i--;
  while (i + 1 < nt && S(i + 1) <= p) i++;
  I = (uint32_t)i;
  J = (uint32_t)(i + (p - S(i)));
}

// Tile geometry: TT x TT elements, row stride TT + 1 in shared memory, each
// warp ROWS rows, each lane COLS elements of a row (lane, lane + 32, ..).
template <int TT>
struct Geom {
  static constexpr int P = TT + 1;
  static constexpr int ROWS = TT / kTW;
  static constexpr int COLS = TT / 32;
};

// Rows r0 + warp + kTW * k of one tile (columns c0 ..) into shared memory:
// all of a thread's loads first, then its stores.  (Issuing both tiles'
// loads before either store was slower: 1.05 vs 0.98 ms at 16K x 16K f64.)
template <typename V, int TT>
__device__ __forceinline__ void load_tile(const V *x, uint64_t n, uint64_t r0, uint64_t c0, V *T) {
  using G = Geom<TT>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V v[G::ROWS * G::COLS];
  const uint64_t c = c0 + lane;
  const V *row = x + (r0 + warp) * n + c;  // this thread's element of its first row
#pragma unroll
  for (int k = 0; k < G::ROWS; k++) {
    const bool rin = r0 + warp + kTW * k < n;
#pragma unroll
    for (int h = 0; h < G::COLS; h++) v[G::COLS * k + h] = (rin && c + 32 * h < n) ? row[32 * h] : V(0);
    row += kTW * n;
  }
#pragma unroll
  for (int k = 0; k < G::ROWS; k++)
#pragma unroll
    for (int h = 0; h < G::COLS; h++) T[(warp + kTW * k) * G::P + lane + 32 * h] = v[G::COLS * k + h];
}

// y rows r0 + .. (columns c0 + ..) = P[r][c] + Q[c][r].
template <typename V, int TT>
__device__ __forceinline__ void store_tile(V *y, uint64_t n, uint64_t r0, uint64_t c0, const V *P, const V *Q) {
  using G = Geom<TT>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t c = c0 + lane;
  V *row = y + (r0 + warp) * n + c;
#pragma unroll
  for (int k = 0; k < G::ROWS; k++) {
    const int rr = warp + kTW * k;
    if (r0 + rr < n) {
#pragma unroll
      for (int h = 0; h < G::COLS; h++)
        if (c + 32 * h < n) row[32 * h] = add(P[rr * G::P + lane + 32 * h], Q[(lane + 32 * h) * G::P + rr]);
    }
    row += kTW * n;
  }
}

// Three blocks per SM: a pair of 64-edge tiles of 8-byte elements takes
// 67 KB of shared memory.
template <typename V, int TT>
__global__ void __launch_bounds__(kTW * 32, 3)
    k_transpose_add(const V *x, V *y, uint64_t n, uint32_t nt, uint64_t npairs) {
  extern __shared__ __align__(16) unsigned char smem[];
  V *A = (V *)smem;                  // x tile (I, J)
  V *B = A + TT * Geom<TT>::P;       // x tile (J, I)
  for (uint64_t p = blockIdx.x; p < npairs; p += gridDim.x) {
    uint32_t I, J;
    pair_of(p, nt, I, J);
    const uint64_t rI = (uint64_t)I * TT, rJ = (uint64_t)J * TT;
    load_tile<V, TT>(x, n, rI, rJ, A);
    if (I != J) load_tile<V, TT>(x, n, rJ, rI, B);
    __syncthreads();
    if (I == J) {
      store_tile<V, TT>(y, n, rI, rI, A, A);
    } else {
      store_tile<V, TT>(y, n, rI, rJ, A, B);
      store_tile<V, TT>(y, n, rJ, rI, B, A);
    }
    __syncthreads();
  }
}

template <typename V, int TT>
int launch_tt(const void *x, void *y, uint64_t n, cudaStream_t s) {
  const uint32_t nt = (uint32_t)((n + TT - 1) / TT);
  const uint64_t npairs = (uint64_t)nt * (nt + 1) / 2;
  const size_t sm = 2 * (size_t)TT * Geom<TT>::P * sizeof(V);
  MDJ_CUDA_TRY(cudaFuncSetAttribute(k_transpose_add<V, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  MDJ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transpose_add<V, TT>, kTW * 32, sm));
  if (per_sm < 1) return MDJ_ERR_INTERNAL;
  const uint64_t most = (uint64_t)num_sms() * per_sm;
  const unsigned grid = (unsigned)(npairs < most ? npairs : most);
  TraceScope tr("transpose_add", s);
  k_transpose_add<V, TT><<<grid, kTW * 32, sm, s>>>((const V *)x, (V *)y, n, nt, npairs);
  MDJ_LAUNCH_CHECK();
  return MDJ_OK;
}

// Tile edge 64: measured faster than 32 (0.98 vs 1.65 ms at 16K x 16K f64).
template <typename V>
int launch(const void *x, void *y, uint64_t n, cudaStream_t s) {
  return launch_tt<V, 64>(x, y, n, s);
}

}  // namespace
}  // namespace mdj

extern "C" int mdj_transpose_add(const void *x, void *y, uint64_t n, int32_t dtype, void *stream) {
  using namespace mdj;
  const int w = dtype_width(dtype);
  if (w == 0) return MDJ_ERR_UNSUPPORTED_DTYPE;
  if (n == 0) return MDJ_OK;
  if (!x || !y) return MDJ_ERR_INVALID_ARG;
  if (n >= (1ull << 32)) return MDJ_ERR_TOO_LARGE;
  const uint64_t bytes = n * n * (uint64_t)w;
  const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
  if (xa != ya && xa < ya + bytes && ya < xa + bytes) return MDJ_ERR_INVALID_ARG;  // partial overlap
  if (xa % w || ya % w) return MDJ_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  switch (dtype) {
    case MDJ_F32: return launch<float>(x, y, n, s);
    case MDJ_F64: return launch<double>(x, y, n, s);
    case MDJ_I32: case MDJ_U32: return launch<uint32_t>(x, y, n, s);  // wraparound add
    default: return launch<uint64_t>(x, y, n, s);
  }
}
