/*
 * mdj.h - C ABI of libmdj.so: a GB300 (sm_103a) hash-partitioned shuffle and
 * hash join of two key/payload tables (inner, and its left / right / outer
 * and key-tuple variants).
 *
 * What the calls compute comes from the cuDF merge workload of arXiv 2101.08878
 * (Sec. V-B "cuDF Merge", Fig. 8, and Sec. V-C, Fig. 9(b,c)): tables are
 * repartitioned by key hash ("Shuffle: True") so that equal keys meet in one
 * partition, then each partition pair is merged.  The paper moves partitions
 * between Dask workers over MPI (Sec. IV-B, the Isend/Irecv coroutines); on one
 * GPU that exchange is the on-device scatter done by mdj_partition, and the
 * partition region p in device memory plays worker p's receive buffer.  The
 * paper names no hash, join algorithm or output layout; the readings below are
 * this library's contract.
 *
 * Conventions shared by every call:
 *  - Pointers inside mdj_col / output arrays are DEVICE pointers of the current
 *    CUDA device; structs passed by pointer (mdj_table, mdj_result, ...) live in
 *    HOST memory.  Input columns are read-only and remain owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call is asynchronous on that stream, except mdj_join / mdj_merge /
 *    mdj_count_checksum, the batch, stream, tuple and host calls, which read
 *    small counts back to the host to size their outputs (the joins: the output
 *    row count, with the work-item count and flags, in one stream
 *    synchronisation; one more pass when an optimistic size was too small).
 *  - Workspace and join outputs come from the caller's allocator (mdj_allocator);
 *    a NULL allocator means cudaMallocAsync / cudaFreeAsync on `stream`.
 *  - Keys are signed integers (MDJ_I32 or MDJ_I64); both sides of a join must use
 *    the same key dtype.  Every other column is a payload of width 4 or 8 bytes
 *    whose bits are copied, never interpreted (NaN patterns survive).
 *  - Row counts must be < 2^32 (row ids are uint32); larger inputs give
 *    MDJ_ERR_TOO_LARGE.  Output counts and offsets are 64-bit.
 *  - Hash: h = fmix64((uint64)(int64)key), the 64-bit finalizer of MurmurHash3;
 *    partition p = h mod P (unsigned).  int32 and int64 keys with equal values
 *    land in the same partition.
 *  - Return value: MDJ_OK (0) or a negative mdj_status.  On error no output
 *    buffer is left allocated and the caller's buffers hold unspecified data.
 */
#ifndef MDJ_H
#define MDJ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MDJ_API __attribute__((visibility("default")))
#else
#define MDJ_API
#endif

#define MDJ_VERSION 1
#define MDJ_MAX_COLS 16      /* columns per table, key included */
#define MDJ_MAX_PARTITIONS 65536u

typedef enum {
    MDJ_OK = 0,
    MDJ_ERR_INVALID_ARG = -1,       /* null pointer, P == 0 or > 65536, bad key index, key dtype mismatch */
    MDJ_ERR_UNSUPPORTED_DTYPE = -2, /* key not I32/I64, or a column of unknown dtype */
    MDJ_ERR_TOO_LARGE = -3,         /* nrows >= 2^32 */
    MDJ_ERR_OOM = -4,               /* the allocator returned NULL */
    MDJ_ERR_CUDA = -5,              /* a CUDA runtime call failed */
    MDJ_ERR_DEVICE_TIMEOUT = -6,    /* a bounded device-side wait gave up */
    MDJ_ERR_INTERNAL = -7,          /* a device-side consistency check failed */
    MDJ_ERR_ABORTED = -8            /* a caller's sink asked to stop (mdj_merge_host) */
} mdj_status;

typedef enum {
    MDJ_I32 = 1,
    MDJ_I64 = 2,
    MDJ_F32 = 3,
    MDJ_F64 = 4,
    MDJ_U32 = 5,
    MDJ_U64 = 6
} mdj_dtype;

/* One column: `data` is a device pointer to nrows elements of `dtype`. */
typedef struct {
    const void *data;
    int32_t dtype;
} mdj_col;

/* A table: `ncols` columns (1..MDJ_MAX_COLS), all with `nrows` rows. */
typedef struct {
    const mdj_col *cols;
    int32_t ncols;
    uint64_t nrows;
} mdj_table;

/* Device-memory allocator.  alloc returns a device pointer aligned to at least
 * 256 bytes (or NULL on failure) usable in stream order on `stream`;
 * release gives it back in stream order. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx, void *stream);
    void (*release)(void *ptr, void *ctx, void *stream);
    void *ctx;
} mdj_allocator;

/* A join result.  Every array has `nrows` elements and was obtained from the
 * allocator passed to the call (release it with mdj_result_release).
 *   key        : the join key (key dtype of the inputs)
 *   left_row   : 0-based row index in the left input table
 *   right_row  : 0-based row index in the right input table
 *   left_cols  : the left table's non-key columns, in table order
 *   right_cols : the right table's non-key columns, in table order
 * Row order is unspecified; the rows, as a multiset, are exactly the inner
 * equi-join (every pair (l, r) with key_L[l] == key_R[r], duplicates
 * included).  With nrows == 0 every pointer is NULL. */
typedef struct {
    uint64_t nrows;
    int32_t key_dtype;
    int32_t n_left_cols;
    int32_t n_right_cols;
    int32_t left_dtypes[MDJ_MAX_COLS];
    int32_t right_dtypes[MDJ_MAX_COLS];
    void *key;
    uint32_t *left_row;
    uint32_t *right_row;
    void *left_cols[MDJ_MAX_COLS];
    void *right_cols[MDJ_MAX_COLS];
} mdj_result;

/*
 * mdj_partition - the shuffle step (Sec. V-B, "Shuffle: True"; the exchange of
 * Sec. IV-B done on one device).  Stable hash partition of table `in` by column
 * `key_col` into P partitions.
 *   out_cols[j]   : caller-allocated device buffer of nrows elements of column
 *                   j's dtype; receives column j with the rows of partition 0
 *                   first, then partition 1, ...; inside a partition rows keep
 *                   their input order.
 *   out_row_ids   : caller-allocated device uint32[nrows]; out_row_ids[i] is
 *                   the input row now at position i.  May be NULL.
 *   out_offsets   : caller-allocated device int64[P+1]; partition p occupies
 *                   positions [out_offsets[p], out_offsets[p+1]).
 * Output buffers must not overlap the inputs.  1 <= P <= 65536.  nrows may be 0.
 * Workspace comes from `alloc` and is released before return (stream order).
 */
MDJ_API int mdj_partition(const mdj_table *in, int32_t key_col, uint32_t P,
                  void *const *out_cols, uint32_t *out_row_ids, int64_t *out_offsets,
                  const mdj_allocator *alloc, void *stream);

/*
 * mdj_partition_noalloc - mdj_partition for callers that cannot allocate.
 * The paper has no counterpart to this call; it exists for users of the
 * library.  Some callers may not call cudaMalloc or any other device
 * allocator where they need a partition: code that runs inside another
 * framework's memory pool which owns the device budget, loops where an
 * allocation could stall the device or fail half-way, or plugins that their
 * host process keeps away from the allocator.  They own their inputs and
 * outputs but cannot supply working memory, so this call takes its working
 * memory from a fixed array inside the library and allocates nothing
 * (no cudaMalloc / cudaMallocAsync / cudaFree, no allocator callback).
 *   Arguments and results are those of mdj_partition (same stable layout, same
 *   out_offsets), without the allocator.
 *   Limits: 1 <= P <= 1024, and the working set must fit the 16 MiB array:
 *   P * T + ceil(P * T / 4096) + P + 1 <= 4194304 words, T = ceil(nrows / 4096)
 *   (e.g. up to 16,764,928 rows at P = 1024, 2,146,951,168 rows at P = 8, and
 *   any nrows < 2^32 at P <= 2).  Larger
 *   inputs return MDJ_ERR_TOO_LARGE before any work; P > 1024 returns
 *   MDJ_ERR_INVALID_ARG.
 *   The array (16 MiB of device memory) is held on every GPU that loads the
 *   library until the process exits.  The first call on a device looks up the
 *   array's device address (a one-time set-up for that device, done with it
 *   current); make that first call before any stream capture.  All calls on a
 *   device share the one array and leave their data in it: calls whose GPU work
 *   can overlap (other streams, other threads) race and must be ordered by the
 *   caller.
 */
MDJ_API int mdj_partition_noalloc(const mdj_table *in, int32_t key_col, uint32_t P,
                                  void *const *out_cols, uint32_t *out_row_ids,
                                  int64_t *out_offsets, void *stream);

/*
 * mdj_join - the per-partition merge of the co-located partitions (the cuDF
 * merge step of Sec. V-B, after the shuffle).  Inner equi-join of `left` (build side)
 * and `right` (probe side) on left column `left_key` = right column
 * `right_key`, with no shuffle.  Internally the rows are bucketed by hash so
 * every hash table lives in one SM's shared memory; a count pass sizes the
 * output (one count read back to the host), a write pass fills it.
 * Outputs are allocated with `alloc` and described in *out.
 */
MDJ_API int mdj_join(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
             const mdj_allocator *alloc, void *stream, mdj_result *out);

/*
 * mdj_merge - the whole cuDF-merge hot path (Sec. V-B, Fig. 8: "Shuffle: True";
 * P emulates P workers): hash-partition both tables into P partitions (the
 * shuffle), then join every partition pair (left p with right p).  The result is
 * the same multiset of rows as mdj_join for every P.
 */
MDJ_API int mdj_merge(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
              uint32_t P, const mdj_allocator *alloc, void *stream, mdj_result *out);

/*
 * mdj_count_checksum - the merge of mdj_merge without materialising its rows,
 * for joins too large to store.  Returns (host pointers):
 *   *count    = number of joined pairs = sum over keys of lc(k) * rc(k);
 *   *checksum = sum over joined pairs (l, r) of f(l) * g(r) mod 2^64, with
 *     f(l) = fmix64(sext64(key_L[l]) ^ 0x9E3779B97F4A7C15 * (l + 1) ^ bits(lpay[l]))
 *     g(r) = fmix64(0xC2B2AE3D27D4EB4F * (r + 1) ^ bits(rpay[r]))
 *   where lpay / rpay is the first non-key column of each side (bits
 *   zero-extended to 64; 0 if the side has no other column) and l, r are
 *   0-based input row indices.
 * Synchronises `stream` before returning.
 */
MDJ_API int mdj_count_checksum(const mdj_table *left, int32_t left_key, const mdj_table *right,
                       int32_t right_key, uint32_t P, const mdj_allocator *alloc, void *stream,
                       uint64_t *count, uint64_t *checksum);

/* Tuning of the join tables and blocks (0 in a field = default). */
typedef struct {
    uint32_t table_rows;    /* build rows per shared-memory hash table, 256..8192 (default 4096) */
    uint32_t fill_pct;      /* target mean build rows per bucket, percent of table_rows, 10..100 (default 85) */
    uint32_t join_threads;  /* threads of a join block, 256 or 512 (default 512); each item probes
                               8 rows per thread, so this also sets the probe rows per item */
    uint32_t reserved[5];
} mdj_tuning;

/*
 * mdj_join_batch - many independent partition-pair merges (the per-partition
 * merge of Sec. V-B for every worker's pair at once) in a fixed number of
 * launches, however many pairs there are.  Pair i joins rows
 * [left_offsets[i], left_offsets[i+1]) of `left` with rows
 * [right_offsets[i], right_offsets[i+1]) of `right` (host arrays of npairs+1
 * nondecreasing offsets, first 0, last nrows).  Each pair is split into its
 * own hash buckets, all pairs' buckets are joined by one persistent kernel,
 * and the output holds pair 0's rows, then pair 1's, ...: pair i's rows are
 * [pair_offsets[i], pair_offsets[i+1]) (host array of npairs+1, filled by the
 * call).  left_row / right_row index the whole `left` / `right` tables.
 * Within a pair the rows are those of mdj_join on the pair's two slices.
 * `tuning` may be NULL.  Synchronises `stream` before returning.
 */
MDJ_API int mdj_join_batch(const mdj_table *left, int32_t left_key, const uint64_t *left_offsets,
                           const mdj_table *right, int32_t right_key, const uint64_t *right_offsets,
                           int32_t npairs, const mdj_tuning *tuning, const mdj_allocator *alloc,
                           void *stream, mdj_result *out, uint64_t *pair_offsets);

/*
 * mdj_merge_batch - many independent merge requests (the whole hot path of
 * Sec. V-B per request: shuffle into P[i] partitions, then join every
 * partition pair) in a fixed number of launches.  Request i's tables are rows
 * [left_offsets[i], left_offsets[i+1]) of `left` and [right_offsets[i],
 * right_offsets[i+1]) of `right`; its rows are hash partitioned into P[i]
 * partitions (1 <= P[i] <= 1024) inside its own region of the shuffled copy,
 * and the output holds request 0's rows, then request 1's, ...: request i's
 * rows are [req_offsets[i], req_offsets[i+1]) (host array of nreq+1, filled).
 * left_row / right_row index the whole `left` / `right` tables.  Within a
 * request the rows are those of mdj_merge on its two slices with P[i].
 * Synchronises `stream` before returning.
 */
MDJ_API int mdj_merge_batch(const mdj_table *left, int32_t left_key, const uint64_t *left_offsets,
                            const mdj_table *right, int32_t right_key, const uint64_t *right_offsets,
                            int32_t nreq, const uint32_t *P, const mdj_tuning *tuning,
                            const mdj_allocator *alloc, void *stream, mdj_result *out,
                            uint64_t *req_offsets);

/*
 * Streamed output: the join of mdj_merge written window by window into
 * buffers the caller owns, for results too large to hold at once (the
 * many-to-many merge of Sec. V-B with skewed keys, where one heavy key can
 * produce more rows than device memory holds).  The paper's runtime moves a
 * large message in bounded pieces (its 1 GB chunking of transfers, Sec. IV-B);
 * this is the same idea applied to the merge's output.
 *
 * mdj_stream_open - the merge of mdj_merge (shuffle into P partitions, then
 * every partition pair) up to its output: both tables are shuffled, in every
 * partition pair the build (left) rows are grouped by key, and every probe
 * (right) row learns its key's group.  That fixes an order on the join's
 * rows: right rows in shuffled order (the matching ones, or all with
 * MDJ_RIGHT / MDJ_OUTER), each followed through the left rows of its key,
 * then (MDJ_LEFT / MDJ_OUTER) the left rows no right row matched, grouped by
 * key.  Row q of that order is the same in every later window.
 *   how         : an mdj_how (else MDJ_ERR_INVALID_ARG)
 *   *out        : the handle (close it with mdj_stream_close)
 *   *total_rows : the number of joined rows (exact, 64-bit)
 * Skew is handled on either side with no special input: a key may have any
 * number of rows on either side.  The handle holds on the device the shuffled
 * right table (key, columns, uint32 row id), the grouped left row ids and
 * columns (and keys, for MDJ_LEFT / MDJ_OUTER), and 16 bytes per right row
 * plus, for MDJ_LEFT / MDJ_OUTER, 16 bytes per left row, until
 * mdj_stream_close.
 * The input tables must stay valid and unchanged until mdj_stream_close (with
 * P = 1 and a small left table the right table is read in place).  The
 * allocator struct is copied; its callbacks and ctx must stay valid until
 * mdj_stream_close.  Synchronises `stream`; later calls on the handle run on
 * that stream.  Errors: those of mdj_merge; on error *out is NULL.
 */
typedef struct mdj_stream mdj_stream;

/* Which rows a streamed join keeps (the usual merge variants):
 *   MDJ_INNER : matching pairs only
 *   MDJ_LEFT  : also every left row without a match, once, with no right row
 *   MDJ_RIGHT : also every right row without a match, once, with no left row
 *   MDJ_OUTER : both
 * A missing side has row id 0xFFFFFFFF (UINT32_MAX) and all-zero bits in its
 * columns; the key is the present side's. */
typedef enum { MDJ_INNER = 0, MDJ_LEFT = 1, MDJ_RIGHT = 2, MDJ_OUTER = 3 } mdj_how;

/* One window of output rows: device buffers owned by the caller, each with
 * room for the window's rows.  A NULL pointer skips that column.
 *   key, left_row, right_row, left_cols, right_cols : as in mdj_result (the
 *   columns of each side are its non-key columns in table order). */
typedef struct {
    void *key;
    uint32_t *left_row;
    uint32_t *right_row;
    void *left_cols[MDJ_MAX_COLS];
    void *right_cols[MDJ_MAX_COLS];
} mdj_window;

MDJ_API int mdj_stream_open(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
                            uint32_t P, int32_t how, const mdj_allocator *alloc, void *stream, mdj_stream **out,
                            uint64_t *total_rows);

/* Writes rows [first_row, first_row + nrows) of the handle's order into
 * out's buffers (element i of a buffer = row first_row + i).  Any window may
 * be written, in any order, any number of times; each call is one kernel
 * launch on the open stream and does not synchronise.  first_row + nrows
 * must not exceed total_rows (else MDJ_ERR_INVALID_ARG); nrows = 0 is a no-op. */
MDJ_API int mdj_stream_emit(mdj_stream *s, uint64_t first_row, uint64_t nrows, const mdj_window *out);

/* The resumable cursor: writes the next min(max_rows, rows left) rows after
 * the handle's cursor (initially 0) into out, reports them as
 * [*first_row, *first_row + *nrows) and advances the cursor; *nrows = 0 once
 * every row has been written. */
MDJ_API int mdj_stream_next(mdj_stream *s, uint64_t max_rows, const mdj_window *out, uint64_t *first_row,
                            uint64_t *nrows);

/* total_rows of the handle (0 for NULL). */
MDJ_API uint64_t mdj_stream_rows(const mdj_stream *s);

/* Releases every device buffer of the handle (stream order) and the handle. */
MDJ_API void mdj_stream_close(mdj_stream *s);

/*
 * mdj_merge_multi - the merge of mdj_merge on several key columns (a merge
 * variant: the key is the tuple of columns left_keys[a] = right_keys[a],
 * a < nkeys).  Inner join: every pair (l, r) whose tuples are equal column by
 * column.  Each tuple is hashed to a 64-bit surrogate, the surrogates are
 * merged as mdj_merge does (P partitions), and every candidate row's two
 * tuples are then compared, so hash collisions never reach the result.
 *   left_keys, right_keys : host arrays of nkeys distinct column indices
 *                           (1 <= nkeys <= 8); key columns are I32 / I64 /
 *                           U32 / U64, equal dtypes pairwise, compared as bits
 * The result has no `key` array (NULL, key_dtype 0): left_cols holds the left
 * key columns in left_keys order, then the left table's other columns in
 * table order; right_cols holds the right table's non-key columns.  Tables
 * may have at most MDJ_MAX_COLS - 1 columns.  Synchronises `stream`.
 */
MDJ_API int mdj_merge_multi(const mdj_table *left, const int32_t *left_keys, const mdj_table *right,
                            const int32_t *right_keys, int32_t nkeys, uint32_t P, const mdj_allocator *alloc,
                            void *stream, mdj_result *out);

/*
 * mdj_merge_multi_how - mdj_merge_multi for every join type (`how`: inner,
 * left, right or outer; a merge variant on key tuples).  The inner merge's
 * verified pairs come first; then, for left and outer, every left row that no
 * right row matches on the whole tuple, once; then, for right and outer,
 * every unmatched right row, once.  Layout as mdj_merge_multi: left_cols =
 * the key columns in left_keys order, then the left table's other columns;
 * right_cols = the right table's other columns.  A missing side has row id
 * 0xFFFFFFFF and all-zero bits in its columns, except that the key columns
 * of a right-only row hold that row's tuple (the key is the present side's,
 * as in mdj_stream_open).  Errors as mdj_merge_multi, and MDJ_ERR_INVALID_ARG
 * for another `how`.  Synchronises `stream`.
 */
MDJ_API int mdj_merge_multi_how(const mdj_table *left, const int32_t *left_keys, const mdj_table *right,
                                const int32_t *right_keys, int32_t nkeys, uint32_t P, int32_t how,
                                const mdj_allocator *alloc, void *stream, mdj_result *out);

/*
 * mdj_merge_host - the merge of HOST-resident tables that need not fit device
 * memory.  The paper's runtime sends messages above MPI's 2 GB count limit as
 * 1 GB chunks (Sec. IV-B); here the tables themselves pass through the device
 * in pieces bounded by `device_budget`:
 *   1. each table goes to the device in chunks; every chunk is hash
 *      partitioned into B buckets (bucket = h mod B, as mdj_partition) and
 *      returns to a host staging area with the rows' input row ids;
 *   2. for each bucket b, both tables' bucket b go to the device (bucket b + 1
 *      is copied in meanwhile), their merge is opened as a stream
 *      (mdj_stream_open with P and `how`; with one partition when P is a
 *      power of two no larger than B, since every row of the bucket would then
 *      share one partition), and its rows are written window by window; each
 *      window's row ids are mapped back to the input tables and the window is
 *      handed to `sink`.
 * When both tables together (with 4-byte row ids) take at most a seventh of
 * the budget, B = 1: phase 1 is skipped, each column goes to the device with
 * one copy, and an inner merge runs mdj_merge there and hands its result to
 * the sink in windows that point into it (other join types stream as in 2.).
 * Where the device reads pageable host memory directly, reads of host memory
 * are copy kernels and copies back go through the copy engines; elsewhere
 * every copy is a cudaMemcpyAsync.
 *   left, right   : tables whose column pointers are HOST pointers (pageable
 *                   or pinned), read only
 *   device_budget : bytes of device memory the call sizes its pieces for
 *                   (>= 64 MiB, else MDJ_ERR_INVALID_ARG): B, the chunk rows
 *                   and the window rows follow from it
 *   sink          : called once per window with a result whose arrays are
 *                   DEVICE pointers valid only during the call (copy what you
 *                   keep); first_row counts the rows handed over before it.
 *                   Returning non-zero stops the merge with MDJ_ERR_ABORTED.
 *   *total_rows   : rows handed to the sink
 * Row ids index the input tables; a missing side (outer joins) is
 * 0xFFFFFFFF as in mdj_stream_open.  Rows arrive bucket by bucket, each
 * bucket in its stream order.  All rows of one key share a bucket, so a key
 * whose rows exceed about a seventh of the budget gives MDJ_ERR_OOM.  Host
 * memory for the buckets (the tables' size again, plus 4 bytes per row) is
 * the library's own.  Synchronises `stream`.
 */
typedef int (*mdj_sink)(const mdj_result *piece, uint64_t first_row, void *ctx);

MDJ_API int mdj_merge_host(const mdj_table *left, int32_t left_key, const mdj_table *right, int32_t right_key,
                           uint32_t P, int32_t how, uint64_t device_budget, mdj_sink sink, void *sink_ctx,
                           const mdj_allocator *alloc, void *stream, uint64_t *total_rows);

/*
 * mdj_transpose_add - the paper's second application benchmark, the sum of an
 * array and its transpose (Sec. V-B "Sum of cuPy Array and its Transpose",
 * Fig. 7: 16K x 16K; Sec. V-C, Fig. 9(a): 20E3 x 20E3).  y = x + x^T for an
 * n x n row-major matrix: y[i][j] = x[i][j] + x[j][i].  In the paper the
 * array is split into chunks held by different Dask workers, so each output
 * chunk needs the mirrored chunk from another worker; on one GPU that is a
 * read of the mirrored tile.
 *   x, y  : device pointers to n * n elements of `dtype`, aligned to the
 *           element size; y may equal x (in place) but may not otherwise
 *           overlap it (MDJ_ERR_INVALID_ARG)
 *   dtype : MDJ_F64 / MDJ_F32 (one IEEE addition per element, so y is exact
 *           and symmetric), MDJ_I64 / MDJ_U64 / MDJ_I32 / MDJ_U32 (addition
 *           modulo 2^64 / 2^32)
 * n = 0 is a no-op; n >= 2^32 gives MDJ_ERR_TOO_LARGE.  Asynchronous on
 * `stream`; allocates nothing.
 */
MDJ_API int mdj_transpose_add(const void *x, void *y, uint64_t n, int32_t dtype, void *stream);

/* Releases every array of *res with `alloc` (stream order) and zeroes *res. */
MDJ_API void mdj_result_release(mdj_result *res, const mdj_allocator *alloc, void *stream);

/* Static, human-readable text for a status code. */
MDJ_API const char *mdj_status_string(int status);

/* Text of the CUDA error behind the calling thread's last MDJ_ERR_CUDA ("" if
 * none); valid until that thread's next call. */
MDJ_API const char *mdj_last_error(void);

/* MDJ_VERSION of the loaded library. */
MDJ_API int mdj_version(void);

/*
 * Per-kernel timing (tracing).  While enabled, every kernel the library
 * launches is bracketed by CUDA events recorded on the launch stream.
 * mdj_profile_collect synchronises those events and accumulates, per kernel
 * name, the launch count and total device milliseconds; mdj_profile_get reads
 * entry i (0 <= i < mdj_profile_count()).  Enabling adds two event records per
 * launch; it is off by default.
 */
MDJ_API void mdj_profile_enable(int on);
MDJ_API void mdj_profile_reset(void);
MDJ_API int mdj_profile_collect(void);
MDJ_API int mdj_profile_count(void);
MDJ_API int mdj_profile_get(int i, const char **name, uint64_t *launches, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* MDJ_H */
