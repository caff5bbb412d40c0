/*
 * CPU oracle for the hash-partitioned shuffle + inner equi-join ("cuDF merge",
 * Sec. V-B "cuDF Merge" and Fig. 8 / Fig. 9(b,c) of arXiv 2101.08878).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may call this file.  Only the tests, the package's smoke
 * entry point and the CPU-baseline leg of the benchmark use it.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * The paper's benchmark merges cuDF data frames after a shuffle (Sec. V-B,
 * Fig. 8 settings "Shuffle: True, Fraction Match: 0.3") but prints no
 * algorithm, hash or output schema.  This file therefore writes out the plain
 * definitions of what the method computes:
 *
 *   partition  - every row goes to partition p = fmix64(sext64(key)) mod P,
 *                rows keep their original order inside a partition (a stable
 *                counting sort).  fmix64 is the 64-bit finalizer of Austin
 *                Appleby's MurmurHash3 (public domain), written here from its
 *                description: xor-shift by 33, multiply, xor-shift by 33,
 *                multiply, xor-shift by 33.
 *   merge      - the inner equi-join: every pair (l, r) with key_L[l] == key_R[r],
 *                emitted in canonical order (key, l, r).  Computed as a
 *                sort-merge join: sort each side's (key, row) pairs, walk equal
 *                key runs, emit the cross product of each matching run.
 *   count_checksum - count = sum over keys of lc(k) * rc(k); checksum =
 *                sum over joined pairs of f(l) * g(r) mod 2^64, computed per key
 *                group as (sum of f over the group) * (sum of g over the group).
 *
 * Integer arithmetic only; payloads are never interpreted, only their bits are
 * read (for the checksum).  Row indices are 0-based positions in the inputs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- hashing */

/* MurmurHash3 64-bit finalizer (fmix64). */
uint64_t oracle_fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* Key i of a column of 4-byte or 8-byte signed integers, sign-extended to 64
 * bits, so that equal values of int32 and int64 columns compare and hash equal. */
static int64_t key_at(const void *keys, int key_bytes, uint64_t i)
{
    if (key_bytes == 4)
        return (int64_t)((const int32_t *)keys)[i];
    return ((const int64_t *)keys)[i];
}

/* Partition id of one key: p = fmix64(sext64(key)) mod P (unsigned). */
uint32_t oracle_partition_of(int64_t key, uint32_t P)
{
    return (uint32_t)(oracle_fmix64((uint64_t)key) % (uint64_t)P);
}

/* ------------------------------------------------------------- partition */

/*
 * Stable partition (counting sort by partition id).
 *   offsets[P+1]: offsets[p] = first output position of partition p,
 *                 offsets[P] = n.
 *   perm[n]:      perm[j] = input row placed at output position j.
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_partition(const void *keys, int key_bytes, uint64_t n, uint32_t P,
                     int64_t *offsets, uint32_t *perm)
{
    if (P == 0 || (key_bytes != 4 && key_bytes != 8))
        return -1;
    int64_t *cursor = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
    uint32_t *pid = (uint32_t *)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    if (!cursor || !pid) {
        free(cursor);
        free(pid);
        return -1;
    }
    /* 1. partition id and count of every partition */
    for (uint64_t i = 0; i < n; i++) {
        pid[i] = oracle_partition_of(key_at(keys, key_bytes, i), P);
        cursor[pid[i]] += 1;
    }
    /* 2. exclusive prefix sum of the counts = partition offsets */
    int64_t run = 0;
    for (uint32_t p = 0; p < P; p++) {
        int64_t c = cursor[p];
        offsets[p] = run;
        cursor[p] = run;
        run += c;
    }
    offsets[P] = run;
    /* 3. place rows in input order (stable) */
    for (uint64_t i = 0; i < n; i++)
        perm[cursor[pid[i]]++] = (uint32_t)i;
    free(cursor);
    free(pid);
    return 0;
}

/* ------------------------------------------------------------ sort-merge */

typedef struct {
    int64_t key;
    uint32_t row;
} key_row;

static int cmp_key_row(const void *a, const void *b)
{
    const key_row *x = (const key_row *)a, *y = (const key_row *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    if (x->row != y->row)
        return x->row < y->row ? -1 : 1;
    return 0;
}

/* (key, row) pairs of one side sorted by key, then row. */
static key_row *sorted_side(const void *keys, int key_bytes, uint64_t n)
{
    key_row *s = (key_row *)malloc((size_t)(n ? n : 1) * sizeof(key_row));
    if (!s)
        return NULL;
    for (uint64_t i = 0; i < n; i++) {
        s[i].key = key_at(keys, key_bytes, i);
        s[i].row = (uint32_t)i;
    }
    qsort(s, (size_t)n, sizeof(key_row), cmp_key_row);
    return s;
}

/*
 * Inner equi-join by sort-merge.  Writes at most `cap` pairs in canonical order
 * (key, left row, right row) and sets *m to the full pair count (which may be
 * larger than cap: call once with cap = 0 to size the output).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_merge(const void *lkeys, uint64_t nl, const void *rkeys, uint64_t nr,
                 int key_bytes, uint32_t *out_lrow, uint32_t *out_rrow,
                 uint64_t cap, uint64_t *m)
{
    if (key_bytes != 4 && key_bytes != 8)
        return -1;
    key_row *L = sorted_side(lkeys, key_bytes, nl);
    key_row *R = sorted_side(rkeys, key_bytes, nr);
    if (!L || !R) {
        free(L);
        free(R);
        return -1;
    }
    uint64_t i = 0, j = 0, out = 0;
    while (i < nl && j < nr) {
        if (L[i].key < R[j].key) {
            i++;
        } else if (L[i].key > R[j].key) {
            j++;
        } else {
            /* equal-key runs [i, ie) and [j, je) */
            int64_t k = L[i].key;
            uint64_t ie = i, je = j;
            while (ie < nl && L[ie].key == k)
                ie++;
            while (je < nr && R[je].key == k)
                je++;
            for (uint64_t a = i; a < ie; a++)
                for (uint64_t b = j; b < je; b++) {
                    if (out < cap) {
                        out_lrow[out] = L[a].row;
                        out_rrow[out] = R[b].row;
                    }
                    out++;
                }
            i = ie;
            j = je;
        }
    }
    *m = out;
    free(L);
    free(R);
    return 0;
}

/* ------------------------------------------------------- count + checksum */

/* Bits of payload value i (4- or 8-byte column), zero-extended to 64 bits. */
static uint64_t pay_bits(const void *pay, int pay_bytes, uint64_t i)
{
    if (pay_bytes == 4)
        return (uint64_t)((const uint32_t *)pay)[i];
    return ((const uint64_t *)pay)[i];
}

/* Per-left-row term f(l) = fmix64(sext64(key) ^ A*(l+1) ^ bits(lpay[l])). */
uint64_t oracle_checksum_f(int64_t key, uint32_t lrow, uint64_t lpay_bits)
{
    return oracle_fmix64((uint64_t)key ^ (0x9E3779B97F4A7C15ULL * ((uint64_t)lrow + 1)) ^
                         lpay_bits);
}

/* Per-right-row term g(r) = fmix64(B*(r+1) ^ bits(rpay[r])). */
uint64_t oracle_checksum_g(uint32_t rrow, uint64_t rpay_bits)
{
    return oracle_fmix64((0xC2B2AE3D27D4EB4FULL * ((uint64_t)rrow + 1)) ^ rpay_bits);
}

/*
 * count = number of joined pairs = sum over keys k of lc(k) * rc(k);
 * checksum = sum over joined pairs (l, r) of f(l) * g(r)  (mod 2^64)
 *          = sum over keys k of (sum_{l in k} f(l)) * (sum_{r in k} g(r)).
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int oracle_count_checksum(const void *lkeys, const void *lpay, int lpay_bytes, uint64_t nl,
                          const void *rkeys, const void *rpay, int rpay_bytes, uint64_t nr,
                          int key_bytes, uint64_t *count, uint64_t *checksum)
{
    if (key_bytes != 4 && key_bytes != 8)
        return -1;
    key_row *L = sorted_side(lkeys, key_bytes, nl);
    key_row *R = sorted_side(rkeys, key_bytes, nr);
    if (!L || !R) {
        free(L);
        free(R);
        return -1;
    }
    uint64_t i = 0, j = 0, cnt = 0, sum = 0;
    while (i < nl && j < nr) {
        if (L[i].key < R[j].key) {
            i++;
        } else if (L[i].key > R[j].key) {
            j++;
        } else {
            int64_t k = L[i].key;
            uint64_t lc = 0, rc = 0, F = 0, G = 0;
            while (i < nl && L[i].key == k) {
                F += oracle_checksum_f(k, L[i].row, pay_bits(lpay, lpay_bytes, L[i].row));
                lc++;
                i++;
            }
            while (j < nr && R[j].key == k) {
                G += oracle_checksum_g(R[j].row, pay_bits(rpay, rpay_bytes, R[j].row));
                rc++;
                j++;
            }
            cnt += lc * rc;
            sum += F * G;
        }
    }
    *count = cnt;
    *checksum = sum;
    free(L);
    free(R);
    return 0;
}

/* ------------------------------------------------------- array helpers */

/* out[i] = fmix64(in[i]) for i < n. */
void oracle_fmix64_array(const uint64_t *in, uint64_t n, uint64_t *out)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = oracle_fmix64(in[i]);
}

/* out[i] = partition id of key i (see oracle_partition_of). */
void oracle_partition_ids(const void *keys, int key_bytes, uint64_t n, uint32_t P, uint32_t *out)
{
    for (uint64_t i = 0; i < n; i++)
        out[i] = oracle_partition_of(key_at(keys, key_bytes, i), P);
}

/* f(l) for every row of a left table and g(r) for every row of a right table. */
void oracle_checksum_terms(const void *lkeys, int key_bytes, const void *lpay, int lpay_bytes,
                           uint64_t nl, const void *rpay, int rpay_bytes, uint64_t nr,
                           uint64_t *f, uint64_t *g)
{
    for (uint64_t i = 0; i < nl; i++)
        f[i] = oracle_checksum_f(key_at(lkeys, key_bytes, i), (uint32_t)i,
                                 pay_bits(lpay, lpay_bytes, i));
    for (uint64_t i = 0; i < nr; i++)
        g[i] = oracle_checksum_g((uint32_t)i, pay_bits(rpay, rpay_bytes, i));
}

/*
 * count + checksum for keys known to lie in [0, K): per-key sums in arrays
 * (lc, rc, F = sum of f, G = sum of g), then count = sum_k lc*rc and
 * checksum = sum_k F*G (mod 2^64).  Same definitions as
 * oracle_count_checksum, computed without sorting, for large skewed inputs.
 * Returns 0, or -1 on a key outside [0, K) or allocation failure.
 */
int oracle_count_checksum_dense(const void *lkeys, const void *lpay, int lpay_bytes, uint64_t nl,
                                const void *rkeys, const void *rpay, int rpay_bytes, uint64_t nr,
                                int key_bytes, uint64_t K, uint64_t *count, uint64_t *checksum)
{
    if ((key_bytes != 4 && key_bytes != 8) || K == 0)
        return -1;
    uint64_t *lc = (uint64_t *)calloc(K, sizeof(uint64_t));
    uint64_t *rc = (uint64_t *)calloc(K, sizeof(uint64_t));
    uint64_t *F = (uint64_t *)calloc(K, sizeof(uint64_t));
    uint64_t *G = (uint64_t *)calloc(K, sizeof(uint64_t));
    int rcode = 0;
    if (!lc || !rc || !F || !G) {
        rcode = -1;
        goto done;
    }
    for (uint64_t i = 0; i < nl; i++) {
        int64_t k = key_at(lkeys, key_bytes, i);
        if (k < 0 || (uint64_t)k >= K) {
            rcode = -1;
            goto done;
        }
        lc[k] += 1;
        F[k] += oracle_checksum_f(k, (uint32_t)i, pay_bits(lpay, lpay_bytes, i));
    }
    for (uint64_t i = 0; i < nr; i++) {
        int64_t k = key_at(rkeys, key_bytes, i);
        if (k < 0 || (uint64_t)k >= K) {
            rcode = -1;
            goto done;
        }
        rc[k] += 1;
        G[k] += oracle_checksum_g((uint32_t)i, pay_bits(rpay, rpay_bytes, i));
    }
    {
        uint64_t cnt = 0, sum = 0;
        for (uint64_t k = 0; k < K; k++) {
            cnt += lc[k] * rc[k];
            sum += F[k] * G[k];
        }
        *count = cnt;
        *checksum = sum;
    }
done:
    free(lc);
    free(rc);
    free(F);
    free(G);
    return rcode;
}
