/*
 * bcf_oracle.c -- CPU oracle for the bank-conflict-free merge sort library.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's shared object.  The GPU
 * library neither links, includes nor calls it, and the two share no code,
 * header, table or helper.
 *
 * What it computes.  Every operation here has a unique correct answer, so the
 * oracle is that answer's plain definition written out, not a restatement of
 * the GPU algorithm:
 *
 *   sort          "sort N keys" (Sec. 3, opening paragraph): the keys in
 *                 ascending (or descending) order; with payloads, the STABLE
 *                 order -- equal keys keep their input order in both
 *                 directions (the paper never discusses ties; stability is
 *                 the reading this library takes).
 *   merge_runs    "merge sorted sequences" (Sec. 3.2, "Binary merging";
 *                 Algorithm 6): merging k sorted runs stably, ties broken by
 *                 run index and then by position, is by definition the stable
 *                 sort of the runs concatenated in index order.
 *   segmented     the sort above applied to every segment [off[i], off[i+1])
 *                 independently.
 *   colored prefix sums (Appendix A): d independent prefix sums, one per
 *                 color, over a sequence of (value, color) elements.
 *
 * Method.  A top-down merge sort over a permutation array with one auxiliary
 * buffer (the textbook mergesort the paper builds on, Sec. 3 and Knuth vol. 3).
 * The merge step takes the element of the LEFT run unless the right one is
 * strictly smaller, which is what makes it stable.
 *
 * Key order.  u16, u32 and u64: the integers' natural order.  i16, i32 and
 * i64: C's signed comparison of the two's-complement values.  f32 and f64: IEEE 754
 * totalOrder (IEEE 754-2008 Sec. 5.10), written as a case analysis on sign and
 * magnitude bits: every negative-signed value precedes every positive-signed
 * one; among positive-signed values a larger magnitude field (exponent and
 * fraction, read as an unsigned integer) is larger; among negative-signed
 * values a larger magnitude field is smaller.  This puts -NaN < -inf < ... <
 * -0 < +0 < ... < +inf < +NaN and orders NaNs by payload.  Keys are moved
 * bit-for-bit; NaN payloads and the sign of zero are preserved.  The paper
 * sorts unsigned integers only (Sec. 4); the other types are the library's
 * extension and their orders are the standard ones named here.
 * Descending order reverses the key order only; ties still keep input order.
 *
 * nthreads > 1 is used only to time the oracle on all host cores: each thread
 * sorts one contiguous chunk with the same routine, then chunks are merged
 * pairwise with the same stable merge.  The single-thread path is the
 * correctness authority; tests check that both agree.
 *
 * Parity pins for this file are in tests/test_oracle_pins.py.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORACLE_U32 = 0, ORACLE_U64 = 1, ORACLE_F32 = 2, ORACLE_I32 = 3, ORACLE_I64 = 4,
       ORACLE_F64 = 5, ORACLE_U16 = 6, ORACLE_I16 = 7 };

typedef struct {
    const void* keys;
    int dtype;
    int descending;
} order_ctx;

/* IEEE 754 totalOrder on binary32 bit patterns: 1 if a strictly precedes b. */
static int f32_total_less(uint32_t a, uint32_t b)
{
    uint32_t sign_a = a >> 31, sign_b = b >> 31;
    uint32_t mag_a = a & 0x7FFFFFFFu, mag_b = b & 0x7FFFFFFFu;
    if (sign_a != sign_b)
        return sign_a == 1; /* the negative-signed one comes first */
    if (sign_a == 0)
        return mag_a < mag_b;
    return mag_a > mag_b;
}

/* IEEE 754 totalOrder on binary64 bit patterns: the same case analysis. */
static int f64_total_less(uint64_t a, uint64_t b)
{
    uint64_t neg_a = a >> 63, neg_b = b >> 63;
    uint64_t abs_a = a & 0x7FFFFFFFFFFFFFFFull, abs_b = b & 0x7FFFFFFFFFFFFFFFull;
    if (neg_a != neg_b)
        return neg_a == 1;
    if (neg_a == 0)
        return abs_a < abs_b;
    return abs_a > abs_b;
}

static size_t key_size(int dtype)
{
    if (dtype == ORACLE_U16 || dtype == ORACLE_I16)
        return 2;
    return (dtype == ORACLE_U64 || dtype == ORACLE_I64 || dtype == ORACLE_F64) ? 8 : 4;
}

static uint64_t key_bits(const order_ctx* c, uint64_t i)
{
    switch (key_size(c->dtype)) {
    case 8:  return ((const uint64_t*)c->keys)[i];
    case 2:  return ((const uint16_t*)c->keys)[i];
    default: return ((const uint32_t*)c->keys)[i];
    }
}

/* Strict "a goes before b" under the ascending key order of dtype. */
static int bits_less(int dtype, uint64_t a, uint64_t b)
{
    switch (dtype) {
    case ORACLE_F32: return f32_total_less((uint32_t)a, (uint32_t)b);
    case ORACLE_F64: return f64_total_less(a, b);
    case ORACLE_I32: return (int32_t)(uint32_t)a < (int32_t)(uint32_t)b;
    case ORACLE_I64: return (int64_t)a < (int64_t)b;
    case ORACLE_I16: return (int16_t)(uint16_t)a < (int16_t)(uint16_t)b;
    default:         return a < b;
    }
}

/* Strict precedence of the key at index i over the key at index j. */
static int precedes(const order_ctx* c, uint64_t i, uint64_t j)
{
    uint64_t a = key_bits(c, i), b = key_bits(c, j);
    return c->descending ? bits_less(c->dtype, b, a) : bits_less(c->dtype, a, b);
}

/* Stable merge of left[0..nl) and right[0..nr) into out. */
static void merge(const uint64_t* left, uint64_t nl, const uint64_t* right, uint64_t nr,
                  uint64_t* out, const order_ctx* c)
{
    uint64_t i = 0, j = 0, o = 0;
    while (i < nl && j < nr) {
        if (precedes(c, right[j], left[i]))
            out[o++] = right[j++];
        else
            out[o++] = left[i++];
    }
    while (i < nl) out[o++] = left[i++];
    while (j < nr) out[o++] = right[j++];
}

/* Top-down merge sort of perm[0..n), aux has room for n entries. */
static void merge_sort(uint64_t* perm, uint64_t* aux, uint64_t n, const order_ctx* c)
{
    if (n < 2)
        return;
    uint64_t half = n / 2;
    merge_sort(perm, aux, half, c);
    merge_sort(perm + half, aux + half, n - half, c);
    merge(perm, half, perm + half, n - half, aux, c);
    memcpy(perm, aux, n * sizeof(uint64_t));
}

/* ---- optional multi-threaded driver (timing only) ---------------------- */

typedef struct {
    uint64_t* perm;
    uint64_t* aux;
    uint64_t lo, mid, hi; /* sort: [lo, hi); merge: [lo, mid) + [mid, hi) */
    const order_ctx* c;
    int is_merge;
} task;

static void* run_task(void* p)
{
    task* t = (task*)p;
    if (!t->is_merge) {
        merge_sort(t->perm + t->lo, t->aux + t->lo, t->hi - t->lo, t->c);
    } else {
        merge(t->perm + t->lo, t->mid - t->lo, t->perm + t->mid, t->hi - t->mid,
              t->aux + t->lo, t->c);
        memcpy(t->perm + t->lo, t->aux + t->lo, (t->hi - t->lo) * sizeof(uint64_t));
    }
    return NULL;
}

static int sort_perm(uint64_t* perm, uint64_t n, const order_ctx* c, int nthreads)
{
    uint64_t* aux = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!aux)
        return -1;
    if (nthreads <= 1 || n < (uint64_t)nthreads * 1024) {
        merge_sort(perm, aux, n, c);
        free(aux);
        return 0;
    }
    int nt = nthreads;
    uint64_t* bounds = (uint64_t*)malloc((nt + 1) * sizeof(uint64_t));
    task* tasks = (task*)malloc(nt * sizeof(task));
    pthread_t* th = (pthread_t*)malloc(nt * sizeof(pthread_t));
    if (!bounds || !tasks || !th) {
        free(aux); free(bounds); free(tasks); free(th);
        return -1;
    }
    for (int i = 0; i <= nt; ++i)
        bounds[i] = n * (uint64_t)i / (uint64_t)nt;
    for (int i = 0; i < nt; ++i) {
        tasks[i] = (task){perm, aux, bounds[i], 0, bounds[i + 1], c, 0};
        pthread_create(&th[i], NULL, run_task, &tasks[i]);
    }
    for (int i = 0; i < nt; ++i)
        pthread_join(th[i], NULL);
    /* merge neighbouring chunks, doubling the chunk width each level */
    for (int width = 1; width < nt; width *= 2) {
        int m = 0;
        for (int i = 0; i + width < nt; i += 2 * width) {
            int hi = i + 2 * width < nt ? i + 2 * width : nt;
            tasks[m] = (task){perm, aux, bounds[i], bounds[i + width], bounds[hi], c, 1};
            pthread_create(&th[m], NULL, run_task, &tasks[m]);
            ++m;
        }
        for (int i = 0; i < m; ++i)
            pthread_join(th[i], NULL);
    }
    free(aux); free(bounds); free(tasks); free(th);
    return 0;
}

static void gather(void* keys_out, uint32_t* vals_out, const void* keys_in,
                   const uint32_t* vals_in, const uint64_t* perm, uint64_t n, int dtype)
{
    size_t ks = key_size(dtype);
    for (uint64_t i = 0; i < n; ++i) {
        memcpy((char*)keys_out + i * ks, (const char*)keys_in + perm[i] * ks, ks);
        if (vals_out)
            vals_out[i] = vals_in[perm[i]];
    }
}

/* ---- exported entry points -------------------------------------------- */

/* Strict ascending-order test on raw key bits; exported for the order pins. */
int oracle_key_less(int dtype, uint64_t a, uint64_t b)
{
    return bits_less(dtype, a, b);
}

/* Stable sort of n keys (+ optional u32 payloads).  Returns 0, or -1 on bad
 * arguments / allocation failure.  Output buffers must not alias inputs. */
int oracle_sort(void* keys_out, uint32_t* vals_out, const void* keys_in,
                const uint32_t* vals_in, uint64_t n, int dtype, int descending, int nthreads)
{
    if (dtype < ORACLE_U32 || dtype > ORACLE_I16)
        return -1;
    if ((vals_out == NULL) != (vals_in == NULL))
        return -1;
    if (n == 0)
        return 0;
    uint64_t* perm = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!perm)
        return -1;
    for (uint64_t i = 0; i < n; ++i)
        perm[i] = i;
    order_ctx c = {keys_in, dtype, descending};
    if (sort_perm(perm, n, &c, nthreads) != 0) {
        free(perm);
        return -1;
    }
    gather(keys_out, vals_out, keys_in, vals_in, perm, n, dtype);
    free(perm);
    return 0;
}

/* Stable k-way merge of the sorted runs [off[r], off[r+1]) for r < k: the
 * stable sort of their concatenation in run order. */
int oracle_merge_runs(void* keys_out, uint32_t* vals_out, const void* keys_in,
                      const uint32_t* vals_in, const uint64_t* run_offsets, uint32_t k,
                      int dtype, int descending)
{
    if (k == 0)
        return 0;
    for (uint32_t r = 0; r < k; ++r)
        if (run_offsets[r + 1] < run_offsets[r])
            return -1;
    uint64_t lo = run_offsets[0], n = run_offsets[k] - run_offsets[0];
    size_t ks = key_size(dtype);
    return oracle_sort((char*)keys_out + lo * ks, vals_out ? vals_out + lo : NULL,
                       (const char*)keys_in + lo * ks, vals_in ? vals_in + lo : NULL,
                       n, dtype, descending, 1);
}

/* Stable sort of every segment [off[s], off[s+1]) for s < nseg. */
int oracle_segmented_sort(void* keys_out, uint32_t* vals_out, const void* keys_in,
                          const uint32_t* vals_in, const uint64_t* seg_offsets, uint64_t nseg,
                          int dtype, int descending)
{
    size_t ks = key_size(dtype);
    for (uint64_t s = 0; s < nseg; ++s) {
        uint64_t lo = seg_offsets[s], hi = seg_offsets[s + 1];
        if (hi < lo)
            return -1;
        int rc = oracle_sort((char*)keys_out + lo * ks, vals_out ? vals_out + lo : NULL,
                             (const char*)keys_in + lo * ks, vals_in ? vals_in + lo : NULL,
                             hi - lo, dtype, descending, 1);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* ---- colored prefix sums ------------------------------------------------ */

/* Colored prefix sums (Appendix A; the experiment of Sec. 2.2): every element
 * i carries a value v[i] and a color c[i] in [0, d); out[i] is the sum of the
 * values of the elements of color c[i] at positions <= i (inclusive) or < i
 * (exclusive), i.e. d independent prefix sums, one per color.  Sums are taken
 * modulo 2^32 (unsigned 32-bit arithmetic).  Plain definition, one running
 * sum per color.  Returns 0, or -1 for a color >= d or d outside [1, 256]. */
int oracle_colored_prefix_sums(uint32_t* out, const uint32_t* values, const uint8_t* colors,
                               uint64_t n, uint32_t d, int exclusive)
{
    if (d < 1 || d > 256)
        return -1;
    uint32_t acc[256];
    for (uint32_t c = 0; c < d; ++c)
        acc[c] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t c = colors[i];
        if (c >= d)
            return -1;
        if (exclusive) {
            out[i] = acc[c];
            acc[c] += values[i];
        } else {
            acc[c] += values[i];
            out[i] = acc[c];
        }
    }
    return 0;
}
