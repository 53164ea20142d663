/*
 * bcfsort.h -- C ABI of the GB300 bank-conflict-free comparison merge sort.
 *
 * The library implements the hot path of Sitchinava & Weichert, "Bank Conflict
 * Free Comparison-based Sorting On GPUs" (arXiv 1306.5076): a shared-memory
 * block sort with no bank conflicts (Sec. 3.1) followed by BCFMergesort's
 * global merge passes (Sec. 3.2, Lemma 2), redesigned for sm_103a.
 *
 * Conventions shared by every call below
 * --------------------------------------
 *  - Memory.  Every key / value pointer is DEVICE memory owned by the caller
 *    and must be 16-byte aligned when the element count is non-zero.  Keys are
 *    arrays of the key type (2 bytes for BCF_U16 / BCF_I16, 4 for BCF_U32 /
 *    BCF_I32 / BCF_F32, 8 for BCF_U64 / BCF_I64 / BCF_F64);
 *    values are uint32_t arrays of the same length.  Arrays are contiguous.
 *  - Workspace.  The library allocates nothing on the sort path.  Calls that
 *    need scratch take a caller-provided device workspace `ws` of at least
 *    bcf_workspace_bytes(...) bytes, 256-byte aligned.  Its contents on entry
 *    are irrelevant and on return undefined.
 *  - Aliasing.  keys_out == keys_in (and vals_out == vals_in) is allowed; any
 *    other overlap between an output and an input, or with `ws`, is BCF_EINVAL.
 *  - Asynchrony.  Calls enqueue work on `stream` and return after launching;
 *    results are valid once the stream has reached that point.  Errors that
 *    can be seen on the host (null pointers, misalignment, short workspace,
 *    bad dtype, decreasing offsets) are returned before anything is launched.
 *    A launch failure returns BCF_ECUDA.  Device-side bounded waits that run
 *    out set a device error word that bcf_last_device_error() reports.
 *  - Order.  Keys are compared after an order-preserving map to unsigned
 *    integers: u16 / u32 / u64 as-is, i16 / i32 / i64 in two's-complement
 *    order, f32 / f64 under IEEE 754 totalOrder
 *    (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN).  Keys are returned
 *    bit-for-bit (NaN payloads and the sign of zero survive).  Descending
 *    order reverses the key order; ties ALWAYS keep input order (stable), in
 *    both directions.  The paper sorts integer keys and never discusses ties
 *    or floats; stability and totalOrder are this library's reading.
 *  - Edge sizes.  n == 0 is a no-op returning BCF_OK; n == 1 copies.
 *  - Determinism.  The output is a function of the input alone: it does not
 *    depend on the stream, tuning parameters or what else runs on the GPU.
 *  - Threads.  Calls may be made from several host threads at once as long as
 *    they use different workspaces.
 */
#ifndef BCFSORT_H
#define BCFSORT_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key types.  The paper sorts unsigned integers (Sec. 4) and is silent on any
 * other type; the signed and floating-point orders are this library's
 * extension, each reduced to an unsigned order by a bijective map applied when
 * a key is first loaded and undone when it is last stored. */
typedef enum {
    BCF_U32 = 0, /* uint32_t, natural order */
    BCF_U64 = 1, /* uint64_t, natural order */
    BCF_F32 = 2, /* IEEE 754 binary32, totalOrder */
    BCF_I32 = 3, /* int32_t, two's-complement order */
    BCF_I64 = 4, /* int64_t, two's-complement order */
    BCF_F64 = 5, /* IEEE 754 binary64, totalOrder */
    BCF_U16 = 6, /* uint16_t, natural order (sorted as zero-extended 32-bit keys) */
    BCF_I16 = 7  /* int16_t, two's-complement order (sorted as sign-extended i32) */
} bcf_dtype;

typedef enum {
    BCF_OK = 0,
    BCF_EINVAL = 1,       /* bad argument, detected on the host before any launch */
    BCF_ENOMEM = 2,       /* workspace smaller than bcf_workspace_bytes() */
    BCF_ECUDA = 3,        /* a CUDA launch or runtime call failed */
    BCF_ETIMEOUT = 4,     /* a device-side bounded wait ran out (see bcf_last_device_error) */
    BCF_EUNSUPPORTED = 5  /* valid request this library does not handle (e.g. too many segments) */
} bcf_status;

/* Sorting algorithms (bcf_opts.algorithm).  Both give the identical, stable
 * result; they differ in speed by input distribution. */
enum {
    BCF_ALGO_MERGE = 0,        /* block sort + ceil(log2(n / T)) merge passes (Sec. 3.2) */
    BCF_ALGO_PIVOT_BUCKETS = 1, /* BCFMergesortPB (Sec. 3.2, "Duplicate keys"): the block
                                * sort, then a distribution into 255 splitter buckets
                                * plus one bucket per splitter for the keys equal to it;
                                * the equal buckets are final, the others are sorted by
                                * the segmented sort.  Fastest on duplicate-heavy keys;
                                * needs bcf_workspace_bytes(BCF_OP_SORT_PB, ...) and
                                * n < 2^32 (larger n takes the merge path). */
    BCF_ALGO_AUTO = 2          /* one of the two, chosen per call: a sample of at least
                                * 16384 keys (every 256th to every 4096th key) is sorted,
                                * splitters are picked from it as pivot buckets would,
                                * and pivot buckets are taken when at least 1/3 of the
                                * sample keys, not counting the splitters' own
                                * occurrences, equal a splitter (those keys would be
                                * final after one distribution), else the merge path.
                                * Needs the BCF_OP_SORT_PB workspace.  The decision reads
                                * two words back to the host, so the call synchronises
                                * `stream` once (not for graph capture). */
};

typedef struct {
    int descending;      /* 0: ascending, 1: descending (ties keep input order) */
    int stable_required; /* accepted for API symmetry; output is always stable */
    int algorithm;       /* BCF_ALGO_MERGE (default), BCF_ALGO_PIVOT_BUCKETS or BCF_ALGO_AUTO */
} bcf_opts;              /* a NULL bcf_opts* means ascending, BCF_ALGO_MERGE */

/* Operation codes for bcf_workspace_bytes. */
enum { BCF_OP_SORT = 0, BCF_OP_MERGE = 1, BCF_OP_SEGMENTED = 2, BCF_OP_CPS = 3,
       BCF_OP_SORT_PB = 4, BCF_OP_SORT_HOST = 5, BCF_OP_SORT_HOST_PB = 6, BCF_OP_SORT_WIDE = 7 };

/*
 * Workspace size in bytes for an operation.
 *   op        BCF_OP_SORT: sort n keys (pairs if has_vals);
 *             BCF_OP_MERGE: merge nseg_or_k runs totalling n keys;
 *             BCF_OP_SEGMENTED: nseg_or_k segments totalling n keys;
 *             BCF_OP_CPS: colored prefix sums of n elements with nseg_or_k
 *             colors (kt must be BCF_U32, has_vals 0);
 *             BCF_OP_SORT_PB: sort n keys with BCF_ALGO_PIVOT_BUCKETS or
 *             BCF_ALGO_AUTO (pairs if has_vals; also enough for BCF_ALGO_MERGE);
 *             BCF_OP_SORT_HOST / BCF_OP_SORT_HOST_PB: bcf_sort_*_host with the
 *             merge / pivot-bucket algorithm;
 *             BCF_OP_SORT_WIDE: bcf_sort_pairs_wide (either algorithm; the
 *             payload width does not matter).
 * Returns 0 for an unknown op or dtype.  The size is about one extra copy of
 * the keys (+ values) -- the merge is not in place, as in the paper (Sec. 4
 * remarks that BCFMergesort needs less extra space than its competitors) --
 * plus O(n / tile) split points and a small header.
 */
size_t bcf_workspace_bytes(int op, uint64_t n, uint64_t nseg_or_k, bcf_dtype kt, int has_vals);

/*
 * Sort n keys.  "Sort N keys" is the problem of Sec. 3; the method is the
 * base-case block sort (Sec. 3.1) followed by ceil(log2(n / T)) global merge
 * passes (Sec. 3.2, Lemma 2), T being the block tile of bcf_sort_plan().
 *   keys_out  device, n keys, written with the sorted keys (may equal keys_in)
 *   keys_in   device, n keys, read only
 * Errors: BCF_EINVAL (null pointer with n > 0, misalignment, bad dtype,
 * partial overlap), BCF_ENOMEM (ws too small), BCF_ECUDA.
 */
bcf_status bcf_sort_keys(void* keys_out, const void* keys_in, uint64_t n, bcf_dtype kt,
                         const bcf_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Stable sort of n (key, value) pairs: values follow their keys, and pairs
 * with equal keys keep their input order.  Same method and errors as
 * bcf_sort_keys.  vals_out may equal vals_in.
 */
bcf_status bcf_sort_pairs(void* keys_out, uint32_t* vals_out, const void* keys_in,
                          const uint32_t* vals_in, uint64_t n, bcf_dtype kt,
                          const bcf_opts* opts, void* ws, size_t ws_bytes, cudaStream_t stream);

/*
 * Merge k sorted runs into one sorted array ("merge sorted sequences",
 * Sec. 3.2, Algorithm 6; the final merge phase merges many runs per bucket).
 * Run r occupies [run_offsets_host[r], run_offsets_host[r+1]) of keys_in;
 * offsets are HOST memory, k+1 entries, non-decreasing, run_offsets_host[0]
 * is usually 0 and the output covers the same index range.  Each run must be
 * sorted under the requested order (a precondition that is not checked, as
 * in Algorithm 6).  Ties are broken by run index, then position.  Runs are
 * merged pairwise in a balanced tree of ceil(log2 k) passes.
 *   vals_in / vals_out  NULL for keys only (both or neither).
 * Errors: as bcf_sort_keys, plus BCF_EINVAL for decreasing offsets or k == 0.
 */
bcf_status bcf_merge_runs(void* keys_out, uint32_t* vals_out, const void* keys_in,
                          const uint32_t* vals_in, const uint64_t* run_offsets_host, uint32_t k,
                          bcf_dtype kt, const bcf_opts* opts, void* ws, size_t ws_bytes,
                          cudaStream_t stream);

/*
 * Sort each of nseg segments independently (the paper's "segmented" sorts are
 * intra-tile only, Sec. 3.1 and Algorithm 5; sorting many independent arrays
 * in one launch is this library's batching extension).  Segment s occupies
 * [seg_offsets_dev[s], seg_offsets_dev[s+1]) of keys_in; offsets are DEVICE
 * memory, nseg+1 non-decreasing uint64 entries with seg_offsets_dev[nseg] ==
 * n_total.  vals may be NULL (both or neither).  Offsets are read on the
 * device; a decreasing offset is not detected on the host and yields an
 * unspecified (but memory-safe) result.  n_total may exceed 2^32 (and one
 * segment may be that long); nseg must be below 2^32 (BCF_EUNSUPPORTED
 * otherwise).  The call makes two launches: a plan and one persistent wave
 * that sorts tiny segments and tiles and, by default, also runs the merge
 * passes.  Where the tuning table's segmented row for the size band names a
 * merge configuration, the wave only sorts, and the merge passes of segments
 * of two or more tiles follow as one partition and one merge launch per
 * possible pass count, ceil(log2((n_total - 1) / T + 2)) pairs for sort tile
 * T; a pair with no segment that long finds no work.  The launch sequence is
 * fixed by the arguments, so the call can be captured in a CUDA graph; ws is
 * sized by bcf_workspace_bytes(BCF_OP_SEGMENTED, n_total, nseg, kt, has_vals).
 */
bcf_status bcf_segmented_sort(void* keys_out, uint32_t* vals_out, const void* keys_in,
                              const uint32_t* vals_in, const uint64_t* seg_offsets_dev,
                              uint64_t nseg, uint64_t n_total, bcf_dtype kt,
                              const bcf_opts* opts, void* ws, size_t ws_bytes,
                              cudaStream_t stream);

/* Human-readable name of a status code (static string, never NULL). */
const char* bcf_status_string(bcf_status status);

/*
 * Synchronise `stream`, then read and clear the current device's error word.
 * After BCF_ETIMEOUT the outputs of the calls that ran since the last check are
 * undefined.  When the wait that ran out was a merge pass's wait for its bulk
 * copies, copies still in flight when the CTA gave up may land in shared
 * memory that a later CTA on that SM already uses, so the results of OTHER
 * launches that ran on the device at the same time are undefined as well.
 * Returns BCF_ETIMEOUT if a kernel's bounded wait ran out since the last call,
 * BCF_EINVAL if the only error seen was a color >= d in
 * bcf_colored_prefix_sums, BCF_ECUDA if the synchronisation failed, else
 * BCF_OK.
 */
bcf_status bcf_last_device_error(cudaStream_t stream);

/*
 * Self-test of the failure path: one thread waits, bounded by limit_us
 * microseconds of the GPU's global timer, for a device flag that nothing ever
 * sets -- the same bounded wait the library's kernels use -- then records a
 * wait that ran out in the device error word and exits.  The caller then sees
 * BCF_ETIMEOUT from bcf_last_device_error(stream), and the context stays
 * usable.  BCF_EINVAL for limit_us == 0 or above 2,000,000.
 */
bcf_status bcf_selftest_bounded_wait(uint32_t limit_us, cudaStream_t stream);

/*
 * Limit of every device-side bounded wait the library's kernels make (the
 * merge pass's wait for its bulk copies, the segmented sort's wait for a work
 * item to be published, the colored prefix sums' look-back), in microseconds
 * of the GPU's global timer.  0 restores the default of 2,000,000 (2 s);
 * BCF_EINVAL above 60,000,000.  Process-wide; a launch uses the value set when
 * it is enqueued.  No wait of a correct run comes near the default: the limit
 * only bounds how long a kernel can hang before it reports BCF_ETIMEOUT.
 * bcf_wait_limit_us() returns the current value.
 */
bcf_status bcf_set_wait_limit_us(uint32_t limit_us);
uint32_t bcf_wait_limit_us(void);

/*
 * Self-test of the segmented sort's own bounded wait.  One CTA of the real
 * segmented-sort worker (32-bit keys) runs on a work queue that announces one
 * item whose slot the host set-up leaves unpublished, so the worker's wait for
 * it runs out after the current wait limit (bcf_set_wait_limit_us).  The
 * worker then records the timeout in the device error word and exits without
 * reading or writing any keys; bcf_last_device_error(stream) returns
 * BCF_ETIMEOUT and the context stays usable.
 *   ws  device scratch of at least 512 bytes, 256-byte aligned (BCF_ENOMEM if
 *       smaller or NULL, BCF_EINVAL if misaligned); its contents are
 *       overwritten.
 */
bcf_status bcf_selftest_segmented_wait(void* ws, size_t ws_bytes, cudaStream_t stream);

/* ---- plan introspection and building blocks ------------------------------ */

typedef struct {
    uint32_t block_tile;   /* T: keys per CTA in the block sort (Sec. 3.1 "M") */
    uint32_t merge_tile;   /* output keys per CTA in a merge pass */
    uint32_t merge_passes; /* ceil(log2(n / T)) global merge passes (Lemma 2) */
    uint32_t launches;     /* kernel launches one bcf_sort_* call makes */
    uint64_t bytes_per_pass; /* algorithmic bytes of one pass: 2 n (key + value size) */
} bcf_plan;

/* Fill *plan for sorting n keys of type kt (pairs if has_vals). */
bcf_status bcf_sort_plan(uint64_t n, bcf_dtype kt, int has_vals, bcf_plan* plan);

/*
 * Per-kernel timing of the library's own launches, for benchmarking.  When
 * enabled, the library brackets every kernel it launches with CUDA events on
 * the launch stream (events are created once, on first use).  Kinds:
 * 0 block sort, 1 merge-path partition, 2 merge pass, 3 segmented sort,
 * 4 colored prefix sums, 5 pivot-bucket distribution (sampling, splitters,
 * bucket counts, scatter).
 */
#define BCF_PROFILE_KINDS 6
typedef struct {
    uint32_t launches[BCF_PROFILE_KINDS];
    double total_ms[BCF_PROFILE_KINDS];
} bcf_profile;

bcf_status bcf_profile_enable(int on);
/* Synchronise the recorded events, accumulate their times into *out, clear. */
bcf_status bcf_profile_collect(bcf_profile* out);
/*
 * The same, and also each launch on its own, in launch order: kinds[i] and
 * ms[i] for the first min(count of launches, max) of them (host arrays of max
 * entries, owned by the caller; either may be NULL when max is 0).  *count
 * gets the number of launches recorded.  BCF_EINVAL for a NULL out or count.
 */
bcf_status bcf_profile_collect_launches(bcf_profile* out, int* kinds, float* ms, uint32_t max,
                                        uint32_t* count);

/*
 * Profiling control: launch the block sort and the merge pass with at least
 * `bytes` of dynamic shared memory (0, the default, launches them as built).
 * A floor above half an SM's shared memory leaves one CTA per SM, which
 * isolates each CTA's own shared-memory traffic from its neighbours' in
 * hardware counters.  Results never change; only speed does.  BCF_EINVAL
 * above 232,448 bytes (227 KB, the per-CTA maximum).  Process-wide.
 */
bcf_status bcf_profile_set_smem_floor(uint32_t bytes);

/* Version string of the library. */
const char* bcf_version(void);

/* ---- payloads wider than 32 bits ------------------------------------------ */

/*
 * Stable sort by key with a payload row of `val_bytes` bytes per key (a
 * multiple of 4, up to 4096: u64 row ids, pointers, small structs).  The keys
 * are sorted with 32-bit row indices as payload (bcf_sort_pairs, either
 * algorithm), then the rows are gathered in the sorted order; the result is
 * the stable order, ties in input order.
 *   keys_out  device, n keys (may equal keys_in); 16-byte aligned
 *   vals_out  device, n rows; must not overlap vals_in (the gather reads the
 *             rows in any order); 4-byte aligned (16 for the fastest copies)
 *   ws        bcf_workspace_bytes(BCF_OP_SORT_WIDE, n, 0, kt, 1) bytes
 * n must be below 2^32 (BCF_EUNSUPPORTED otherwise).
 */
bcf_status bcf_sort_pairs_wide(void* keys_out, void* vals_out, const void* keys_in,
                               const void* vals_in, uint64_t n, uint32_t val_bytes, bcf_dtype kt,
                               const bcf_opts* opts, void* ws, size_t ws_bytes,
                               cudaStream_t stream);

/* ---- sorting host buffers --------------------------------------------------- */

/*
 * Sort n keys (pairs: key-value pairs) that live in HOST memory: copy in, sort,
 * copy out, all enqueued asynchronously on `stream`.  The host buffers must
 * stay valid, and the input unchanged, until the stream has passed the call.
 * Page-locked (pinned) host buffers give full copy bandwidth and let the copies
 * of calls on different streams overlap each other and other calls' sorting.
 * With BCF_ALGO_MERGE the input is copied in eight pieces on a library-owned
 * copy stream, and the block sort of each piece starts as soon as it has
 * landed.  The result is the one bcf_sort_keys / bcf_sort_pairs give.
 *   keys_out_host, vals_out_host   host, n keys / values, written (may equal the inputs)
 *   keys_in_host, vals_in_host     host, n keys / values
 *   ws        device workspace of bcf_workspace_bytes(BCF_OP_SORT_HOST, n, 0, kt,
 *             has_vals) bytes (BCF_OP_SORT_HOST_PB with BCF_ALGO_PIVOT_BUCKETS):
 *             device copies of the input and output plus the sort's workspace
 * Errors: as bcf_sort_keys; a null host pointer with n > 0 is BCF_EINVAL.
 */
bcf_status bcf_sort_keys_host(void* keys_out_host, const void* keys_in_host, uint64_t n,
                              bcf_dtype kt, const bcf_opts* opts, void* ws, size_t ws_bytes,
                              cudaStream_t stream);
bcf_status bcf_sort_pairs_host(void* keys_out_host, uint32_t* vals_out_host,
                               const void* keys_in_host, const uint32_t* vals_in_host, uint64_t n,
                               bcf_dtype kt, const bcf_opts* opts, void* ws, size_t ws_bytes,
                               cudaStream_t stream);

/* ---- colored prefix sums ------------------------------------------------ */

/*
 * Colored prefix sums: the paper's demonstration that bank conflicts decide
 * the runtime (Sec. 2.2, Fig. 2; algorithm in Appendix A).  Element i has a
 * value values[i] and a color colors[i] in [0, d); out[i] is the sum, modulo
 * 2^32, of values[j] over the j <= i (exclusive: j < i) with colors[j] ==
 * colors[i] -- d independent prefix sums in one pass over the data.
 *   out       device, n uint32_t; may equal `values` exactly (in place)
 *   values    device, n uint32_t
 *   colors    device, n uint8_t, each < d
 *   d         number of colors, 1..64 (the paper stops at 16 for lack of
 *             shared memory; one CTA holds d x 256 counters)
 *   exclusive 0: inclusive sums; 1: exclusive
 *   layout    BCF_CPS_BANKED: every thread keeps its per-color counters in
 *             its own shared-memory bank (the paper's conflict-free layout);
 *             BCF_CPS_ROWS: a thread's d counters are contiguous, so lanes
 *             collide on banks as d grows (the paper's conflicting baseline,
 *             kept for that comparison).  Results are identical.
 *   ws        workspace of bcf_workspace_bytes(BCF_OP_CPS, n, d, BCF_U32, 0)
 *             bytes (per-tile, per-color look-back words); cleared by the call
 * Pointers must be 16-byte aligned.  A color >= d is a precondition
 * violation: that element adds nothing, its output is 0, and
 * bcf_last_device_error() then returns BCF_EINVAL.
 */
enum { BCF_CPS_BANKED = 0, BCF_CPS_ROWS = 1 };
bcf_status bcf_colored_prefix_sums(uint32_t* out, const uint32_t* values, const uint8_t* colors,
                                   uint64_t n, uint32_t d, int exclusive, int layout, void* ws,
                                   size_t ws_bytes, cudaStream_t stream);

/* ---- tuning --------------------------------------------------------------- */

/*
 * Elements per thread (E) and threads per CTA (NT) of the block sort, the merge
 * pass and the segmented sort are chosen per operation, key width, payload flag
 * and size band from a table.  The paper fixes them by hand (Sec. 4: p = 128,
 * M = w^2 = 1024); here the project's autotuner measures every compiled
 * configuration on the GPU and writes the table.  Without a call to
 * bcf_tuning_set the library reads tuning/gb300.tsv of its package (rows "op
 * key_bytes has_vals n_min n_max block_cfg merge_cfg seg_cfg"); configurations
 * are indices into the lists that bcf_tuning_config enumerates.  In a
 * BCF_OP_SEGMENTED row, block_cfg is unused and merge_cfg says who runs the
 * merge passes: -1 the persistent worker, else launches of that merge
 * configuration, whose tile must not exceed the seg_cfg tile (BCF_EINVAL
 * otherwise).  Results never depend on the tuning.
 */
typedef struct {
    int op;              /* BCF_OP_SORT, BCF_OP_MERGE or BCF_OP_SEGMENTED */
    int key_bytes;       /* 4 (u32 / f32) or 8 (u64) */
    int has_vals;
    uint64_t n_min, n_max; /* the row applies to n_min <= n < n_max */
    int block_cfg, merge_cfg, seg_cfg;
} bcf_tuning_entry;

/* Replace the table (count 0: built-in defaults; count -1: the package's table
 * file again).  BCF_EINVAL if a row names an unsupported configuration; the
 * table is then left unchanged. */
bcf_status bcf_tuning_set(const bcf_tuning_entry* entries, int count);
/* Configuration `index` of kind 0 (block sort), 1 (merge) or 2 (segmented):
 * returns 1 and its E and NT, or 0 past the end of the list. */
int bcf_tuning_config(int kind, int index, int* elems_per_thread, int* threads);
/* 1 if configuration `index` of `kind` is built for that key width / payload. */
int bcf_tuning_supported(int kind, int index, int key_bytes, int has_vals);

/* ---- continuous-batching request server ---------------------------------- */

/*
 * A request server for sort and merge requests (the paper measures one sort at
 * a time, Sec. 4; serving many requests is this library's extension).  The
 * caller provides a device arena and drives the server from ONE host thread:
 * bcf_server_submit() queues requests, bcf_server_step() reaps finished work
 * (event polling, no blocking), frees its arena space and admits queued
 * requests by memory, bcf_server_poll() returns completion records.
 *
 * BCF_SERVE_BATCHED (continuous batching): requests of at most small_max keys
 * are coalesced -- per key type, order and payload flag -- into one segmented
 * sort over a packed batch in the arena (a merge of sorted runs equals the
 * stable sort of their concatenation, so small merges batch too); larger
 * requests run as their own sort / merge with the workspace in the arena,
 * round-robin over `streams` streams.  Requests that arrive while others are
 * on the GPU are admitted on the next step as memory frees up; small requests
 * may overtake a large one that does not fit yet.
 * BCF_SERVE_PLAIN (baseline): each request is its own launch chain, in arrival
 * order, on one stream.
 * Results are the same in both modes and the same as a call on its own.
 */
typedef struct bcf_server bcf_server;
enum { BCF_SERVE_BATCHED = 0, BCF_SERVE_PLAIN = 1 };

typedef struct {
    void* arena;             /* device memory owned by the caller, 256-byte aligned */
    uint64_t arena_bytes;
    int streams;             /* parallel streams in batched mode (1..64) */
    int mode;                /* BCF_SERVE_BATCHED or BCF_SERVE_PLAIN */
    uint64_t small_max;      /* requests up to this many keys are coalesced */
    uint64_t batch_max_keys; /* keys per coalesced launch (0: 2^22) */
} bcf_server_config;

typedef struct {
    int op;                  /* BCF_OP_SORT or BCF_OP_MERGE */
    bcf_dtype kt;
    int descending;
    uint64_t n;
    const void* keys_in;     /* device, caller-owned; must stay valid until completion */
    const uint32_t* vals_in; /* NULL for keys only (then vals_out NULL too) */
    void* keys_out;          /* device, caller-owned, n keys */
    uint32_t* vals_out;
    const uint64_t* run_offsets; /* merge: host, k+1 offsets from 0 to n (copied on submit) */
    uint32_t k;
    uint64_t tag;            /* returned in the completion record */
} bcf_request;

typedef struct {
    uint64_t tag;
    bcf_status status;
    double submit_s, admit_s, done_s; /* server clock (bcf_server_now) */
} bcf_completion;

typedef struct {
    uint64_t pending, inflight, arena_used, arena_peak, launched_units, launched_batches;
} bcf_server_stats_t;

/* Create: streams and a pinned staging ring are created here (set-up, not the
 * request path).  BCF_EINVAL for a bad config. */
bcf_status bcf_server_create(const bcf_server_config* cfg, bcf_server** out);
/* Seconds since the server was created (steady clock). */
double bcf_server_now(const bcf_server* s);
/* Queue a request (host bookkeeping only).  BCF_EINVAL for a malformed request,
 * BCF_ENOMEM if it can never fit in the arena. */
bcf_status bcf_server_submit(bcf_server* s, const bcf_request* r);
/* Reap finished work, admit and launch queued requests; *inflight (may be
 * NULL) gets the number of launch units still on the GPU.  Never blocks. */
bcf_status bcf_server_step(bcf_server* s, int* inflight);
/* Move up to max completion records into out; returns how many. */
int bcf_server_poll(bcf_server* s, bcf_completion* out, int max);
bcf_status bcf_server_stats(const bcf_server* s, bcf_server_stats_t* out);
/* Block until every submitted request completed. */
bcf_status bcf_server_drain(bcf_server* s);
bcf_status bcf_server_destroy(bcf_server* s);

/* The server's arena allocator on its own: first fit over [0, bytes) with a
 * coalescing free list, 256-byte granules.  Host bookkeeping only (no device
 * memory), exported for testing.  bcf_arena_free takes back exactly a live
 * range that bcf_arena_alloc returned (offset and the requested size); any
 * other range -- a double free, a wrong offset or size -- is BCF_EINVAL and
 * changes nothing. */
typedef struct bcf_arena bcf_arena;
bcf_status bcf_arena_create(uint64_t bytes, bcf_arena** out);
bcf_status bcf_arena_alloc(bcf_arena* a, uint64_t bytes, uint64_t* offset);
bcf_status bcf_arena_free(bcf_arena* a, uint64_t offset, uint64_t bytes);
bcf_status bcf_arena_usage(const bcf_arena* a, uint64_t* used, uint64_t* largest_free);
bcf_status bcf_arena_destroy(bcf_arena* a);

/* ---- sort without a caller workspace ------------------------------------ */

/*
 * bcf_sort_keys_static: bcf_sort_keys for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is a deployment convenience.
 *
 * Some callers cannot call cudaMalloc: a framework or plugin host that owns
 * every device allocation and hands a plugin only its input and output
 * buffers, a process whose device memory is carved up by an external pool it
 * must not go around, or a latency-critical loop that must not take
 * cudaMalloc's implicit device synchronisation.  They pass only keys_in /
 * keys_out; the merge passes' scratch (ping-pong copy and split array) lives
 * in a device array inside the library.
 *
 *   - n <= BCF_STATIC_MAX_KEYS, else BCF_EUNSUPPORTED before any launch; keys
 *     only; 16-bit keys are not available here (BCF_EUNSUPPORTED);
 *     BCF_ALGO_PIVOT_BUCKETS and BCF_ALGO_AUTO take the merge path (same
 *     result); otherwise
 *     the arguments, results and errors of bcf_sort_keys (an unknown
 *     opts->algorithm is BCF_EINVAL).
 *   - The array (about 8 MiB) is held by every GPU that loads the library until
 *     the process exits.  The call allocates nothing.
 *   - All calls share the array: calls whose GPU work overlaps in time (other
 *     streams, other host threads) race and give wrong results.  Serialise them.
 *     Nothing in it needs to start at zero; it keeps the last call's contents.
 *   - The first call on a device looks up the array's device address with that
 *     device current.
 */
#define BCF_STATIC_MAX_KEYS (1u << 20)
bcf_status bcf_sort_keys_static(void* keys_out, const void* keys_in, uint64_t n, bcf_dtype kt,
                                const bcf_opts* opts, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BCFSORT_H */
