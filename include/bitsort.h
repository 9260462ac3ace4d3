/*
 * bitsort.h -- C ABI of the GB300 (sm_103a) bitmap sort.
 *
 * The operation is the paper's bitwise sort of an integer array (K. Yordzhev,
 * "The bitwise operations related to a fast sorting algorithm", Section V,
 * Algorithm 1; Theorem 1: the result is the array in ascending order;
 * Theorem 2: linear time).  It is computed here in its bit-set form: key x
 * sets bit (x mod 32) of word floor(x / 32) of a bitmap with OR and a shifted
 * one (Table I; Example 2); the words are then read in index order and the
 * positions of the set bits, bit 0 first inside a word (bit numbering of
 * Section II), are written out.  That form needs two things the paper's own
 * listing does not: the keys must be DISTINCT (one bit cannot count
 * repetitions) and BOUNDED by `max_value` (the bitmap has max_value + 1
 * bits).  Under those two conditions the output equals the paper's result.
 *
 * Conventions for every call below:
 *   - keys/out are DEVICE pointers to uint32_t arrays of n elements unless a
 *     call says otherwise.  out == keys (sorting in place, as the paper's
 *     function does) is allowed; any other overlap of the two ranges is
 *     BITSORT_ERR_INVALID.
 *   - M = max_value + 1 is computed in 64 bits (max_value may be 2^32 - 1).
 *   - Calls are asynchronous with respect to the host: they enqueue work on
 *     `stream` and return.  Host-checkable errors (null pointer with n > 0,
 *     n > M, partial overlap, allocation failure) are returned at once and
 *     nothing is enqueued.  Data-dependent outcomes are written on the device
 *     into a bitsort_result_t and are read after the stream completes.
 *   - Data-dependent outcomes:
 *       BITSORT_OK            out[0..n) = keys in ascending order.
 *       BITSORT_ERR_KEY_RANGE some key > max_value: such keys are skipped;
 *                             out[0..count) = the distinct in-range keys in
 *                             ascending order, out[count..n) unspecified.
 *       BITSORT_ERR_DUPLICATE a key occurs more than once: out[0..count) =
 *                             the distinct keys ascending (count < n),
 *                             out[count..n) unspecified.  KEY_RANGE takes
 *                             precedence when both hold.
 *       BITSORT_ERR_TIMEOUT   a bounded device-side wait ran out (a stalled
 *                             predecessor); out is unspecified.  The context
 *                             resets its scratch when it reports this.
 *   - A context (bitsort_ctx_t) owns the device scratch of the calls made
 *     with it.  Calls that share a context must be ordered on the device
 *     (same stream, or ordered by events); concurrent calls on different
 *     streams need different contexts.
 */
#ifndef BITSORT_H_
#define BITSORT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA headers (same underlying type). */
typedef struct CUstream_st *bitsort_stream_t;

typedef enum {
    BITSORT_OK = 0,
    BITSORT_ERR_INVALID = 1,   /* bad argument (host check) */
    BITSORT_ERR_KEY_RANGE = 2, /* a key above max_value (device) */
    BITSORT_ERR_DUPLICATE = 3, /* repeated keys (device) */
    BITSORT_ERR_NOMEM = 4,     /* device or host allocation failed */
    BITSORT_ERR_TIMEOUT = 5,   /* a bounded device wait expired */
    BITSORT_ERR_CUDA = 6,      /* a CUDA runtime call failed */
    BITSORT_ERR_BUDGET = 7     /* a served request can never fit the budget */
} bitsort_status_t;

/* Device-written outcome of one sort: status is a bitsort_status_t value,
 * count the number of values written to out. 16 bytes, 8-byte aligned. */
typedef struct {
    uint32_t status;
    uint32_t reserved;
    uint64_t count;
} bitsort_result_t;

typedef struct bitsort_ctx bitsort_ctx_t;

/* ----------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (made current by the call).
 * Returns BITSORT_ERR_INVALID for a bad device, BITSORT_ERR_NOMEM on failure
 * to allocate its fixed scratch. *ctx receives the handle.
 * Environment read here:
 *   BITSORT_TUNE_CACHE=path  load the tuned table written by
 *                            bitsort_tune_save (a missing or unreadable file
 *                            is noted in bitsort_last_error and ignored);
 *   BITSORT_FORCE_PATH=fused|partition|global  take that path for every
 *                            single sort of the context, tuned or not (the
 *                            size rules still apply: no fused slice beyond
 *                            2^20 values); other values are ignored.
 * Every sorting call opens an NVTX range named after itself (host side, the
 * call's enqueue; no cost unless a profiler is attached). */
bitsort_status_t bitsort_ctx_create(int device, bitsort_ctx_t **ctx);

/* Synchronise the device and free everything the context owns. */
bitsort_status_t bitsort_ctx_destroy(bitsort_ctx_t *ctx);

/* Text for a status code (static storage). */
const char *bitsort_status_string(bitsort_status_t status);

/* Description of the last CUDA error this thread's calls ran into ("" if
 * none), for reports next to BITSORT_ERR_CUDA / BITSORT_ERR_NOMEM.  Thread-
 * local storage, valid until the thread's next library call.  Setting the
 * environment variable BITSORT_VERBOSE also prints each one to stderr. */
const char *bitsort_last_error(void);

/* ------------------------------------------------------------- single sort */

/* Sort n distinct uint32 keys bounded by max_value (Algorithm 1's problem,
 * bitmap form).  Uses a per-device default context created on first use.
 * The data-dependent result is kept in that context; read it with
 * bitsort_sync_status(NULL, stream, &count). */
bitsort_status_t bitsort(const uint32_t *keys, size_t n, uint32_t max_value, uint32_t *out,
                         bitsort_stream_t stream);

/* As bitsort(), with an explicit context (NULL = the current device's default
 * context) and an optional DEVICE pointer `d_result` that receives the
 * outcome (NULL = keep it in the context). */
bitsort_status_t bitsort_ex(bitsort_ctx_t *ctx, const uint32_t *keys, uint64_t n, uint32_t max_value,
                            uint32_t *out, bitsort_result_t *d_result, bitsort_stream_t stream);

/* Sort n distinct SIGNED int32 keys in [min_value, max_value] into ascending
 * signed order (Section III, Algorithm 1's second function: the paper sorts
 * negative and nonnegative keys apart and joins them; here every key is
 * shifted by -min_value modulo 2^32, which maps the range onto
 * 0 .. max_value - min_value in the same order, and sorted as unsigned keys
 * with the shift undone on output).
 *   - keys, out: DEVICE pointers to n int32 values; keys == out sorts in
 *     place; other overlaps -> BITSORT_ERR_INVALID.
 *   - min_value > max_value, n > max_value - min_value + 1 (the keys cannot
 *     be distinct), or misaligned pointers -> BITSORT_ERR_INVALID.
 *   - A key outside [min_value, max_value] -> BITSORT_ERR_KEY_RANGE, repeated
 *     keys -> BITSORT_ERR_DUPLICATE, both reported through d_result (or the
 *     context) like bitsort_ex(); the whole int32 range (min INT32_MIN, max
 *     INT32_MAX) is allowed. */
bitsort_status_t bitsort_i32(bitsort_ctx_t *ctx, const int32_t *keys, uint64_t n, int32_t min_value,
                             int32_t max_value, int32_t *out, bitsort_result_t *d_result, bitsort_stream_t stream);

/* Sort unsigned keys bounded below and above: distinct uint32 keys in
 * [min_value, max_value] (the bitmap covers max_value - min_value + 1
 * values; the same shift as bitsort_i32, without the signed reading).  One
 * rank's share of a sort spread over GPUs by value range (see
 * bitsort_range_split) is such an array.  Same contract as bitsort_i32:
 * keys == out sorts in place; min_value > max_value, n above the span,
 * overlaps or misalignment -> BITSORT_ERR_INVALID; keys outside the range ->
 * BITSORT_ERR_KEY_RANGE, repeats -> BITSORT_ERR_DUPLICATE through d_result
 * (or the context). */
bitsort_status_t bitsort_span(bitsort_ctx_t *ctx, const uint32_t *keys, uint64_t n, uint32_t min_value,
                              uint32_t max_value, uint32_t *out, bitsort_result_t *d_result,
                              bitsort_stream_t stream);

/* The bitmap sort for keys stored in 16, 8 and 64 bits (Algorithm 1 is
 * written for any integer type T; Section V).  Same contract as bitsort_ex()
 * (distinct keys bounded by max_value, keys == out allowed, other overlaps,
 * null pointers, misalignment for the type or n > max_value + 1 ->
 * BITSORT_ERR_INVALID; KEY_RANGE / DUPLICATE through d_result or the
 * context, count = values written).
 *   - bitsort_u16 / bitsort_u8: the whole value range (at most 65,536 values)
 *     is one shared-memory bitmap: one kernel, one CTA.
 *   - bitsort_u64: max_value must be below 2^32 (else BITSORT_ERR_INVALID);
 *     keys are narrowed to 32 bits into a context-owned copy (n x 4 bytes,
 *     grown on demand), sorted by the 32-bit path and widened into out.  A
 *     key above max_value, also one differing only above bit 31, is skipped
 *     and reported as KEY_RANGE. */
bitsort_status_t bitsort_u16(bitsort_ctx_t *ctx, const uint16_t *keys, uint64_t n, uint16_t max_value,
                             uint16_t *out, bitsort_result_t *d_result, bitsort_stream_t stream);
bitsort_status_t bitsort_u8(bitsort_ctx_t *ctx, const uint8_t *keys, uint64_t n, uint8_t max_value, uint8_t *out,
                            bitsort_result_t *d_result, bitsort_stream_t stream);
bitsort_status_t bitsort_u64(bitsort_ctx_t *ctx, const uint64_t *keys, uint64_t n, uint64_t max_value,
                             uint64_t *out, bitsort_result_t *d_result, bitsort_stream_t stream);

/* Sort n uint32 keys that MAY REPEAT, bounded by max_value: the paper's
 * Algorithm 1 itself (Section V, first function): stable splits of the keys
 * by their bits, least significant first, split_bits bits per pass (1..8;
 * 1 = the paper's one bit per pass; 0 = the fewest passes of at most 8 bits
 * that cover the bits of max_value).  Every key is written once per pass;
 * the result is the ascending order of the multiset (Theorem 1).
 *   - keys, out: DEVICE pointers to n uint32; keys == out sorts in place
 *     (through the context's buffer); other overlaps -> BITSORT_ERR_INVALID.
 *   - n >= 2^32, split_bits > 8 or misaligned pointers -> BITSORT_ERR_INVALID,
 *     nothing enqueued.
 *   - A key above max_value -> BITSORT_ERR_KEY_RANGE (out then holds the keys
 *     ordered by the bits below the range's width only); count is always n.
 *     Reported through d_result (DEVICE, nullable = the context) like
 *     bitsort_ex().
 *   - Scratch (grown on demand, owned by the context): a buffer of n keys
 *     (shared with the bitmap path), ceil(n / 8192) x 2^split_bits look-back
 *     words and a 4.4 KB block.  Calls on one context are stream-ordered on
 *     the stream they are given: do not run two at once on one context. */
bitsort_status_t bitsort_multiset(bitsort_ctx_t *ctx, const uint32_t *keys, uint64_t n, uint32_t max_value,
                                  uint32_t split_bits, uint32_t *out, bitsort_result_t *d_result,
                                  bitsort_stream_t stream);

/* As bitsort_multiset() for SIGNED int32 keys in [min_value, max_value]
 * (Algorithm 1's second function sorts the negative and the nonnegative keys
 * apart and joins them; the same order comes from splitting the offsets
 * x - min_value modulo 2^32).  min_value > max_value -> BITSORT_ERR_INVALID;
 * a key outside the range -> BITSORT_ERR_KEY_RANGE. */
bitsort_status_t bitsort_multiset_i32(bitsort_ctx_t *ctx, const int32_t *keys, uint64_t n, int32_t min_value,
                                      int32_t max_value, uint32_t split_bits, int32_t *out,
                                      bitsort_result_t *d_result, bitsort_stream_t stream);

/* bitsort_ex() on keys held in HOST memory: the n keys are copied to device
 * buffers owned by the context (grown on demand), sorted, and the n output
 * slots and the outcome copied back, all enqueued on `stream`; the call
 * returns before they finish (wait on the stream).
 *   - h_keys, h_out: HOST pointers to n uint32 (page-locked memory lets the
 *     copies run asynchronously; pageable memory works, but then the copies
 *     synchronise with the host); h_keys == h_out is allowed.  On DUPLICATE
 *     or KEY_RANGE, h_out[count..n) is unspecified.
 *   - h_result: HOST pointer (nullable) that receives the outcome once the
 *     stream has passed this call.
 *   - The context's buffers serve every call on it: calls on one context are
 *     ordered by the stream they are given; to overlap calls (one's copies
 *     with another's sort), give each stream its own context.
 *   - Errors as bitsort_ex(); BITSORT_ERR_NOMEM if the device buffers cannot
 *     be grown. */
bitsort_status_t bitsort_host(bitsort_ctx_t *ctx, const uint32_t *h_keys, uint64_t n, uint32_t max_value,
                              uint32_t *h_out, bitsort_result_t *h_result, bitsort_stream_t stream);

/* Wait for `stream`, then return the status of the last sort that wrote its
 * outcome into the context (and its count through `count`, nullable). */
bitsort_status_t bitsort_sync_status(bitsort_ctx_t *ctx, bitsort_stream_t stream, uint64_t *count);

/* Sort without allocating any device memory (the paper has no counterpart:
 * this is a deployment variant of bitsort_ex's partition path).  For callers
 * that cannot call cudaMalloc: applications whose device memory is all owned
 * by another allocator (e.g. a framework's caching allocator that has
 * reserved the whole HBM, so a cudaMalloc would fail), and real-time or
 * certified code that forbids allocation after start-up (an allocation can
 * block for an unbounded time and may synchronise the device).
 *   - keys, out: DEVICE pointers to n uint32 keys / outputs, NOT overlapping
 *     (out also serves as the partition buffer; keys == out is rejected).
 *   - d_result: DEVICE pointer (required) that receives the outcome, with
 *     the same meaning as for bitsort_ex().
 *   - Limits: max_value < 2^31 (M <= 2^31 values: the fixed scratch holds
 *     2048 buckets of at most 2^20 values); larger, or keys == out, or a
 *     null d_result -> BITSORT_ERR_INVALID, nothing enqueued.
 *   - Scratch: one 49,408-byte __device__ array in the library, held by
 *     every GPU that loads it until the process exits.  It is shared by all
 *     calls and keeps the last call's contents; each call clears it first.
 *     Calls that overlap on the GPU (other streams, other threads) race:
 *     order them.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address (cudaGetSymbolAddress) and sets the kernels'
 *     shared-memory limit; make that first call before any stream capture.
 * Allocates nothing: no cudaMalloc/cudaFree, no library allocation. */
bitsort_status_t bitsort_noalloc(const uint32_t *keys, uint64_t n, uint32_t max_value, uint32_t *out,
                                 bitsort_result_t *d_result, bitsort_stream_t stream);

/* --------------------------------------------------------------- multi-GPU */

/* One sort of Section V's problem (one array, one ascending result) spread
 * over G GPUs by value range: rank g owns the values [g*W, (g+1)*W) with
 * W = bitsort_range_width(max_value, G).  Each rank groups its keys by owner
 * (bitsort_range_split), the ranks exchange the groups (an all-to-all of the
 * G counts, then of the keys; the host's collective library, not this
 * library, moves them), and each rank sorts what it received with
 * bitsort_span(ctx, keys, n, g*W, min((g+1)*W, M) - 1, ...).  Rank g's output
 * is then the g-th piece of the sorted array; its offset is the sum of the
 * counts of the ranks before it (an all-gather of G counts).  The exchange
 * and the offsets are host logic (paper_1312_0138_gb300/shard.py).
 *
 * bitsort_range_width: W for G = parts ranks: ceil((max_value + 1) / parts)
 * rounded up to a multiple of 128 (0 for parts == 0).
 *
 * bitsort_range_split: keys (DEVICE, n uint32) grouped by owner into out
 * (DEVICE, n entries, not overlapping keys): group g at [o_g, o_g + c_g),
 * the groups in rank order, the keys of a group in no particular order.
 *   - d_counts: DEVICE pointer to `parts` uint64 receiving c_0 .. c_{parts-1}.
 *   - parts in 1 .. 8192; keys == out, overlaps, misalignment, n >= 2^32 or
 *     a null d_counts -> BITSORT_ERR_INVALID.
 *   - Keys above max_value are left out of every group and reported as
 *     BITSORT_ERR_KEY_RANGE through d_result (or the context), whose count is
 *     the number of keys grouped.  Distinctness is not checked here (each
 *     rank's bitsort_span does that).
 *   - Uses the context's scratch and leaves it at zero; enqueued on `stream`. */
uint64_t bitsort_range_width(uint32_t max_value, uint32_t parts);
bitsort_status_t bitsort_range_split(bitsort_ctx_t *ctx, const uint32_t *keys, uint64_t n, uint32_t max_value,
                                     uint32_t parts, uint32_t *out, uint64_t *d_counts, bitsort_result_t *d_result,
                                     bitsort_stream_t stream);

/* ---------------------------------------------------------------- batching */

/* One array of a batch.  keys/out are device pointers; the same rules as
 * bitsort() apply to each array independently. */
typedef struct {
    const uint32_t *keys;
    uint32_t *out;
    uint64_t n;
    uint32_t max_value;
    uint32_t reserved;
} bitsort_desc_t;

typedef struct bitsort_batch_plan bitsort_batch_plan_t;

/* Sort `count` independent arrays in one persistent launch.  `descs` is a
 * HOST array; `d_results` a DEVICE array of `count` outcomes (nullable).
 * Builds a plan, launches it once and frees the plan (stream-ordered). */
bitsort_status_t bitsort_batched(bitsort_ctx_t *ctx, const bitsort_desc_t *descs, size_t count,
                                 bitsort_result_t *d_results, bitsort_stream_t stream);

/* Build a reusable plan for a batch: the per-array strategy (fused shared
 * memory slice, partition + shared-memory slices, or global L2 bitmap), the
 * work list, and the device scratch.  The plan owns its scratch and a device
 * array of `count` outcomes.  The pointers in descs are baked in. */
bitsort_status_t bitsort_batch_plan_create(bitsort_ctx_t *ctx, const bitsort_desc_t *descs, size_t count,
                                           bitsort_batch_plan_t **plan);

/* Enqueue the plan on `stream`.  The first launch on a stream captures the
 * launch sequence into a CUDA graph; later launches replay it.  Launches of
 * one plan must be ordered on the device. */
bitsort_status_t bitsort_batch_plan_launch(bitsort_batch_plan_t *plan, bitsort_stream_t stream);

/* Copy the plan's outcomes to HOST memory `results` (count entries) after
 * synchronising `stream`.  Returns the first non-OK status, or OK. */
bitsort_status_t bitsort_batch_plan_results(bitsort_batch_plan_t *plan, bitsort_stream_t stream,
                                            bitsort_result_t *results);

/* Device pointer to the plan's outcome array (count entries). */
const bitsort_result_t *bitsort_batch_plan_device_results(const bitsort_batch_plan_t *plan);

bitsort_status_t bitsort_batch_plan_destroy(bitsort_batch_plan_t *plan);


/* ----------------------------------------------------------------- serving */

typedef struct bitsort_server bitsort_server_t;

/* A continuous-batching sort server on `device`.  Requests are admitted in
 * arrival order while the bytes their bitmap and output need
 * (ceil(M/8) + 4n, M = max_value + 1), plus the device memory the server's
 * stream contexts keep (their partition buffers and global bitmaps, held at
 * their high-water sizes) and the growth of that memory a request's plain
 * sort asks for, fit in `budget_bytes`.  Admitted requests are launched at
 * once: a request of at least 2^20 keys alone as a plain sort, smaller ones
 * together as batches of up to 64 MiB of work (8n + M/4 bytes each).
 * `max_inflight` streams (1..64) take the batches: large requests stream 0,
 * one after another (concurrent large sorts were measured slower: each one's
 * partition output leaves L2 before its bucket phase reads it), batches of
 * small requests the others; each holds several queued behind one another,
 * so that the device never waits for the scheduler and work on different
 * streams overlaps. */
bitsort_status_t bitsort_server_create(int device, uint64_t budget_bytes, int max_inflight,
                                       bitsort_server_t **server);

/* Queue one request (device pointers, caller-owned until it completes).
 * Returns BITSORT_ERR_BUDGET if the request alone (with the scratch of its
 * plain sort) exceeds the budget,
 * BITSORT_ERR_INVALID for bad arguments.  *ticket identifies it. */
bitsort_status_t bitsort_server_submit(bitsort_server_t *server, const uint32_t *keys, uint64_t n,
                                       uint32_t max_value, uint32_t *out, uint64_t *ticket);

/* Block until request `ticket` has completed; its outcome, count and latency
 * (completion minus submission, seconds) are returned (pointers nullable). */
bitsort_status_t bitsort_server_wait(bitsort_server_t *server, uint64_t ticket, bitsort_status_t *status,
                                     uint64_t *count, double *latency_s);

/* Counters since creation: completed requests, keys sorted, launched batches,
 * and the largest number of batches seen in flight at once (nullable). */
bitsort_status_t bitsort_server_stats(bitsort_server_t *server, uint64_t *completed, uint64_t *keys,
                                      uint64_t *batches, uint64_t *max_concurrent);

/* Drain outstanding requests, stop the scheduler and free the server. */
bitsort_status_t bitsort_server_destroy(bitsort_server_t *server);

/* -------------------------------------------------------------- autotuning */

/* Strategies a plan may use for one array. */
typedef enum {
    BITSORT_PATH_AUTO = 0,
    BITSORT_PATH_FUSED = 1,     /* one CTA, bitmap in shared memory (M <= 2^20) */
    BITSORT_PATH_PARTITION = 2, /* high-bit partition, one shared-memory slice per bucket */
    BITSORT_PATH_GLOBAL = 3     /* atomicOr into a global (L2-resident) bitmap, then scan */
} bitsort_path_t;

/* One configuration of the sort of one array.
 *   path            see bitsort_path_t.
 *   slice_values    values per shared-memory bitmap slice (bucket or scan
 *                   tile), a multiple of 128, at most 2^20.
 *   block_threads   256 or 512.
 *   words_per_lane  bitmap words each lane takes per scan step: 1, 2 or 4.
 *   stage           1: set-bit positions are staged per warp in shared
 *                   memory and leave in coalesced stores (words_per_lane 1).
 *   layout          PARTITION path: 0 = exact bucket ranges from a histogram
 *                   pass (n-entry buffer, the output buffer when it does not
 *                   alias the keys); 1 = fixed capacity min(slice, n) per
 *                   bucket in a context buffer, no histogram pass.
 *   persistent      1: all phases in one persistent launch; 0: one kernel
 *                   per phase.
 *   emit            0 = the lanes walk the set bits of their bitmap words;
 *                   1 = rank: the per-word popcount prefix is kept next to
 *                   the bitmap and every key writes itself at its index among
 *                   the set bits (prefix of its word + popcount of the lower
 *                   bits), through a shared-memory copy of the slice's output
 *                   (for sparse bitmaps; falls back to 0 for a slice with
 *                   more outputs than expected).
 *   part_stream     1: the partition phase streams its tiles into shared
 *                   memory with bulk copies (double-buffered) when the keys
 *                   are 16-byte aligned; 0: the threads load them.
 *   summary         1: a slice with at most one key per four bitmap words
 *                   also sets a summary bitmap (one bit per non-empty word)
 *                   and counts and emits only the non-empty words, clearing
 *                   them behind; 0: every slice walks all its words.
 *   part_threads    block size of the histogram and partition phases of a
 *                   one-kernel-per-phase plan (256, 512 or 1024); 0 = the
 *                   built-in rule (512 threads, 1024 from 1024 buckets).
 *   part_tile_keys  keys per partition tile when that phase runs at 512 or
 *                   1024 threads and its tiles are not streamed: 16 keys a
 *                   thread (8192 / 16384), or 32 (16384 / 32768: wide tiles,
 *                   a counting sort per tile, with the next tile copied in
 *                   while the current one is written out); 0 = the built-in
 *                   rule (wide when the shared memory holds such a tile and
 *                   there are at least three tiles per SM at 1024 threads,
 *                   four at 512).  A value that matches neither size of the
 *                   phase's block size counts as 0.
 *   ms              measured time when tuned (output only). */
typedef struct {
    int32_t path;
    uint32_t slice_values;
    uint32_t block_threads;
    uint32_t words_per_lane;
    uint32_t stage;
    uint32_t layout;
    uint32_t persistent;
    uint32_t emit;
    uint32_t part_stream;
    uint32_t summary;
    uint32_t part_threads;
    uint32_t part_tile_keys;
    double ms;
} bitsort_config_t;

/* Time the candidate configurations on representative DEVICE data: n
 * distinct keys bounded by max_value in `keys` (left unchanged) and a
 * separate DEVICE buffer `out` of n elements (keys and out must not
 * overlap).  Each candidate runs once to warm up, then five times with L2
 * flushed in between; the one with the smallest median time goes into the
 * context's table for the size class (ceil(log2 n), ceil(log2 M)) and is
 * reported in *best (nullable).  Synchronises the device. */
bitsort_status_t bitsort_autotune(bitsort_ctx_t *ctx, const uint32_t *keys, uint32_t *out, uint64_t n,
                                  uint32_t max_value, bitsort_config_t *best);

/* Force a configuration for the size class of (n, max_value).  slice_values,
 * block_threads and words_per_lane left 0 take the default; stage, layout
 * and persistent are taken as given; path BITSORT_PATH_AUTO removes the
 * entry (back to the built-in rule).  The
 * configuration is adjusted to what the size allows (e.g. no fused path
 * beyond 2^20 values, at most 8192 slices). */
bitsort_status_t bitsort_set_config(bitsort_ctx_t *ctx, uint64_t n, uint32_t max_value,
                                    const bitsort_config_t *config);

/* The configuration the context would use for (n, max_value). */
bitsort_status_t bitsort_get_config(bitsort_ctx_t *ctx, uint64_t n, uint32_t max_value, bitsort_config_t *config);

/* Shape of a plan (bitsort_plan_rule). */
typedef struct {
    uint32_t slices;          /* bitmap slices (buckets, or scan slices of the global bitmap; 1 when fused) */
    uint32_t tile_keys;       /* keys per partition / scatter tile */
    uint32_t part_threads;    /* block size of the histogram and partition phases */
    uint32_t bucket_threads;  /* block size of the bucket phase */
    uint32_t smem_bytes;      /* largest dynamic shared memory a launch of the plan asks for, per block */
    uint32_t reserved;
    uint64_t scratch_bytes;   /* partition buffer of the capacity layout (0 for the other layouts) */
} bitsort_plan_shape_t;

/* The built-in plan rule for an array of n distinct keys bounded by
 * max_value, out of place, keys 16-byte aligned, on a device with `sms`
 * streaming multiprocessors and `smem_per_block` bytes of opt-in shared
 * memory per block: the plan a context uses when its table holds no tuned
 * entry for the size class.  Host logic only: needs no GPU and no context,
 * launches nothing.  *shape is nullable.  INVALID: sms < 1,
 * smem_per_block == 0, config NULL, or n > max_value + 1. */
bitsort_status_t bitsort_plan_rule(int sms, uint32_t smem_per_block, uint64_t n, uint32_t max_value,
                                   bitsort_config_t *config, bitsort_plan_shape_t *shape);

/* Batch policy of a context (used by plans created afterwards).  Arrays whose
 * values fit one slice (max_value + 1 <= slice_values) are each sorted by one
 * fused shared-memory slice; the others take `path` (BITSORT_PATH_PARTITION:
 * high-bit partition + shared-memory slices; BITSORT_PATH_GLOBAL: global
 * bitmap in L2) with slices of slice_values values.  Also used:
 * block_threads (256/512), words_per_lane, stage; other fields ignored. */
bitsort_status_t bitsort_set_batch_config(bitsort_ctx_t *ctx, const bitsort_config_t *config);
bitsort_status_t bitsort_get_batch_config(bitsort_ctx_t *ctx, bitsort_config_t *config);

/* Time candidate batch policies (path x slice size x block size x words per
 * lane) on the given batch (device data; the outputs are overwritten) and
 * keep the fastest as the context's batch policy, reported in *best
 * (nullable).  Synchronises. */
bitsort_status_t bitsort_batch_autotune(bitsort_ctx_t *ctx, const bitsort_desc_t *descs, size_t count,
                                        bitsort_config_t *best);

/* Save / load the tuned table as JSON text at `path`. */
bitsort_status_t bitsort_tune_save(bitsort_ctx_t *ctx, const char *path);
bitsort_status_t bitsort_tune_load(bitsort_ctx_t *ctx, const char *path);

/* ------------------------------------------------------------- diagnostics */

/* Upper bound of every bounded device-side wait, in milliseconds (default
 * 4000).  A wait that runs out reports BITSORT_ERR_TIMEOUT instead of
 * hanging the GPU. */
bitsort_status_t bitsort_set_wait_limit_ms(bitsort_ctx_t *ctx, uint32_t ms);

/* Launch a partition-path sort of keys/n/max_value whose bucket stage waits
 * for one partition tile that is never scheduled: every bounded wait must
 * run out and the outcome must be BITSORT_ERR_TIMEOUT.  For testing the
 * failure path; the context stays usable afterwards. */
bitsort_status_t bitsort_debug_stalled_launch(bitsort_ctx_t *ctx, const uint32_t *keys, uint64_t n,
                                              uint32_t max_value, uint32_t *out, bitsort_stream_t stream);

/* Per-phase timing of single sorts on this context (off by default).  When
 * on, every bitsort_ex() call records a CUDA event on its stream before its
 * first kernel and after each kernel (this can cost the overlap between
 * consecutive kernels).  bitsort_phase_times() waits for the last recorded
 * event and writes the last call's kernel durations in milliseconds to
 * ms[0..*count) in launch order, with each kernel's item type in kinds[]
 * (0 histogram, 1 partition, 2 bucket slices, 3 global scatter, 4 global
 * scan, 5 partition streamed through bulk copies, 6 partition in wide
 * tiles, 16 multiset histogram, 17 multiset split, -1 persistent); both
 * arrays need room for 8 entries. */
bitsort_status_t bitsort_set_phase_timing(bitsort_ctx_t *ctx, int enable);
bitsort_status_t bitsort_phase_times(bitsort_ctx_t *ctx, float *ms, int *kinds, int *count);

/* Number of kernels the library enqueued since the context was created. */
uint64_t bitsort_kernel_launches(const bitsort_ctx_t *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BITSORT_H_ */
