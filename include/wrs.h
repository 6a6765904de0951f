/*
 * wrs.h -- C ABI of libwrs: Walker alias tables built on a GB300 GPU with the
 * parallel split construction, and bulk weighted sampling with replacement.
 *
 * The operations follow L. Huebschle-Schneider and P. Sanders, "Parallel
 * Weighted Random Sampling":
 *   - problem WRS-1 / WRS-R (Sec. 1): draw items X with P[X = i] = w_i / W,
 *     k times independently;
 *   - the alias table (Sec. 2.2): n buckets of capacity W/n, bucket i holds
 *     part w'_i of item i and at most one other item, its alias a_i;
 *   - its construction (Alg. 2, Sec. 4.1; Alg. 3 "PSA", Sec. 4.2) and its
 *     query: a uniform bucket r and a biased coin, heads -> r, tails -> a_r
 *     (Sec. 2.2; k queries: Sec. 5, Cor. "kWR").
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are CUDA device pointers, h_* are host pointers.
 *     No torch or CUDA types appear here: a stream is a cudaStream_t passed
 *     as void* (NULL = the legacy default stream).
 *   - Work is enqueued on the given stream and the call returns without
 *     waiting, unless its comment says it synchronises.
 *   - Argument errors are returned at once and enqueue nothing.  Errors the
 *     GPU detects (invalid weights, exact range exceeded, a bounded wait that
 *     ran out, a broken invariant) are stored in the table's device status
 *     word; wrs_table_status() reads it.  A sample call on a table whose
 *     build failed writes nothing.
 *   - Determinism: the table is a pure function of the weights, and sample s
 *     of a call is a pure function of (table, seed, stream_id, s); neither
 *     depends on the launch configuration.
 */
#ifndef WRS_H
#define WRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WRS_OK = 0,
    WRS_EINVAL = 1,     /* bad argument or invalid weights (NaN, Inf, sign bit set, all zero) */
    WRS_ENOMEM = 2,     /* a device or pinned-host allocation failed */
    WRS_EOVERFLOW = 3,  /* the weights' exact sum needs more than 95 bits */
    WRS_ETIMEOUT = 4,   /* a bounded wait between thread blocks gave up */
    WRS_EDEVICE = 5,    /* a CUDA runtime call failed */
    WRS_EINTERNAL = 6   /* an invariant of exact arithmetic failed (never expected) */
} wrs_status;

typedef enum {
    WRS_U32 = 0,        /* uint32 weights: item i has exact weight q_i = w_i */
    WRS_F32 = 1         /* IEEE binary32 weights >= +0, finite; exact, see below */
} wrs_dtype;

/*
 * One bucket of the table, 16 bytes, array of structures (Sec. 10 "Sequential
 * Performance": one cache access per query).  With Q the exact weight total
 * in integer units (below), shift = max(0, bitlen(Q) - 64) and qp = Q >> shift,
 * the coin of bucket r comes up heads for a 64-bit uniform v iff
 * floor(v * qp / 2^64) < thr.  thr = bw >> shift, where bw in [0, Q] is the
 * part of item r that the bucket holds, in units where every bucket holds Q
 * and item i weighs n * q_i.  A full bucket points to itself.
 */
typedef struct {
    uint64_t thr;
    uint32_t alias;
    uint32_t reserved; /* zero */
} wrs_bucket;

/*
 * Exact integer units: u32 weights are used as they are (q_i = w_i, beta = 0).
 * For binary32 weights, beta is the smallest exponent of a set bit over all
 * nonzero weights and q_i = w_i * 2^-beta, an exact integer.  Q = sum q_i
 * must stay below 2^95, else the build fails with WRS_EOVERFLOW.
 */
typedef struct {
    uint64_t n;          /* number of items / buckets */
    uint64_t q_lo, q_hi; /* Q, the exact weight total in integer units */
    int32_t beta;        /* exponent of the integer unit (binary32 weights) */
    uint32_t shift;      /* thr = bw >> shift */
    uint64_t qp;         /* Q >> shift, the coin denominator */
    uint64_t n_light;    /* items with n * q_i <= Q (Sec. 2.2: light) */
    uint32_t light_max;  /* an item is light iff its raw 32-bit word <= light_max */
    int32_t status;      /* wrs_status of the last build */
} wrs_table_info;

typedef struct wrs_table wrs_table; /* opaque; device memory owned by the library */

/* Allocate a table (buckets and workspace) for up to capacity_n weights.
 * capacity_n in [1, 2^32 - 1].  Synchronous (stream-ordered allocation on a
 * stream of the table's own, waited for before returning); the table can be
 * rebuilt any number of times.  Every later call on a table records CUDA
 * events on the streams it is given, so that the host-side calls below wait
 * for this table's work only.  Device memory: 16 B per bucket plus about
 * 0.09 B per weight of workspace.  Errors: WRS_EINVAL, WRS_ENOMEM. */
wrs_status wrs_table_create(uint64_t capacity_n, wrs_table **out);

/* Build the alias table of n weights (Alg. 3 "PSA", Sec. 4.2, with the exact
 * split of Alg. 2's state; identical bucket for bucket to Alg. 2).  d_weights:
 * n words of dtype, device memory, 4-byte aligned, read only; the caller may
 * free or overwrite it once the build has completed on `stream`.  n in [1,
 * capacity].  Allocates nothing; asynchronous.  Device-detected errors go to
 * the table's status word.  Errors returned at once: WRS_EINVAL. */
wrs_status wrs_table_build(wrs_table *t, const void *d_weights, uint64_t n,
                           wrs_dtype dtype, void *stream);

/* Build options.  The table does not depend on any of them (Alg. 3 gives
 * Alg. 2's table for every split count, Sec. 4.2); they choose how the work
 * is cut and which exact arithmetic the pack uses.
 *   splits  number of subproblems of Alg. 3's pack (one per block of the
 *           sweep, each a run of consecutive 2048-weight tiles); 0: the
 *           library's choice (8 tiles per subproblem); at most the number
 *           of tiles, ceil(n / 2048)
 *   tile    0 or 2048 (the tile is fixed)
 *   window  0 or 2048: the sweep merges a subproblem's lights with the
 *           heavy items of one stream tile at a time (its window; fixed)
 *   acc     WRS_ACC_AUTO: 64-bit bucket arithmetic when Q < 2^64, else
 *           128-bit; WRS_ACC_U64: the build fails with WRS_EOVERFLOW (in
 *           the status word) when Q >= 2^64; WRS_ACC_U128: 128-bit
 *           arithmetic throughout.  Keys are 128-bit in every mode.  There
 *           is no binary64 mode: every mode is exact.
 *   flags   0 */
typedef enum { WRS_ACC_AUTO = 0, WRS_ACC_U64 = 1, WRS_ACC_U128 = 2 } wrs_acc;
typedef struct {
    uint32_t splits;
    uint32_t tile;
    uint32_t window;
    uint32_t acc;   /* a wrs_acc */
    uint32_t flags;
} wrs_build_opts;

/* wrs_table_build with options (NULL: the defaults).  Errors returned at
 * once: WRS_EINVAL (as wrs_table_build, or an option out of range). */
wrs_status wrs_table_build_opts(wrs_table *t, const void *d_weights, uint64_t n, wrs_dtype dtype,
                                const wrs_build_opts *opts, void *stream);

/* Build the alias table of n weights with PSA+ (Sec. 4.2 "Performance
 * Optimization in Practice"): every tile of 2048 consecutive items first runs
 * Alg. 2 on its own items, in the global units (capacity Q, item i weighs
 * n * q_i), until the next light or the next heavy item it needs lies outside
 * the tile; the heavy item current at that point keeps its unassigned
 * residual, and the items left over from all tiles, in index order, are built
 * by Alg. 2 (PSA) as one list.  Full buckets point to themselves.  The table
 * differs from wrs_table_build's (the tiles pair items locally) but obeys the
 * same contract, and wrs_sample and every other table call accept it.
 * Arguments, ownership and errors as for wrs_table_build.  The first PSA+
 * build of a table allocates 40 B per weight of its capacity (stream-ordered
 * cudaMallocAsync on `stream`), kept until wrs_table_free; later builds
 * allocate nothing.  Asynchronous. */
wrs_status wrs_table_build_psa_plus(wrs_table *t, const void *d_weights, uint64_t n,
                                    wrs_dtype dtype, void *stream);

/* Number of items the last build's tile phase left over (the length of the
 * list the second phase built), when that build was wrs_table_build_psa_plus.
 * Waits for that build (as wrs_table_status).  Errors: WRS_EINVAL (no PSA+
 * build is the table's last), WRS_EDEVICE. */
wrs_status wrs_table_psa_plus_leftovers(const wrs_table *t, uint64_t *n_left);

/* wrs_table_create(n) followed by wrs_table_build(). */
wrs_status wrs_build(const void *d_weights, uint64_t n, wrs_dtype dtype,
                     void *stream, wrs_table **out);

/* Draw k samples with replacement (Sec. 2.2 query, k times; Sec. 5 Cor.
 * "kWR"): for s in [0, k), Philox4x32-10 with counter (s, stream_id) and key
 * seed gives 128 bits; the low 64 bits u pick bucket r = floor(u * n / 2^64),
 * the high 64 bits toss r's coin; d_out[s] = heads ? r : alias_r.  d_out:
 * caller-owned device memory for k uint32.  k may be 0.  Asynchronous,
 * ordered after the last build on the stream the caller chose.  Does not
 * synchronise: if the last build failed on the device, the kernel writes
 * nothing and wrs_table_status() reports why.  Errors returned at once:
 * WRS_EINVAL (bad argument, table never built), or a failed build's status
 * if wrs_table_status()/wrs_table_info_get() already read it. */
wrs_status wrs_sample(const wrs_table *t, uint64_t k, uint64_t seed,
                      uint64_t stream_id, uint32_t *d_out, void *stream);

/* End-to-end variants with HOST buffers: copy h_weights (n words) to the
 * table's device staging buffer, build, and return after enqueueing; and
 * sample into device staging memory and copy the k results to h_out.  The
 * copies are stream-ordered cudaMemcpyAsync calls; pinned host memory makes
 * them asynchronous.  wrs_sample_host synchronises `stream` before it
 * returns, so h_out is ready.  Staging memory is allocated on first use and
 * kept by the table (so the first call allocates; later calls of equal or
 * smaller size do not). */
wrs_status wrs_table_build_host(wrs_table *t, const void *h_weights, uint64_t n,
                                wrs_dtype dtype, void *stream);
wrs_status wrs_sample_host(wrs_table *t, uint64_t k, uint64_t seed,
                           uint64_t stream_id, uint32_t *h_out, void *stream);

/* Wait for the table's last build to complete (the host waits for that
 * build's event only, not for the device or other tables' work) and return
 * its status word. */
wrs_status wrs_table_status(const wrs_table *t);

/* Wait for the table's last build (as wrs_table_status) and fill *info
 * (header of the last build). */
wrs_status wrs_table_info_get(const wrs_table *t, wrs_table_info *info);

/* Device pointer to the n buckets (wrs_bucket[n]) of the last build; owned
 * by the table, valid until the table is freed or rebuilt. */
const wrs_bucket *wrs_table_buckets(const wrs_table *t);

/* Wait for the table's last build (as wrs_table_status) and copy n buckets
 * to h_buckets (bytes >= 16 n). */
wrs_status wrs_table_download(const wrs_table *t, void *h_buckets, uint64_t bytes);

/* Install buckets computed elsewhere (for testing the query on its own):
 * copies n buckets from host memory and sets Q, beta; shift and qp are
 * derived from Q as in a build.  Ordered after every earlier operation on
 * the table, on a stream of the library's own; returns when the copy is
 * complete. */
wrs_status wrs_table_upload(wrs_table *t, const void *h_buckets, uint64_t n,
                            uint64_t q_lo, uint64_t q_hi, int32_t beta);

/* Stage timing: when enabled, every later build records CUDA events on its
 * stream between its six kernels (weight total, total combine, tile
 * classification, look-back scan of the tile sums, split search, sweep).
 * wrs_table_stage_ms waits for the last build and writes the first `count`
 * (<= 6) stage durations in milliseconds.
 * Enabling creates the events (no device memory); errors: WRS_EINVAL when
 * timing is off or no timed build exists. */
wrs_status wrs_table_set_timing(wrs_table *t, int enable);
wrs_status wrs_table_stage_ms(const wrs_table *t, float *ms, uint32_t count);

/* Free the table.  Stream-ordered: the device memory is released once every
 * operation enqueued on the table (builds and samples, on whichever streams
 * the caller used) has completed; the call itself does not wait.  The
 * caller must not enqueue further work on the table.  NULL ok. */
void wrs_table_free(wrs_table *t);

/* Static string for a status code. */
const char *wrs_status_str(wrs_status s);

/* Check build.  libwrs_check.so is this library compiled with WRS_CHECK=1,
 * with the same entry points and the same tables, for verification (it is
 * slower; the standard library is libwrs.so).  In the check build:
 *   - every build first zeroes its bucket array, and every bucket store
 *     adds one to the bucket's reserved word instead of storing 0, so a
 *     build that wrote each bucket exactly once (Alg. 2 and Alg. 3 assign
 *     every bucket to one step) leaves 1 in every reserved word, and a
 *     missed or doubled bucket shows as 0 or 2 in the downloaded table;
 *   - a bucket index or alias outside the table, a shared-memory index of
 *     the sweep outside its window, a sweep subproblem that ends in another
 *     heavy tile than the split search gave the next one (Alg. 3: the state
 *     at the end of one subproblem is the start of the next), and a sampled
 *     bucket whose alias lies outside the table each count as a failed
 *     check: the access is skipped, the table's status becomes
 *     WRS_EINTERNAL and the count goes to the header's first reserved word.
 * wrs_check_build: 1 in the check build, 0 in the standard build.
 * wrs_table_check_failures: wait for the table's last build (as
 *   wrs_table_status) and store in *failures the failed checks counted
 *   since that build began (0 in the standard build; failures of a
 *   sampling are counted once the sampling has completed, so synchronize
 *   its stream first).  WRS_EINVAL for NULL arguments or a table never
 *   built. */
int wrs_check_build(void);
wrs_status wrs_table_check_failures(const wrs_table *t, uint64_t *failures);

/* Device-side wait limit used by the look-back scan of a build, in polls
 * (default 1 << 22, about a second).  Returns the previous value.  A build
 * whose wait runs out stores WRS_ETIMEOUT in the table's status. */
uint32_t wrs_set_wait_limit(uint32_t polls);

/* Test hook: during the next build, block `tile` of the look-back scan (it
 * covers 256 tiles of 2048 weights) publishes nothing, so its successor's
 * bounded wait runs out and the build ends with WRS_ETIMEOUT instead of
 * waiting forever.  -1 (the default) disables it.  For failure-detection
 * tests only. */
void wrs_debug_skip_publish(int64_t tile);

/*
 * Batched build and sampling of many independent tables.
 *
 * The paper treats one distribution; systems that draw from thousands of
 * small and mid-sized distributions at once (Sec. 4.2 notes that PSA's
 * subproblems are independent; Sec. 6 gives every PE its own table) pay a
 * launch sequence per table.  A batch instead runs each stage of the build
 * as ONE launch over all its tables, and all their samples as one more.
 * Table t of a batch gets exactly the buckets wrs_table_build gives its
 * weights, and exactly the samples of wrs_sample(table_t, k_t, seed,
 * stream_id + t): batching changes no result.  A failed table (bad weight,
 * total out of range) reports its own status and leaves the others intact.
 *
 * Layout: the weights of all tables sit in ONE device buffer of dtype words,
 * table t starting at word offset[t] (each table 16-byte aligned: offsets
 * are multiples of 4 words; the gaps are never read).  The buckets follow
 * the same offsets in the batch's own bucket array.  Sample outputs of table
 * t start at k_offset[t] of the caller's output buffer.
 *
 * Nothing passed to a launch changes between builds of the same batch
 * (the look-back generation is kept in device memory), so the caller may
 * capture wrs_batch_build + wrs_batch_sample in a CUDA graph and replay it
 * after rewriting the weights in place.
 */
typedef struct wrs_batch wrs_batch; /* opaque; device memory owned by the library */

/* Word offsets of ntables tables of h_n[t] weights (1 <= h_n[t] < 2^32) in a
 * batch's weight buffer: h_offsets[0..ntables], the last entry the total
 * length in words.  Host only (no device call). */
wrs_status wrs_batch_offsets(uint32_t ntables, const uint64_t *h_n, uint64_t *h_offsets);

/* Allocate a batch (buckets and workspace) for ntables tables of h_n[t]
 * weights, 1 <= ntables < 2^31.  Synchronous.  Errors: WRS_EINVAL, WRS_ENOMEM. */
wrs_status wrs_batch_create(uint32_t ntables, const uint64_t *h_n, wrs_batch **out);

/* The batch's offsets, as wrs_batch_offsets (ntables + 1 entries). */
wrs_status wrs_batch_layout(const wrs_batch *b, uint64_t *h_offsets);

/* Device pointer to the batch's buckets (table t at offset[t]). */
const wrs_bucket *wrs_batch_buckets(const wrs_batch *b);

/* Build every table from d_weights (device, 4-byte aligned, laid out by
 * offset[]).  Asynchronous on `stream`: seven kernel launches, no host
 * synchronisation, no allocation.  Device-detected errors land in the
 * tables' statuses (wrs_batch_status). */
wrs_status wrs_batch_build(wrs_batch *b, const void *d_weights, wrs_dtype dtype, void *stream);

/* Sample plan: table t draws h_k[t] samples (0 allowed).  Writes the output
 * offsets to h_k_offsets[0..ntables] when not NULL (last entry: total).
 * Synchronous; allocates device memory when the plan grows. */
wrs_status wrs_batch_set_samples(wrs_batch *b, const uint64_t *h_k, uint64_t *h_k_offsets);

/* Draw the planned samples of every built table into d_out (device, total
 * entries): table t's k_t samples are those of wrs_sample with stream id
 * stream_id + t.  One launch, asynchronous; a failed table writes nothing. */
wrs_status wrs_batch_sample(const wrs_batch *b, uint64_t seed, uint64_t stream_id, uint32_t *d_out,
                            void *stream);

/* Synchronise and write every table's status to h_status[0..ntables-1]
 * (may be NULL).  Returns the first failing table's status, or WRS_OK. */
wrs_status wrs_batch_status(const wrs_batch *b, int32_t *h_status);

/* Synchronise and fill *info for table `table` of the last build. */
wrs_status wrs_batch_table_info(const wrs_batch *b, uint32_t table, wrs_table_info *info);

/* Synchronise and copy all buckets (offset[ntables] of them) to h_buckets
 * (bytes >= 16 * offset[ntables]); the gaps between tables hold no bucket. */
wrs_status wrs_batch_download(const wrs_batch *b, void *h_buckets, uint64_t bytes);

/* Autotuning of the sweep.  Tables fall in WRS_BATCH_CLASSES size classes by
 * tiles of 2048 weights (1, 2-4, 5-32, 33-256, more); within a class every
 * sweep block takes `group` consecutive tiles of one table (the number of
 * split subproblems of a table is its tiles / group).  wrs_batch_tune builds
 * the batch from d_weights, then for each class present times the sweep
 * with group 1, 2, 4 and 8 (best of three each, CUDA events) and keeps the
 * fastest; finally it rebuilds with the chosen groups and writes the tuned
 * sweep time to *h_sweep_ms when not NULL.  Synchronous.  The groups change
 * speed only, never a bucket. */
#define WRS_BATCH_CLASSES 5
wrs_status wrs_batch_tune(wrs_batch *b, const void *d_weights, wrs_dtype dtype, void *stream,
                          float *h_sweep_ms);
wrs_status wrs_batch_groups(const wrs_batch *b, uint32_t *h_groups);             /* WRS_BATCH_CLASSES entries */
wrs_status wrs_batch_set_groups(wrs_batch *b, const uint32_t *h_groups);         /* each 1..64; synchronous */

/* Free all memory of the batch (synchronises the device first).  NULL ok. */
void wrs_batch_free(wrs_batch *b);

/*
 * Many sample requests in one launch (serving; no counterpart in the paper).
 *
 * A request server coalesces the sample requests that arrive while the GPU
 * is busy into one launch over all the tables they name.  Task i draws k
 * samples from the table (buckets, header) exactly as wrs_sample(table, k,
 * seed, stream_id) would, into d_out[out_offset ...]: coalescing changes no
 * result.
 *
 *   d_tasks   device array of ntasks tasks (16-byte aligned), ordered by
 *             out_offset with out_offset[i+1] = out_offset[i] + k[i]
 *             (k = 0 allowed); buckets/header point into a built table that
 *             stays resident until the launch completes
 *   total_k   out_offset + k of the last task; d_out holds total_k entries
 *
 * Asynchronous on `stream`; one launch; a task whose table failed to build
 * writes nothing.  Errors returned at once: WRS_EINVAL. */
typedef struct {
    const wrs_bucket *buckets; /* device: the table's n buckets */
    const void *header;        /* device: wrs_table_device_header / wrs_batch_device_header */
    uint64_t n;                /* buckets of the table */
    uint64_t k;                /* samples to draw */
    uint64_t seed, stream_id;  /* as wrs_sample */
    uint64_t out_offset;       /* first output entry */
    uint64_t reserved;         /* zero */
} wrs_sample_task;

wrs_status wrs_sample_many(const wrs_sample_task *d_tasks, uint32_t ntasks, uint64_t total_k,
                           uint32_t *d_out, void *stream);

/* Device address of a table's header (for wrs_sample_task.header). */
const void *wrs_table_device_header(const wrs_table *t);
const void *wrs_batch_device_header(const wrs_batch *b, uint32_t table);

/*
 * Two-level ("2lvl-sweep") tables: Sec. 6 "Distributed Alias Table
 * Construction" with the replicated top level, and Sec. 10 "Implementation
 * Details" (2lvl with Alg. 2 as the base case), applied recursively on one GPU.
 *
 * The items are cut into groups of WRS_TABLE2_GROUP consecutive items; each
 * group gets its own Alg. 2 table in the group's units (capacity Q_g = the
 * group's exact total, member m weighs n_g * q_m, n_g = members of the group;
 * buckets encoded as wrs_bucket with the group's shift and qp); the group
 * totals are the items of the next level, up to one group (at most three
 * levels for n < 2^32).  An alias is the member's index within its level.
 * Sample s walks down from the top group: at depth d (0 at the top), Philox
 * with counter (s, stream_id) and key (seed_lo + d * 0x9E3779B9, seed_hi +
 * d * 0xBB67AE85) gives u, v; r = floor(u * n_g / 2^64) picks a bucket of the
 * current group, heads iff floor(v * qp_g / 2^64) < thr keeps r, else the
 * alias; the pick is the group one level down, and at level 0 the sample.
 * With n <= WRS_TABLE2_GROUP the table and the samples are exactly those of
 * wrs_table_build and wrs_sample.  Each item is drawn with probability
 * w_i / W up to the same per-level discretisation as the single table.
 * It is a different table from wrs_table_build's for larger n, built in two
 * passes over the weights (exact total, then one block per group) with no
 * global prefix or split search.
 *
 * Arguments, ownership, streams and errors as for the wrs_table_* calls.
 */
#define WRS_TABLE2_GROUP 2048
#define WRS_TABLE2_MAX_LEVELS 4
typedef struct wrs_table2 wrs_table2;
typedef struct {
    uint64_t qp;        /* Q_g >> shift: the group's coin denominator */
    uint32_t shift;     /* max(0, bitlen(Q_g) - 64) */
    uint32_t members;   /* n_g */
} wrs_group;

wrs_status wrs_table2_create(uint64_t capacity_n, wrs_table2 **out);
wrs_status wrs_table2_build(wrs_table2 *t, const void *d_weights, uint64_t n, wrs_dtype dtype, void *stream);
wrs_status wrs_table2_sample(const wrs_table2 *t, uint64_t k, uint64_t seed, uint64_t stream_id,
                             uint32_t *d_out, void *stream);
/* Synchronise; the build's status (device-detected errors as wrs_table_status). */
wrs_status wrs_table2_status(const wrs_table2 *t);
/* Levels of the last build and their sizes (h_sizes: WRS_TABLE2_MAX_LEVELS entries, may be NULL). */
wrs_status wrs_table2_layout(const wrs_table2 *t, uint32_t *h_levels, uint64_t *h_sizes);
/* Synchronise and copy the buckets of all levels (level 0 first, 16 B each)
 * and the group records (level 0's groups first); either pointer may be NULL. */
wrs_status wrs_table2_download(const wrs_table2 *t, void *h_buckets, uint64_t bucket_bytes,
                               void *h_groups, uint64_t group_bytes);
void wrs_table2_free(wrs_table2 *t);

/* Output-sensitive sampling with replacement, OS-ND variant (Sec. 5 "Output
 * Sensitive Sampling With Replacement"; Sec. 10 "Optimizations": descent
 * aborted for fewer than 128 samples from at least half as many items, no
 * deduplication), over a built two-level table.  Draws k samples and writes
 * them as (item, count) pairs: every item reached by the divide-and-conquer
 * descent once with its count, and one (item, 1) pair per alias query of the
 * base case, in no particular order; the counts add up to k.  Within a group
 * a binary tree over its members (node [a, b) splits at a + (b - a) / 2)
 * gives Binomial(c, W_left / W_node) of a node's c samples to its left
 * child; a group receiving c < 128 samples from at least c/2 members draws
 * them as alias queries.  Random bits: Philox4x32-10, key seed, counter (g,
 * h | level << 12 | j << 14, stream_id) with g the group, h the node's heap
 * index (root 1; 0 for alias queries) and j the draw.  Binomial deviates:
 * inversion when c p < 10, else Hoermann's BTRS, with binary64 log and exp
 * from their series (no library math), so the pairs are a function of the
 * table, the weights, k, seed and stream_id.
 *
 *   d_weights  the words the table was built from (same dtype), device
 *   d_items, d_counts  output, capacity entries each (device)
 *   d_npairs   output (device u64): pairs produced; when it exceeds capacity
 *              the pairs past capacity were not written
 * Asynchronous on `stream`; allocates frontier buffers on first use. */
wrs_status wrs_table2_sample_os(wrs_table2 *t, const void *d_weights, wrs_dtype dtype, uint64_t k, uint64_t seed,
                                uint64_t stream_id, uint32_t *d_items, uint64_t *d_counts, uint64_t capacity,
                                uint64_t *d_npairs, void *stream);

/*
 * Build without allocating (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc -- real-time or embedded processes
 * whose device memory is fixed at start-up, host frameworks that own all
 * device memory through their own pool and forbid allocations behind its
 * back -- this entry point builds the same table as wrs_table_build
 * (bucket for bucket) into memory the caller owns, and keeps its scratch in
 * one static device array inside the library, sized for WRS_NOALLOC_MAX_N
 * weights (about 0.5 MB; every GPU that loads the library holds it until the
 * process exits).  It allocates nothing and calls no allocating routine.
 *
 *   d_weights  n words of dtype, device memory, 4-byte aligned, read only
 *   d_buckets  output: n wrs_bucket, device memory, 16-byte aligned
 *   d_header   output: one wrs_device_header (WRS_DEVICE_HEADER_BYTES),
 *              device memory, 16-byte aligned; its status word reports
 *              device-detected errors as in wrs_table_status()
 *   n          1 .. WRS_NOALLOC_MAX_N; larger n returns WRS_EINVAL at once
 *              (use wrs_table_create/wrs_table_build instead)
 *
 * Asynchronous on `stream`.  The first call on a device looks up the static
 * array's device address (cudaGetSymbolAddress) and sets the sweep kernel's
 * shared-memory attribute; make that first call before any stream capture.
 * All calls share the one array: two calls whose work overlaps on the GPU
 * (different streams, or several host threads) race and corrupt each
 * other's results, so order them (one stream, or events).  The array keeps
 * the last call's contents; the one part that must start at zero, the
 * look-back flags, is cleared by each call on `stream` (cudaMemsetAsync,
 * which allocates nothing) before the scan that reads them. */
#define WRS_NOALLOC_MAX_N (1ull << 22)
#define WRS_DEVICE_HEADER_BYTES 128

/* Every field but reserved2[2..7] is written by every build; the caller
 * only reads them.  The two fields marked "library" are working state of
 * the build: their values after a build carry no meaning for the caller,
 * and the caller must not store into them. */
typedef struct {
    uint32_t status;      /* wrs_status of the build */
    uint32_t tile_counter; /* library: block ids of the look-back scan */
    int32_t beta;         /* exponent of the integer unit */
    uint32_t shift;       /* thr = bw >> shift */
    uint64_t q_lo, q_hi;  /* Q */
    uint64_t qp;          /* Q >> shift: the sampler's coin denominator */
    uint32_t light_max;   /* light iff raw word <= light_max */
    uint32_t f32;         /* library: 1 if the weights were binary32 words */
    uint64_t n;
    uint64_t n_light;
    uint64_t reserved2[8]; /* [0], [1]: zero after a build of libwrs.so; the
                              check build counts failed checks in [0] */
} wrs_device_header;

wrs_status wrs_build_noalloc(const void *d_weights, uint64_t n, wrs_dtype dtype,
                             void *d_buckets, void *d_header, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WRS_H */
