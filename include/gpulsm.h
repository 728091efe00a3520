/*
 * gpulsm.h - C ABI of the GB300-native GPU LSM dictionary.
 *
 * The data structure is the GPU LSM of Ashkiani, Li, Farach-Colton, Amenta and
 * Owens ("GPU LSM: A Dynamic Dictionary Data Structure for the GPU", arXiv
 * 1707.05354): a dictionary of 31-bit keys and 32-bit values, updated in
 * batches of a fixed size b, stored as sorted levels of b * 2^i elements that
 * fill and empty like the bits of a binary counter (§III-B).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Pointers named d_* are caller-owned DEVICE memory on the handle's device
 *    (for instance torch.Tensor.data_ptr()); the library never frees or keeps
 *    them after the call's work has run.  Pointers named h_* are host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; outputs are valid once the stream has
 *    reached that point.  Calls that must read a device value on the host
 *    (documented below) synchronise with the stream before returning.
 *  - Update calls sort each batch on `stream` and fold it into the levels on
 *    an internal stream of the handle, so that the next batch's sort can
 *    overlap the fold.  Once `stream` has passed an update call, the call's
 *    inputs have been consumed; the fold may still be running.  Every later
 *    call that reads or rewrites the levels (lookup, count, range, cleanup,
 *    dump) first orders its stream after the handle's folds, so results are
 *    always those of every update issued before; lsm_stream_wait orders any
 *    other work (a timing event, a copy) the same way.
 *  - Keys are 32-bit unsigned integers; user keys must be < 2^31 - 1.  The key
 *    2^31 - 1 is reserved for the placebo tombstones written by cleanup (§IV-E).
 *    Values are arbitrary 32-bit unsigned integers.
 *  - Inside the structure a key is stored as the "key variable"
 *    (key << 1) | status, status 1 = regular element, 0 = tombstone (§IV-A).
 *  - Errors: a call that returns anything but LSM_OK has changed nothing in
 *    the dictionary (all or nothing), unless its description says otherwise.
 *  - A handle is not thread-safe, and its query calls share one scratch area:
 *    calls on one handle are issued from one thread, and query calls on
 *    different streams are ordered by the caller.  Distinct handles are
 *    independent.
 *  - Batch semantics (§III-A): batches apply in call order; within a batch a
 *    delete of a key beats every insert of it (rule 6) and among several
 *    inserts of one key the last in input order wins (the library's reading
 *    of rule 4, which lets the choice be arbitrary).
 */
#ifndef GPULSM_H
#define GPULSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsm_t lsm_t; /* opaque; owned by the library */

typedef enum {
  LSM_OK = 0,
  LSM_ERR_ARG = 1,        /* null handle/pointer, b = 0, n > b for update, ... */
  LSM_ERR_KEY_RANGE = 2,  /* an update key is >= 2^31 - 1                      */
  LSM_ERR_FULL = 3,       /* the batch would need a level beyond the capacity  */
  LSM_ERR_OOM = 4,        /* a device or pinned allocation failed              */
  LSM_ERR_BUDGET = 5,     /* the allocation would exceed the handle's budget   */
  LSM_ERR_CAPACITY = 6,   /* range output does not fit in the caller's buffer  */
  LSM_ERR_CUDA = 7,       /* a CUDA runtime call or kernel launch failed       */
  LSM_ERR_TIMEOUT = 8     /* a bounded device-side wait gave up                */
} lsm_status;

/* Human-readable name of a status code (static string). */
const char* lsm_status_str(lsm_status s);

/*
 * lsm_create - allocate an empty dictionary with batch size b (§III-A rule 1).
 *   out           receives the handle.
 *   b             batch size, 1 <= b <= 2^26.
 *   max_elements  resident elements (counting stale ones and tombstones) to
 *                 provide room for: the library allocates the smallest number
 *                 of levels L with b * (2^L - 1) >= max_elements (at least 1),
 *                 and at most 2^31 elements in all.
 *   device        CUDA device ordinal; the handle's memory lives there and every
 *                 later call must run with that device's streams.
 * Device memory: 8 bytes per element of every level, plus scratch of about
 * 16 * b bytes for the batch sort.  Levels are laid out in one array, level i
 * after level i - 1 (§IV-A, Fig. 3), each level's start rounded up to a
 * multiple of 32 elements.
 * Errors: LSM_ERR_ARG, LSM_ERR_OOM, LSM_ERR_CUDA.
 */
lsm_status lsm_create(lsm_t** out, uint32_t b, uint64_t max_elements, int device);

/* lsm_destroy - release every allocation of the handle (NULL is accepted).
 * Waits for the handle's outstanding work first. */
void lsm_destroy(lsm_t* h);

/*
 * lsm_insert_batch - insert n (key, value) pairs (§III-B, Fig. 2(a), Fig. 3).
 *   d_keys, d_vals  n keys and n values, device memory, read-only.
 *   n               any count; the ops are applied as ceil(n / b) consecutive
 *                   batches of b ops, a final short batch padded with copies of
 *                   its last op (§IV-A).  n = 0 is a no-op.
 * Each batch is sorted on the full key variable and cascade-merged into level
 * ffz(r), r the number of resident batches (the merge on the handle's
 * internal stream; see the conventions above).  Keys are checked on the
 * device; the call waits for that check (not for the merge) and returns
 * LSM_ERR_KEY_RANGE with nothing applied if any key is >= 2^31 - 1.
 * Errors: LSM_ERR_ARG, LSM_ERR_KEY_RANGE, LSM_ERR_FULL, LSM_ERR_CUDA.
 */
lsm_status lsm_insert_batch(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                            uint64_t n, void* stream);

/*
 * lsm_delete_batch - delete n keys by inserting tombstones (§III-C).
 * Same batching, padding, checks and errors as lsm_insert_batch; tombstones
 * carry the value 0.
 */
lsm_status lsm_delete_batch(lsm_t* h, const uint32_t* d_keys, uint64_t n, void* stream);

/*
 * lsm_update_batch - one mixed batch of n <= b inserts and deletes (§III-A
 * rule 2).  d_is_delete[i] != 0 makes op i a delete (its value is ignored).
 * n < b is padded with copies of op n - 1.
 * Errors: LSM_ERR_ARG (n > b), LSM_ERR_KEY_RANGE, LSM_ERR_FULL, LSM_ERR_CUDA.
 */
lsm_status lsm_update_batch(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                            const uint8_t* d_is_delete, uint64_t n, void* stream);

/*
 * lsm_update_batch_ordered - one mixed batch of n <= b ops that take effect
 * in input order: the last op on a key decides, so a delete followed by an
 * insert of the same key leaves it inserted (applying the ops one by one).
 * Not in the paper, whose rule 6 (§III-A) lets a delete win inside a batch;
 * this is how the serving engine coalesces requests into one batch.  Before
 * the usual sort, every op on a key is replaced on the device by a copy of
 * the last op on that key.  d_vals may be NULL (values 0), d_is_delete NULL
 * (all inserts).  Same checks, errors and asynchrony as lsm_update_batch.
 */
lsm_status lsm_update_batch_ordered(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                                    const uint8_t* d_is_delete, uint64_t n, void* stream);

/*
 * lsm_lookup - point queries (§III-D, §IV-B, Fig. 2(b)).
 *   d_q       nq query keys (any 32-bit value; keys >= 2^31 - 1 are never found).
 *   d_val     nq outputs: the value, or 0 when not found.
 *   d_found   nq outputs: 1 when the key is present, else 0.
 * Full levels are searched from the newest (smallest) to the oldest; the first
 * element of the key found decides: regular -> found, tombstone -> absent.
 * nq = 0 is a no-op.  Asynchronous.
 */
lsm_status lsm_lookup(lsm_t* h, const uint32_t* d_q, uint64_t nq, uint32_t* d_val,
                      uint8_t* d_found, void* stream);

/*
 * lsm_count - number of live keys k with k1[i] <= k <= k2[i] (§III-E, §IV-C,
 * Fig. 2(c)).  Bounds are inclusive; k1 > k2 gives 0; k2 >= 2^31 - 1 is treated
 * as 2^31 - 2.  d_count receives nq counts.  Asynchronous.  Uses the handle's
 * query scratch (4 (nq + 1) bytes, grown on demand; growing it synchronises
 * the device): a query whose level windows hold many elements is counted by
 * a warp of its own (see the note on handles above).
 */
lsm_status lsm_count(lsm_t* h, const uint32_t* d_k1, const uint32_t* d_k2, uint64_t nq,
                     uint32_t* d_count, void* stream);

/*
 * lsm_successor / lsm_predecessor - the order-based queries the paper's
 * problem statement names beside lookup, count and range (§II-A footnote),
 * read inclusively: the live pair with the smallest key >= q (successor) or
 * the largest key <= q (predecessor).  d_key/d_val/d_found receive nq
 * results; found = 0 (and key = value = 0) when there is none.  Keys above
 * 2^31 - 2 are never live.  Asynchronous.
 */
lsm_status lsm_successor(lsm_t* h, const uint32_t* d_q, uint64_t nq, uint32_t* d_key, uint32_t* d_val,
                         uint8_t* d_found, void* stream);
lsm_status lsm_predecessor(lsm_t* h, const uint32_t* d_q, uint64_t nq, uint32_t* d_key, uint32_t* d_val,
                           uint8_t* d_found, void* stream);

/*
 * lsm_range - every live (key, value) with k1[i] <= key <= k2[i] (§III-E,
 * §IV-D, Fig. 2(d)), as compressed rows:
 *   d_offsets  nq + 1 device uint64: query i owns output slots
 *              [d_offsets[i], d_offsets[i+1]).
 *   d_keys, d_vals  output keys (original 31-bit keys, ascending within a
 *              query) and their values; room for `capacity` entries.
 *   total_out  host pointer receiving the total number of results.
 * The call synchronises with the stream to learn the total.  If the total
 * exceeds `capacity`, d_offsets and *total_out are written, nothing else is,
 * and LSM_ERR_CAPACITY is returned (retry with a larger buffer).
 */
lsm_status lsm_range(lsm_t* h, const uint32_t* d_k1, const uint32_t* d_k2, uint64_t nq,
                     uint64_t* d_offsets, uint32_t* d_keys, uint32_t* d_vals,
                     uint64_t capacity, uint64_t* total_out, void* stream);

/*
 * lsm_cleanup - remove every stale element and tombstone and rebuild the
 * levels (§III-F, §IV-E).  Afterwards r = ceil(n' / b) for n' live keys; the
 * sorted live pairs fill the set bits of r in ascending level order (smaller
 * keys in smaller levels) and r * b - n' placebo tombstones of key 2^31 - 1
 * (value 0) end the largest level.  Query results are unchanged.
 * Needs a scratch of 8 bytes per resident element, allocated on first use and
 * kept.  Synchronises with the stream (the host must learn n').
 * Errors: LSM_ERR_OOM, LSM_ERR_CUDA, LSM_ERR_TIMEOUT.
 */
lsm_status lsm_cleanup(lsm_t* h, void* stream);

/*
 * lsm_bulk_build - fill an EMPTY dictionary (r = 0) with n (key, value)
 * pairs at once: the same query results as lsm_insert_batch of the pairs (the
 * last occurrence of a key wins), laid out as a cleanup leaves the levels
 * (the live pairs sorted, filling the set bits of r = ceil(n'/b), placebos
 * after them).  One stable sort of all n pairs (the paper's bulk build, §V)
 * and the cleanup's compaction; needs temporary device memory of about
 * 18 bytes per pair.  Synchronises.
 * Errors: LSM_ERR_ARG (not empty), LSM_ERR_FULL (n > capacity),
 * LSM_ERR_KEY_RANGE, LSM_ERR_OOM, LSM_ERR_CUDA.
 */
lsm_status lsm_bulk_build(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n, void* stream);

/*
 * lsm_stats - host-side state: r = resident batches, resident = r * b
 * elements, b = batch size, levels = number of allocated levels.  Any output
 * pointer may be NULL.  Does not touch the device.
 */
lsm_status lsm_stats(const lsm_t* h, uint64_t* r, uint64_t* resident, uint32_t* b,
                     uint32_t* levels);

/*
 * lsm_level_offset - element offset and size of level i inside the level
 * array (0 size when the level is not allocated).  For tests and tools.
 */
lsm_status lsm_level_offset(const lsm_t* h, uint32_t i, uint64_t* offset, uint64_t* size);

/*
 * lsm_dump_levels - copy every FULL level to host memory at the same element
 * offsets it has on the device (see lsm_level_offset); other positions are
 * left untouched.  h_keys/h_vals need lsm_capacity() elements.  Synchronises.
 */
lsm_status lsm_dump_levels(const lsm_t* h, uint32_t* h_keys, uint32_t* h_vals, void* stream);

/*
 * Checkpoint and resume (not in the paper; the state of a dictionary is its
 * batch size b, its batch count r and its full levels, §III-B).
 *
 * lsm_save - write the full levels, in ascending level order, to host
 * memory: level i (bit i of r set) as b * 2^i key variables ((key << 1) |
 * status, §IV-A) and as many values, one level after another.  h_keys and
 * h_vals hold `capacity` elements; the call needs r * b of them (else
 * LSM_ERR_CAPACITY, nothing written) and stores r in *r_out.  Synchronises
 * with `stream` after the folds in flight.
 *
 * lsm_load - make an empty handle (r = 0) hold a saved state: r and the
 * r * b elements written by lsm_save of a dictionary with the same b.  The
 * handle needs the levels of r (else LSM_ERR_FULL); every level is copied
 * to the device and its prefix index rebuilt.  b mismatch or r = 0 with
 * data: LSM_ERR_ARG.  The arrays are trusted to come from lsm_save (sorted
 * levels); the call does not re-sort them.  Asynchronous on `stream`: the
 * host arrays must stay valid until the stream has passed the call.
 */
lsm_status lsm_save(lsm_t* h, uint32_t* h_keys, uint32_t* h_vals, uint64_t capacity, uint64_t* r_out,
                    void* stream);
lsm_status lsm_load(lsm_t* h, const uint32_t* h_keys, const uint32_t* h_vals, uint64_t r, uint32_t b,
                    void* stream);

/*
 * lsm_reset - drop every element (r = 0).  Host-side only, no device work; the
 * level memory is reused by later batches (after any fold still in flight,
 * which the handle's stream order guarantees).  Waits for nothing.
 */
lsm_status lsm_reset(lsm_t* h);

/*
 * lsm_stream_wait - make `stream` wait (on the device, without blocking the
 * host) until every fold the handle has enqueued so far has finished.  Not in
 * the paper: it exposes the library's two-stream pipelining of updates.
 */
lsm_status lsm_stream_wait(lsm_t* h, void* stream);

/* Number of elements in the level array (all allocated levels, with padding). */
uint64_t lsm_capacity(const lsm_t* h);

/*
 * lsm_sort_pairs - the library's batch sort as a stand-alone call: stable
 * radix sort of n (key, value) pairs on the full 32-bit key (§IV-A sorts each
 * batch with a radix sort over the whole key variable): for n <= 2^20 a
 * bucket sort on the top byte followed by a sort of each bucket on the low
 * 24 bits, above that four 8-bit least-significant-digit passes.
 * d_keys_in/d_vals_in are read, d_keys_out/d_vals_out receive the sorted
 * pairs (they must not overlap the inputs).  Uses the handle's scratch, so
 * n <= b.  Asynchronous.  Used by tests of the sort in isolation.
 */
lsm_status lsm_sort_pairs(lsm_t* h, const uint32_t* d_keys_in, const uint32_t* d_vals_in,
                          uint32_t* d_keys_out, uint32_t* d_vals_out, uint64_t n,
                          void* stream);

/*
 * lsm_sort_pairs_noalloc - the same stable radix sort as lsm_sort_pairs, for
 * callers that must not allocate device memory while they run (for example a
 * process whose device memory all comes from its own pool and which forbids
 * raw cudaMalloc, or a latency-bound loop that cannot take the device-wide
 * synchronisation and unbounded time of a cudaMalloc/cudaFree).  No handle
 * is needed and nothing is allocated: every byte of scratch comes from one
 * fixed array with static storage inside the library (about 17 MB), which
 * each GPU that loads the library keeps until the process exits.
 *   n        at most LSM_SORT_NOALLOC_MAX_PAIRS; larger n is refused with
 *            LSM_ERR_CAPACITY before any work is queued.  n = 0 is a no-op.
 *   inputs/outputs as for lsm_sort_pairs (device memory on the current
 *            device, outputs must not overlap the inputs).  Asynchronous on
 *            `stream`, which must belong to the current device.
 * The first call on a device looks up that device's copy of the array and
 * clears it (queued on `stream`); make that first call before capturing
 * `stream` into anything.  All calls on a device share the one array, which
 * keeps the last call's contents; calls whose work overlaps on the GPU (two
 * streams at once) race on it and must be ordered by the caller.
 * The paper has no counterpart: this entry point exists for the callers above.
 */
#define LSM_SORT_NOALLOC_MAX_PAIRS (1u << 20)
lsm_status lsm_sort_pairs_noalloc(const uint32_t* d_keys_in, const uint32_t* d_vals_in,
                                  uint32_t* d_keys_out, uint32_t* d_vals_out, uint64_t n,
                                  void* stream);

/*
 * lsm_set_option / lsm_get_option - tuning knobs (integers):
 *   LSM_OPT_LOOKUP_MODE  0 = automatic, 1 = one search per query in input
 *                        order, 2 = sort the queries first (§IV-B "bulk").
 *   LSM_OPT_DEVICE_ERROR read-only: sticky device error bits seen so far
 *                        (1 = bad key, 2 = wait timeout, 4 = misaligned
 *                        copy avoided); synchronises; reading clears them.
 *   LSM_OPT_KERNEL_LAUNCHES read-only: CUDA kernels launched by the library
 *                        in this process so far (all handles); h may be NULL.
 *   LSM_OPT_KEY_CHECK    0 (default) = an update call waits for the device
 *                        check of its keys and returns LSM_ERR_KEY_RANGE,
 *                        having changed nothing, if one is >= 2^31 - 1.
 *                        1 = deferred, for callers that validate keys
 *                        upstream and want update calls that never wait:
 *                        a batch holding a bad key is applied as b placebo
 *                        tombstones (the reserved key 2^31 - 1, which no
 *                        query sees and cleanup drops), so it changes no
 *                        query result; r still advances, the call returns
 *                        LSM_OK, and bit 1 of LSM_OPT_DEVICE_ERROR records
 *                        it.  A call of n > b ops is then all or nothing
 *                        per batch.  Handles with b > 2^20 keep the
 *                        synchronous check.  Not in the paper.
 */
typedef enum {
  LSM_OPT_LOOKUP_MODE = 1,
  LSM_OPT_DEVICE_ERROR = 2,
  LSM_OPT_KERNEL_LAUNCHES = 3,
  LSM_OPT_KEY_CHECK = 4
} lsm_option;

lsm_status lsm_set_option(lsm_t* h, lsm_option opt, int64_t value);
lsm_status lsm_get_option(lsm_t* h, lsm_option opt, int64_t* value);

/*
 * Kernel profiler (tracing aid).  While enabled, the library brackets each of
 * its kernel groups with CUDA events on the call's stream and accumulates, per
 * group, the number of launches, their total device time and the ALGORITHMIC
 * bytes they had to move (the bytes an ideal implementation reads and writes
 * in HBM; scratch traffic excluded):
 *   LSM_PROF_SORT       batch sort (two kernels up to 2^20 elements, else a
 *                       histogram and four passes), 16 B per element
 *   LSM_PROF_PARTITION  fold co-rank search, 0 B (pure overhead)
 *   LSM_PROF_MERGE      fold merge into level k, 16 * 2^k * b B
 *   LSM_PROF_LOOKUP     lookup kernels, 9 B per query + 32 B per level probed
 *                       (upper bound: every level) + 4 B per query found
 *   LSM_PROF_COUNT      count / range window kernels, 12 B + 64 B per level
 *   LSM_PROF_EMIT       range output, 8 B per result + 8 B per query
 *   LSM_PROF_CLEANUP    cleanup merge + distribute, 8 B read per resident
 *                       element + 8 B written per element of r' * b
 * lsm_profile(h, 1) enables every group and zeroes the counters,
 * lsm_profile(h, 2 + g) enables group g alone (and zeroes the counters),
 * lsm_profile(h, 0) disables; any other value is LSM_ERR_ARG.
 * lsm_profile_read synchronises the device and fills `out` (LSM_PROF_COUNT_
 * entries).  Profiling adds two event records per launch of a profiled group;
 * an event between two kernels also ends the programmatic launch overlap of
 * the second with the first, so profiling one group (for instance the merge
 * while an insert phase is timed) perturbs the timing less than profiling all.
 */
typedef enum {
  LSM_PROF_SORT = 0,
  LSM_PROF_PARTITION = 1,
  LSM_PROF_MERGE = 2,
  LSM_PROF_LOOKUP = 3,
  LSM_PROF_COUNT = 4,
  LSM_PROF_EMIT = 5,
  LSM_PROF_CLEANUP = 6,
  LSM_PROF_COUNT_ = 7
} lsm_prof_group;

typedef struct {
  uint64_t launches;
  double ms;
  double bytes;
} lsm_profile_entry;

lsm_status lsm_profile(lsm_t* h, int enable);
lsm_status lsm_profile_read(lsm_t* h, lsm_profile_entry* out);


/* ========================================================================
 * Batched form: many independent dictionaries advanced together
 * ========================================================================
 * A multi handle holds n independent GPU LSMs.  Instance i has its own batch
 * size b_i (any integer in [1, 2^20]) and levels of b_i * 2^l elements
 * (§III-B), its own counter r_i and the same batch semantics as a plain
 * handle (§III-A).  A "round" gives every instance at most one batch; all
 * instances are sorted, folded and searched by the same few kernels, and the
 * round runs as one CUDA graph replay.  The paper treats one dictionary; the
 * batched form is this library's extension for many small ones.
 *
 * Input layout of a round: instance i's ops are at positions
 * [in_off_i, in_off_i + count_i) of the caller's d_keys / d_vals /
 * d_is_delete arrays, with in_off_i = b_0 + ... + b_{i-1}
 * (lsm_multi_layout returns it).  count_i = d_counts[i] (device array of n
 * u32; 0 = no batch for i this round) or b_i for every instance when d_counts
 * is NULL.  A short batch is padded like a plain one (copies of its last op).
 *
 * Errors inside a round are per instance and asynchronous: an instance whose
 * batch has a key >= 2^31 - 1, count_i > b_i, or would need a level beyond
 * the capacity keeps its state unchanged and the others proceed;
 * lsm_multi_sync reports it (and per-instance error bits).
 */
typedef struct lsm_multi_t lsm_multi_t; /* opaque; owned by the library */

/* Per-instance shape choices (see the autotuner in the Python package):
 * tile      output elements per merge work item: 1024 or 2048;
 * bin_log2  prefix-index resolution: about 2^bin_log2 elements per bin
 *           (1 .. 6), the fan-out of the first step of every level search. */
typedef struct {
  uint32_t tile;
  uint32_t bin_log2;
} lsm_multi_tuning;

/*
 * lsm_multi_create - n_inst empty instances with batch sizes h_b[0 .. n-1]
 * (host array), each able to take max_batches batches (levels 0 .. L - 1
 * with 2^L > max_batches, L <= 16; b_i * 2^(L-1) < 2^31).  h_tuning: n
 * entries or NULL (tile 2048, bin_log2 3).  Allocates every level, fence and
 * scratch buffer up front (about 2 * max_batches * b_i * 8 bytes per
 * instance plus 4 * b_i * 8 bytes of batch scratch).
 * Errors: LSM_ERR_ARG (bad sizes), LSM_ERR_OOM, LSM_ERR_CUDA.
 */
lsm_status lsm_multi_create(lsm_multi_t** out, uint32_t n_inst, const uint32_t* h_b, uint32_t max_batches,
                            const lsm_multi_tuning* h_tuning, int device);
void lsm_multi_destroy(lsm_multi_t* h);

/*
 * lsm_multi_update - one round of update batches (layout above): for every
 * instance with count_i > 0, encode + pad + stable sort of its batch
 * (§IV-A) and the cascade fold of the batch and levels 0 .. k_i - 1 into
 * level k_i = ffz(r_i) (§III-B, §IV-A); r_i += 1.  d_vals may be NULL (all
 * values 0), d_is_delete NULL (all inserts).  Asynchronous on `stream`; the
 * first call with a given set of pointers captures the round into a CUDA
 * graph, later calls with the same pointers replay it.
 */
lsm_status lsm_multi_update(lsm_multi_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                            const uint8_t* d_is_delete, const uint32_t* d_counts, void* stream);

/*
 * lsm_multi_lookup - LOOKUP (§III-D) for queries of many instances: query g
 * (0 <= g < nq) belongs to instance i with d_qoff[i] <= g < d_qoff[i + 1]
 * (device array of n + 1 u64, d_qoff[n] = nq).  Outputs as lsm_lookup.
 */
lsm_status lsm_multi_lookup(lsm_multi_t* h, const uint32_t* d_q, const uint64_t* d_qoff, uint64_t nq,
                            uint32_t* d_val, uint8_t* d_found, void* stream);

/*
 * lsm_multi_round - lsm_multi_update followed by lsm_multi_lookup (the
 * lookups see the round's batches), as ONE graph replay on `stream`.
 */
lsm_status lsm_multi_round(lsm_multi_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                           const uint8_t* d_is_delete, const uint32_t* d_counts, const uint32_t* d_q,
                           const uint64_t* d_qoff, uint64_t nq, uint32_t* d_val, uint8_t* d_found,
                           void* stream);

/*
 * lsm_multi_sync - synchronises `stream`, returns the first error seen by the
 * rounds since the last sync (LSM_ERR_TIMEOUT, LSM_ERR_KEY_RANGE,
 * LSM_ERR_ARG, LSM_ERR_FULL in that priority) and clears it.  h_flags (n u32
 * or NULL) receives the last round's per-instance bits: 1 bad key,
 * 8 count > b, 16 full.
 */
lsm_status lsm_multi_sync(lsm_multi_t* h, void* stream, uint32_t* h_flags);

/* Counter r_i, batch size b_i and resident elements r_i * b_i of instance i
 * (synchronous device read). */
lsm_status lsm_multi_stats(const lsm_multi_t* h, uint32_t i, uint64_t* r, uint32_t* b, uint64_t* resident);

/* Input offset, merge tile, level-0 prefix-index shift and level count of
 * instance i (host values; any pointer may be NULL). */
lsm_status lsm_multi_layout(const lsm_multi_t* h, uint32_t i, uint64_t* in_off, uint32_t* tile,
                            int32_t* fence_shift0, uint32_t* levels);

/* Full levels of instance i, ascending, as key variables and values into host
 * arrays of r_i * b_i entries (synchronises the device; tests). */
lsm_status lsm_multi_dump_levels(const lsm_multi_t* h, uint32_t i, uint32_t* h_keys, uint32_t* h_vals);

/* Empties every instance (r_i = 0) on `stream`; buffers are kept. */
lsm_status lsm_multi_reset(lsm_multi_t* h, void* stream);

/*
 *   LSM_MULTI_OPT_GRAPH          1 (default) = rounds run as CUDA graph
 *                                replays, 0 = plain launches.
 *   LSM_MULTI_OPT_GRAPH_KERNELS  read-only: kernel nodes of the last round replayed.
 *   LSM_MULTI_OPT_DEVICE_BYTES   read-only: device memory held by the handle.
 */
typedef enum {
  LSM_MULTI_OPT_GRAPH = 1,
  LSM_MULTI_OPT_GRAPH_KERNELS = 2,
  LSM_MULTI_OPT_DEVICE_BYTES = 3
} lsm_multi_option;

lsm_status lsm_multi_set_option(lsm_multi_t* h, int opt, int64_t value);
lsm_status lsm_multi_get_option(const lsm_multi_t* h, int opt, int64_t* value);


/* ========================================================================
 * Serving form: a continuous-batching request loop over one dictionary
 * ========================================================================
 * Not in the paper.  A server owns a dictionary of batch size b and replays
 * a trace of requests (insert, delete, lookup, count, range; each naming a
 * window of device-resident payload pools) in real time: requests become
 * visible at their arrival times, wait in an update queue and a retrieval
 * queue, and are admitted as groups into a few in-flight slots while earlier
 * groups still run:
 *   - an update group is whole update requests, up to b ops, applied as one
 *     ordered batch (lsm_update_batch_ordered), admitted when b ops are
 *     pending, when b/2 are pending and no update group is in flight, when
 *     its oldest request has waited flush_us, or at the end of the trace (a
 *     short batch is padded);
 *   - a retrieval group is every pending lookup / count / range request up
 *     to group_keys keys, admitted as soon as a slot is free.
 * Requests are linearised in admission order: each sees exactly the updates
 * of the groups admitted before its own (result->order gives the group
 * sequence number of every request).  Device memory is admitted against
 * hbm_budget: the dictionary gets the largest level count whose levels,
 * cleanup scratch and batch scratch fit beside the slots' buffers; an update
 * group that would need a level beyond it triggers a cleanup (§III-F) first,
 * and is refused (LSM_ERR_BUDGET for its requests) if the live data still
 * fills every level.  Policy LSM_SERVE_FIXED is the comparison point:
 * requests wait until b ops are pending (or the trace has ended), then all
 * pending work runs to completion before anything else is admitted.
 */
typedef struct lsm_server_t lsm_server_t;

enum { LSM_REQ_INSERT = 0, LSM_REQ_DELETE = 1, LSM_REQ_LOOKUP = 2, LSM_REQ_COUNT = 3, LSM_REQ_RANGE = 4 };
enum { LSM_SERVE_CONTINUOUS = 0, LSM_SERVE_FIXED = 1 };

typedef struct {
  uint32_t b;           /* device batch size, 1 .. 2^20 */
  uint64_t hbm_budget;  /* bytes of device memory the server may hold */
  double flush_us;      /* longest wait of an update before its partial batch is admitted */
  uint32_t group_keys;  /* keys (lookup keys + count/range intervals) per retrieval group */
  uint32_t slots;       /* groups in flight (continuous policy), 1 .. 16 */
  uint32_t range_cap;   /* range results one retrieval group may produce */
  int policy;           /* LSM_SERVE_CONTINUOUS or LSM_SERVE_FIXED */
  int device;
} lsm_server_config;

typedef struct {
  uint64_t n;                /* requests */
  const uint8_t* kind;       /* LSM_REQ_* per request */
  const double* arrival_us;  /* non-decreasing, microseconds after the start of the run */
  const uint64_t* start;     /* request i uses pool entries [start[i], start[i] + size[i]) */
  const uint32_t* size;      /* 1 .. group_keys (and <= b for updates) */
} lsm_trace;

typedef struct {
  /* required, n entries each */
  double* done_us;           /* when the server saw the request's group complete */
  int32_t* status;           /* LSM_OK or LSM_ERR_BUDGET (refused update) */
  uint64_t* order;           /* admission sequence number of the request's group, or NULL */
  /* optional results (NULL: dropped once copied to the server's host buffers) */
  const uint64_t* res_off;   /* n: first per-key result slot of request i */
  uint32_t* val;             /* lookup value / count / range result count, per key */
  uint8_t* found;            /* lookup found flag, per key */
  uint64_t* range_start;     /* range: first result of each interval in rk/rv */
  uint32_t* rk;              /* range results, original keys ascending per interval */
  uint32_t* rv;
  uint64_t range_cap;        /* entries of rk/rv */
  /* filled by the run */
  uint64_t range_total;
  uint64_t update_batches, padded_ops, retrieval_groups, cleanups, refused;
  double wall_us;
  /* where the time went: host microseconds spent admitting update groups,
   * admitting retrieval groups, finishing range groups, completing groups,
   * in cleanups, sleeping; device milliseconds of update and retrieval
   * groups (from the stream reaching a group to its completion event) */
  double host_admit_update_us, host_admit_retrieval_us, host_range_us, host_complete_us, host_cleanup_us,
      host_sleep_us, gpu_update_ms, gpu_retrieval_ms;
  /* device milliseconds of the retrieval groups' phases: payload gathers and
   * sorts, lookups, counts, range counts with their scan, range emits */
  double gpu_prep_ms, gpu_lookup_ms, gpu_count_ms, gpu_range_ms, gpu_emit_ms;
} lsm_trace_result;

/* Creates the server and its dictionary.  Errors: LSM_ERR_ARG,
 * LSM_ERR_BUDGET (not even one level fits), LSM_ERR_OOM, LSM_ERR_CUDA. */
lsm_status lsm_server_create(lsm_server_t** out, const lsm_server_config* cfg);
void lsm_server_destroy(lsm_server_t* s);

/* Registers the payload pools (device arrays of n u32, kept by the caller
 * while the server runs): d_a = keys of updates and lookups and the lower
 * bounds of count/range intervals, d_b = insert values, d_c = upper bounds.
 * Every key of d_a must be < 2^31 - 1 (checked here once, so that update
 * batches need no per-batch check): else LSM_ERR_KEY_RANGE.  Waits for all
 * device work first, so the pools may be written on any stream. */
lsm_status lsm_server_set_pool(lsm_server_t* s, const uint32_t* d_a, const uint32_t* d_b, const uint32_t* d_c,
                               uint64_t n);

/* Inserts n pairs into the dictionary before a run (synchronous; waits for
 * all device work first, so the pairs may come from any stream). */
lsm_status lsm_server_preload(lsm_server_t* s, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n);

/* Replays the trace in real time (blocking until every request completed). */
lsm_status lsm_server_run(lsm_server_t* s, const lsm_trace* t, lsm_trace_result* r);

/* Dictionary counter and resident elements, level count chosen for the
 * budget, and the device bytes the budget accounts for. */
lsm_status lsm_server_stats(const lsm_server_t* s, uint64_t* r, uint64_t* resident, uint32_t* levels,
                            uint64_t* device_bytes);

/* The server's dictionary (owned by the server), for queries between runs. */
lsm_t* lsm_server_dict(lsm_server_t* s);

/*
 * Fault injection for tests (the paper has no counterpart).  Both calls exist
 * so that the error paths of the failure design can be exercised without a
 * real out-of-memory condition and without faulting or hanging a GPU.
 *
 * lsm_debug_fail_allocs - from now on, let `skip` device or pinned-host
 * allocations of the library succeed, then make the next `count` fail as if
 * the memory were exhausted (the call that needed them returns LSM_ERR_OOM
 * and, being all or nothing, leaves its handle as it was).  Nothing is
 * allocated for a failed request.  Process-wide, all devices; (0, 0) disarms.
 * Host-only: needs no device.
 */
lsm_status lsm_debug_fail_allocs(uint64_t skip, uint64_t count);

/*
 * lsm_debug_wait_flag - one device thread waits, with the same bounded spin
 * as every wait inside the library (look-back scans, bulk-copy barriers),
 * until the device word *d_flag is non-zero, giving up after limit_ns
 * nanoseconds of the GPU's global timer.  d_status is a device word the call
 * zeroes first; a wait that gives up sets bit 2 there (the library's timeout
 * bit).  Synchronises with `stream`.  Returns LSM_OK when the flag was seen,
 * LSM_ERR_TIMEOUT when the wait gave up (the context stays usable),
 * LSM_ERR_ARG for null pointers or limit_ns = 0 or above 10 s.
 */
lsm_status lsm_debug_wait_flag(const uint32_t* d_flag, uint32_t* d_status, uint64_t limit_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GPULSM_H */
