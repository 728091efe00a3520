// Internal interface between the host orchestrator (lsm_api.cu) and the
// kernel translation units.  Plain structs of device pointers and sizes.
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

namespace gpulsm {

// Launches `kernel` with programmatic stream serialization: its blocks may be
// scheduled while the previous kernel in the stream finishes; the kernel
// itself calls pdl_wait() before touching anything that kernel wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Raises a kernel's dynamic shared-memory limit, an attribute of the current
// device, once per device and thread-safely: `f` keeps one flag per device
// ordinal for that kernel.
constexpr int kMaxDevices = 64;
struct PerDeviceFlags {
  std::atomic<bool> done[kMaxDevices] = {};
  std::mutex mu;
};
template <typename K>
cudaError_t set_smem_attr_once(K kernel, size_t bytes, int dev, PerDeviceFlags& f) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (f.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(f.mu);
  if (f.done[dev].load(std::memory_order_relaxed)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e == cudaSuccess) f.done[dev].store(true, std::memory_order_release);
  return e;
}

// Allocation fault injection (lsm_debug_fail_allocs): every device or
// pinned-host allocation of the library asks the gate first, and gets
// cudaErrorMemoryAllocation instead of memory while a failure is armed.
cudaError_t alloc_gate();

// Number of kernels this library has launched (all handles); read through
// LSM_OPT_KERNEL_LAUNCHES.  Incremented by every launcher below.
void count_launches(uint64_t n);
uint64_t launches_so_far();

constexpr int kMaxLevels = 32;                 // levels a handle may allocate
constexpr int kMaxSources = kMaxLevels + 1;    // fold: the batch + every level
constexpr uint32_t kMaxUserKey = 0x7FFFFFFEu;  // 2^31 - 2
constexpr uint32_t kPlaceboKv = 0xFFFFFFFEu;   // key 2^31 - 1 as a tombstone
constexpr uint32_t kSlack = 32;                // elements readable past every buffer end
constexpr uint32_t kLevelAlign = 32;           // level starts: multiples of 32 elements

// Sticky device error bits (a device word, copied to the host on demand).
constexpr uint32_t kErrBadKey = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrAlign = 4u;

// Spin-wait bound for decoupled look-back and mbarrier waits, in
// nanoseconds of globaltimer: a wait that exceeds it sets kErrTimeout and
// gives up instead of hanging the GPU.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// ------------------------------------------------------------------ sort ---
enum SortInput : int {
  kSortPairs = 0,     // (keys[i], vals[i]) as given
  kSortInsert = 1,    // batch of inserts: encode, reverse, pad
  kSortDelete = 2,    // batch of deletes: tombstones, value 0
  kSortUpdate = 3,    // mixed batch, per-op delete flag
  kSortQueries = 4    // (keys[i], i): sort query keys with their positions
};

// Tuning of the batch sort (compile-time): items per thread (tile =
// 256 * LSM_SORT_IPT elements), minimum resident CTAs per SM requested from
// the compiler, and the number of predecessor tiles read per look-back step.
#ifndef LSM_SORT_IPT
#define LSM_SORT_IPT 16
#endif
#ifndef LSM_SORT_MINB
#define LSM_SORT_MINB 1
#endif
#ifndef LSM_SORT_LBW
#define LSM_SORT_LBW 8
#endif
constexpr int kSortPasses = 4;
constexpr int kSortTile = 256 * LSM_SORT_IPT;  // elements per CTA tile of a pass

struct SortArgs {
  int mode;
  const uint32_t* in_keys;
  const uint32_t* in_vals;
  const uint8_t* in_del;
  uint64_t n_in;        // ops available in the input (batch modes)
  uint32_t n;           // elements to sort (b for a batch)
  uint32_t* out_keys;   // destination; also used as ping-pong space
  uint32_t* out_vals;
  uint32_t* tmp_keys;   // n elements of scratch
  uint32_t* tmp_vals;
  uint32_t* fence;      // prefix index of the sorted output to write, or null
  int fshift;
  // Deferred key check (bucket path only): when set, a batch holding a key
  // above the user range is written as n placebo tombstones instead of being
  // sorted, and kErrBadKey is ORed into *defer_err; nothing waits on the host.
  uint32_t* defer_err;
};

struct SortWorkspace {
  uint32_t* ctl;        // two halves of kSortCtlWords: [hist 4*256][tile counters 4][pad]
  int flip;             // the half the next sort uses; it is all zero on entry
  uint64_t* lookback;   // kSortPasses * max_tiles * 256 words
  uint32_t max_tiles;
  uint32_t epoch;       // bumped per sort; 0 never used
  uint32_t* sticky;     // persistent device error word (wait timeouts)
  uint32_t* tilecnt;    // msd_ws_words(n) words for every sort of n <= kMsdMaxN it serves, or null
};
// The bucket sort (n <= kMsdMaxN): the run table (per bucket and tile, the
// start and length of the bucket's run in the tile), then the spill area of
// buckets too large for shared memory (n keys, then n values).
constexpr uint32_t kMsdMaxN = 1u << 20;
constexpr uint32_t kMsdTile = 4096;
constexpr uint32_t kMsdMaxTiles = kMsdMaxN / kMsdTile;
constexpr uint32_t kMsdRunWords = 2 * kMsdMaxTiles * 256;
// Workspace words for sorts of at most max_n <= kMsdMaxN elements (the spill
// area holds a sort's n keys, then its n values).
constexpr uint64_t msd_ws_words(uint64_t max_n) { return kMsdRunWords + 2 * max_n; }
constexpr uint64_t kMsdWsWords = msd_ws_words(kMsdMaxN);
constexpr int kSortCtlWords = kSortPasses * 256 + kSortPasses + 4;
constexpr int kSortCtlStatus = kSortPasses * 256 + kSortPasses;

// Enqueues the whole sort.  If `status` is given (a device-visible word,
// typically mapped pinned host memory), the first kernel stores kErrBadKey
// there when a key is out of range, and `ev` is recorded right after that
// kernel, so the host can learn about bad keys before the sort ends.
cudaError_t sort_launch(const SortArgs& a, SortWorkspace& ws, cudaStream_t st,
                        uint32_t* status, cudaEvent_t ev);

// Device key check alone over n keys (multi-batch calls check all first).
cudaError_t check_keys_launch(const uint32_t* keys, uint64_t n, uint32_t* status,
                              cudaStream_t st);

// ------------------------------------------------------------------ fold ---
constexpr int kFoldTile = 2048;  // output elements per merge CTA

// Prefix index ("fence") of a sorted run: with bin(kv) = kv >> fshift,
// fence[P] = number of elements whose bin is < P, for P = 0 .. 2^(32-fshift):
// the start of the run of key variables in [P << fshift, (P + 1) << fshift).
// One table per level and one for the sorted batch, written whenever the run
// is written.  fshift is chosen per run so that a bin holds about 2^e
// elements (e = 3: a 32-byte sector of keys), with between 2^lo and 2^24
// bins.  A table at shift s also answers at any coarser shift s' >= s: entry
// P' << (s' - s).
__host__ __device__ inline uint32_t fence_bin(uint32_t kv, int fshift) { return kv >> fshift; }
__host__ __device__ inline uint32_t fence_bins(int fshift) { return 1u << (32 - fshift); }
inline int fence_shift_for(uint64_t n, int e = 3, int lo = 16) {
  int lg = 0;
  while ((2ull << lg) <= n) ++lg;      // floor(log2 n)
  int fb = lg - e;
  fb = fb < lo ? lo : (fb > 24 ? 24 : fb);
  return 32 - fb;
}
inline uint64_t fence_words(int fshift) { return uint64_t(fence_bins(fshift)) + 4; }

struct FoldSources {
  const uint32_t* keys[kMaxSources];
  const uint32_t* vals[kMaxSources];
  const uint32_t* fence[kMaxSources];
  uint32_t n[kMaxSources];
  int fshift[kMaxSources];
  int count;  // rank order: newest first
};

struct FoldArgs {
  FoldSources src;
  uint64_t total;
  uint32_t* out_keys;
  uint32_t* out_vals;
  uint32_t* part;        // (ntiles + 1) * count co-ranks
  uint32_t* out_fence;   // prefix index of the output (plain fold), or null
  int out_fshift;
  uint32_t* status;
  // cleanup only: keep the first element of every key if regular, compacted
  bool cleanup;
  uint64_t* lookback;    // ntiles words, zeroed by the launcher
  uint32_t* tile_ctr;    // zeroed by the launcher
  uint64_t* out_count;   // number of kept elements
};

inline uint64_t fold_tiles(uint64_t total) { return (total + kFoldTile - 1) / kFoldTile; }

// fold_launch = fold_partition_launch + fold_merge_launch.
cudaError_t fold_launch(const FoldArgs& a, cudaStream_t st);
cudaError_t fold_partition_launch(const FoldArgs& a, cudaStream_t st);
cudaError_t fold_merge_launch(const FoldArgs& a, cudaStream_t st);

struct DistributeArgs {
  const uint32_t* src_keys;  // compacted live pairs
  const uint32_t* src_vals;
  uint64_t n_live;
  uint32_t* keys;            // level array
  uint32_t* vals;
  int nlevels;
  uint64_t level_off[kMaxLevels];    // destination offset of each filled level
  uint64_t level_start[kMaxLevels];  // first compacted index it receives
  uint64_t level_size[kMaxLevels];
  uint64_t total;                    // r' * b
};
cudaError_t distribute_launch(const DistributeArgs& a, cudaStream_t st);

// ------------------------------------------------------ many dictionaries ---
// The batched form: n independent dictionaries, each with its own batch size
// b_i and levels b_i * 2^l, advanced together.  A round gives every instance
// at most one batch; all per-round decisions (which level each fold fills,
// how many tiles it has) are taken on the device from the instances' counters
// r_i, so one captured sequence of launches serves every round.
constexpr int kMultiMaxLevels = 16;            // levels per instance
constexpr int kMultiPartStride = kMultiMaxLevels + 1;  // co-rank words per tile boundary
constexpr uint32_t kMultiMaxB = 1u << 20;      // largest per-instance batch
constexpr uint32_t kMultiSortTile = 4096;      // elements per sort tile (count/scatter CTA)

// Per-instance error bits of a round (also ORed into the device status word).
constexpr uint32_t kErrArg = 8u;     // more ops than the batch size
constexpr uint32_t kErrFull = 16u;   // the fold would need a level beyond the capacity

struct MultiInst {           // fixed at creation
  uint64_t in_off;           // first op of its batch in the caller's input arrays (sum of earlier b)
  uint64_t boff;             // its sorted batch / sort scratch start (a multiple of kLevelAlign)
  uint32_t b;                // batch size
  uint32_t levels;           // allocated levels: a batch is refused once ffz(r) >= levels
  uint32_t msd_bits;         // d: the batch sort's buckets are the top d bits of the key variable
  uint32_t tile;             // merge tile: 1024 or 2048 output elements
  uint32_t stile0;           // first global sort tile
  uint32_t bucket0;          // first global bucket
  int32_t fshift0;           // prefix-index shift of the sorted batch and level 0
  uint32_t pad_;
  uint64_t batch_fence;      // fence arena offset of the sorted batch's prefix index
  uint64_t lvl_off[kMultiMaxLevels];    // level arena offset of level l
  uint64_t lvl_fence[kMultiMaxLevels];  // fence arena offset of level l's prefix index
  int32_t lvl_fshift[kMultiMaxLevels];
};

struct MultiArena {
  const MultiInst* inst;     // n descriptors
  uint32_t n;
  uint32_t* keys;            // level arena
  uint32_t* vals;
  uint32_t* bkeys;           // sorted batches (at boff)
  uint32_t* bvals;
  uint32_t* tkeys;           // bucket scatter scratch (at boff)
  uint32_t* tvals;
  uint32_t* fence;           // fence arena
  const uint64_t* stile_prefix;   // n + 1: sort tiles before instance i
  const uint64_t* bucket_prefix;  // n + 1: buckets before instance i
  uint64_t total_stiles, total_buckets;
  uint32_t* tilecnt;         // per sort tile 256 bucket counts, then 256 output offsets
  uint32_t* bstart;          // per global bucket: start in the instance's batch
  uint32_t* bcnt;            // per global bucket: element count
  // device state
  uint32_t* r;               // batches applied per instance
  int32_t* k;                // this round's fold target level, -1 when the instance has no batch
  uint32_t* badkey;          // per instance: a key out of range this round (cleared by the prep kernel)
  uint32_t* flags;           // per instance: error bits of the last round
  uint64_t* tile_prefix;     // n + 1: merge tiles before instance i this round
  uint64_t* part_prefix;     // n + 1: partition boundaries before instance i
  uint32_t* part;            // co-ranks, kMultiPartStride words per boundary
  uint32_t* work_ctr;        // head of the persistent merge's work queue
  uint32_t* status;          // sticky device status word
};

// One round's input: instance i's ops are keys/vals/del[in_off_i ..
// in_off_i + counts[i]); counts null means b_i ops for every instance.
struct MultiBatch {
  const uint32_t* keys;
  const uint32_t* vals;      // null: values 0 (pure deletes need none)
  const uint8_t* del;        // null: every op an insert
  const uint32_t* counts;
};

// Enqueues one round of updates for every instance: bucket counts, the
// round's plan (prep), offsets, scatter, bucket sort (into level 0 when
// k_i = 0, else the sorted-batch buffer), co-rank partition and the
// persistent merge.  Launch shapes depend only on the arena, never on the
// device state, so the sequence can be captured once and replayed.
cudaError_t multi_update_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st);

// Sets the kernels' launch attributes once (before any capture).
cudaError_t multi_prepare_kernels();
cudaError_t multi_sort_prepare();

// The parts of multi_update_launch (exposed for the launch list and tests).
cudaError_t multi_sort_count_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st);
cudaError_t multi_prep_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st);
cudaError_t multi_sort_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st);
cudaError_t multi_fold_launch(const MultiArena& ar, cudaStream_t st);

// Lookups: query g belongs to the instance i with qoff[i] <= g < qoff[i + 1]
// (qoff has n + 1 entries, qoff[n] = nq).
cudaError_t multi_lookup_launch(const MultiArena& ar, const uint32_t* q, const uint64_t* qoff, uint64_t nq,
                                uint32_t* val, uint8_t* found, cudaStream_t st);

// --------------------------------------------------------------- serving ---
// Ordered batch: (sk, sv) = the batch's keys sorted stably with their input
// positions; op p of the output is a copy of the last op (input order) on
// key(p).  vals / del may be null (0 / insert).
cudaError_t resolve_last_launch(const uint32_t* sk, const uint32_t* sv, uint32_t n, const uint32_t* keys,
                                const uint32_t* vals, const uint8_t* del, uint32_t* out_k, uint32_t* out_v,
                                uint8_t* out_d, cudaStream_t st);

// Gathers windows of device-resident payload arrays: request j (of nreq,
// dst_off ascending) fills dst[dst_off[j] + t] = src[start[j] + t] for the
// positions up to the next request's offset (or `total`); up to two arrays
// at once (src_b / dst_b may be null).
cudaError_t gather_windows_launch(const uint32_t* src_a, const uint32_t* src_b, const uint64_t* start,
                                  const uint64_t* dst_off, uint32_t nreq, uint64_t total, uint32_t* dst_a,
                                  uint32_t* dst_b, cudaStream_t st);

// Gathers whole update requests into a batch the same way: keys from pool_k,
// values from pool_v (0 for a delete request), the request's delete flag
// per op.
cudaError_t gather_update_launch(const uint32_t* pool_k, const uint32_t* pool_v, const uint64_t* start,
                                 const uint64_t* dst_off, const uint8_t* is_del, uint32_t nreq, uint64_t total,
                                 uint32_t* out_k, uint32_t* out_v, uint8_t* out_d, cudaStream_t st);

// ----------------------------------------------------------------- query ---
struct LevelSet {
  const uint32_t* keys[kMaxLevels];
  const uint32_t* vals[kMaxLevels];
  const uint32_t* fence[kMaxLevels];
  uint32_t n[kMaxLevels];
  int fshift[kMaxLevels];
  int count;  // full levels, newest (smallest) first
};

// Prefix index of a sorted run of n key variables (fence_words(fshift) words).
cudaError_t build_fence_launch(const uint32_t* keys, uint32_t n, uint32_t* fence, int fshift, cudaStream_t st);

cudaError_t lookup_launch(const LevelSet& ls, const uint32_t* q, uint64_t nq,
                          uint32_t* val, uint8_t* found, cudaStream_t st);

// Lookup of queries already sorted by key (kSortQueries output): results go
// to positions idx[i] of the output arrays.
cudaError_t lookup_sorted_launch(const LevelSet& ls, const uint32_t* sq, const uint32_t* idx,
                                 uint64_t nq, uint32_t* val, uint8_t* found, cudaStream_t st);

// Count per query; when `bounds` is not null also stores, per query and
// level, the window [lo, hi) (2 * count words per query).  With `perm`, the
// queries come sorted by k1 (k1 = sorted lower bounds, perm = their
// positions; k2 stays in query order) and results go to position perm[i].
// With `wide` (nq + 1 words of scratch), queries with many elements in their
// windows are counted by a warp each (a second kernel); the list of them is
// left in `wide` for range_emit_launch.
cudaError_t count_launch(const LevelSet& ls, const uint32_t* k1, const uint32_t* k2,
                         uint64_t nq, uint32_t* count, uint32_t* bounds, cudaStream_t st,
                         const uint32_t* perm = nullptr, uint32_t* wide = nullptr);

// Successor (smallest live key >= q) or predecessor (largest live key <= q)
// of every query: key, value and found flag (0 / 0 / 0 when none).
cudaError_t neighbor_launch(const LevelSet& ls, const uint32_t* q, uint64_t nq, bool successor, uint32_t* key,
                            uint32_t* val, uint8_t* found, cudaStream_t st);

// Exclusive scan of n u32 into n + 1 u64 (out[n] = total).
cudaError_t scan_launch(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* lookback,
                        uint32_t* tile_ctr, uint32_t* status, cudaStream_t st);
inline uint64_t scan_tiles(uint64_t n) { return (n + 2047) / 2048; }

// Range output from the windows of count_launch; with `perm`, thread i
// serves query perm[i] (neighbouring threads, neighbouring windows).
// With `wide` (the list count_launch left), the wide queries are emitted by
// a warp each, from their bounds k1 / k2.
cudaError_t range_emit_launch(const LevelSet& ls, uint64_t nq, const uint32_t* bounds,
                              const uint64_t* offsets, uint32_t* keys, uint32_t* vals,
                              cudaStream_t st, const uint32_t* perm = nullptr, const uint32_t* k1 = nullptr,
                              const uint32_t* k2 = nullptr, const uint32_t* wide = nullptr);

}  // namespace gpulsm
