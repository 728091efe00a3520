// Host orchestrator and C ABI of the GPU LSM (include/gpulsm.h).
//
// The host owns the binary counter r (§III-B): level i is full iff bit i of r
// is set, and an update batch lands in level ffz(r).  The host waits only
// where the interface says so (the key check of an update, the totals of
// range and cleanup).
//
// Two streams.  A batch is sorted on the caller's stream into one of three
// sorted-batch buffers; its fold into level k runs on the handle's internal
// stream, so the next batch's sort overlaps it.  A batch that lands in level
// 0 (k = 0) is not copied: its buffer becomes level 0 until the next fold
// consumes it.  Every call that reads or rewrites the levels first makes the
// caller's stream wait for the internal one; a buffer is reused only after
// the fold that read it (an event per buffer).
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <cstring>
#include <new>
#include <vector>

#include "gpulsm.h"
#include "lsm_internal.h"

using namespace gpulsm;

namespace gpulsm {
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// lsm_debug_fail_allocs: allocations still allowed, then failures to give.
static std::mutex g_fail_mu;
static uint64_t g_fail_skip = 0, g_fail_count = 0;
static std::atomic<bool> g_fail_armed{false};
cudaError_t alloc_gate() {
  if (!g_fail_armed.load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(g_fail_mu);
  if (g_fail_skip) {
    --g_fail_skip;
    return cudaSuccess;
  }
  if (g_fail_count) {
    if (--g_fail_count == 0) g_fail_armed.store(false, std::memory_order_release);
    return cudaErrorMemoryAllocation;
  }
  return cudaSuccess;
}
void debug_fail_allocs(uint64_t skip, uint64_t count) {
  std::lock_guard<std::mutex> lock(g_fail_mu);
  g_fail_skip = skip;
  g_fail_count = count;
  g_fail_armed.store(count != 0, std::memory_order_release);
}
}  // namespace gpulsm

struct lsm_t {
  int device = 0;
  uint32_t b = 0;
  uint32_t L = 0;
  uint64_t r = 0;
  uint64_t level_off[kMaxLevels + 1] = {};
  uint64_t capacity = 0;
  uint32_t* d_keys = nullptr;
  uint32_t* d_vals = nullptr;
  uint32_t* d_bk = nullptr;  // kBatchBufs sorted-batch buffers of bpad elements
  uint32_t* d_bv = nullptr;
  uint64_t bpad = 0;
  int l0_buf = -1;           // the buffer holding level 0, or -1 (level 0 in the level array)
  int last_buf = 0;          // buffer of the latest batch
  cudaStream_t side = nullptr;           // folds
  cudaEvent_t ev_sorted = nullptr;       // caller's stream, after a batch's sort
  cudaEvent_t ev_side = nullptr;         // internal stream, after its latest work
  cudaEvent_t ev_free[kBatchBufs] = {};  // internal stream, after the fold that read buffer j
  bool side_pending = false;
  uint32_t* d_tk = nullptr;  // sort ping-pong (b + slack)
  uint32_t* d_tv = nullptr;
  SortWorkspace sws{};
  uint32_t* d_part = nullptr;
  uint64_t part_words = 0;
  uint32_t* d_fence = nullptr;  // prefix index per level (L tables) + the sorted batch's
  uint64_t fence_off[kMaxLevels + kBatchBufs + 1] = {};  // L levels, then the batch buffers
  int fshift[kMaxLevels + kBatchBufs + 1] = {};  // per level; [L ..] = the batch buffers
  uint32_t* d_misc = nullptr;  // [0] sticky errors [1] key check [2] tile ctr [3] tile ctr
  uint64_t* d_u64 = nullptr;   // [0] cleanup count
  uint32_t* h_status = nullptr;  // mapped pinned word: key check of the current batch
  uint32_t* d_status_map = nullptr;
  uint64_t* h_u64 = nullptr;
  cudaEvent_t ev = nullptr;
  // cleanup scratch (allocated on first cleanup)
  uint32_t* d_ck = nullptr;
  uint32_t* d_cv = nullptr;
  uint64_t* d_clb = nullptr;
  uint64_t clean_cap = 0;
  // query scratch (grown on demand)
  unsigned char* d_q = nullptr;
  size_t q_bytes = 0;
  // sorted-lookup workspace (grown on demand)
  SortWorkspace qsws{};
  uint32_t* d_qctl = nullptr;
  int lookup_mode = 0;
  bool key_check_deferred = false;  // LSM_OPT_KEY_CHECK
  // kernel profiler
  uint32_t prof = 0;  // profiled groups: bit g for lsm_prof_group g
  struct ProfRec {
    int group;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  lsm_profile_entry prof_acc[LSM_PROF_COUNT_] = {};
};

namespace {

enum { kMiscSticky = 0, kMiscCheck = 1, kMiscCtrA = 2, kMiscCtrB = 3, kMiscWords = 8 };

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

lsm_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LSM_OK;
  cudaGetLastError();  // clear non-sticky errors
  return e == cudaErrorMemoryAllocation ? LSM_ERR_OOM : LSM_ERR_CUDA;
}

#define LSM_TRY(expr)                              \
  do {                                             \
    lsm_status _s = cuda_status(expr);             \
    if (_s != LSM_OK) return _s;                   \
  } while (0)

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

int ffz(uint64_t r) {
  int i = 0;
  while ((r >> i) & 1u) ++i;
  return i;
}

template <typename T>
cudaError_t dalloc(T** p, uint64_t count) {
  const cudaError_t g = alloc_gate();
  if (g != cudaSuccess) return g;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

void free_all(lsm_t* h) {
  void* dptrs[] = {h->d_keys, h->d_vals, h->d_bk, h->d_bv, h->d_tk, h->d_tv, h->sws.ctl, h->sws.lookback,
                   h->sws.tilecnt, h->d_part, h->d_fence, h->d_misc, h->d_u64, h->d_ck, h->d_cv, h->d_clb,
                   h->d_q, h->qsws.lookback, h->qsws.tilecnt, h->d_qctl};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_sorted) cudaEventDestroy(h->ev_sorted);
  if (h->ev_side) cudaEventDestroy(h->ev_side);
  for (cudaEvent_t e : h->ev_free)
    if (e) cudaEventDestroy(e);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_u64) cudaFreeHost(h->h_u64);
  if (h->ev) cudaEventDestroy(h->ev);
  for (auto& p : h->prof_pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : h->prof_pool) cudaEventDestroy(e);
}

// Brackets a kernel group with timing events while the profiler is on.
struct ProfScope {
  lsm_t* h;
  int group;
  double bytes;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  static cudaEvent_t get(lsm_t* h) {
    if (!h->prof_pool.empty()) {
      cudaEvent_t e = h->prof_pool.back();
      h->prof_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  ProfScope(lsm_t* h_, int g, double by, cudaStream_t s) : h(h_), group(g), bytes(by), st(s) {
    if (((h->prof >> group) & 1u) && (a = get(h))) cudaEventRecord(a, st);
  }
  ~ProfScope() {
    if (!((h->prof >> group) & 1u) || !a) return;
    cudaEvent_t b = get(h);
    if (!b) return;
    cudaEventRecord(b, st);
    h->prof_pending.push_back({group, a, b, bytes});
  }
};

uint32_t* buf_keys(const lsm_t* h, int j) { return h->d_bk + uint64_t(j) * h->bpad; }
uint32_t* buf_vals(const lsm_t* h, int j) { return h->d_bv + uint64_t(j) * h->bpad; }
uint32_t* buf_fence(const lsm_t* h, int j) { return h->d_fence + h->fence_off[h->L + j]; }
// Level i's storage; level 0 may be a sorted-batch buffer.
uint32_t* level_keys(const lsm_t* h, int i) {
  return (i == 0 && h->l0_buf >= 0) ? buf_keys(h, h->l0_buf) : h->d_keys + h->level_off[i];
}
uint32_t* level_vals(const lsm_t* h, int i) {
  return (i == 0 && h->l0_buf >= 0) ? buf_vals(h, h->l0_buf) : h->d_vals + h->level_off[i];
}
uint32_t* level_fence(const lsm_t* h, int i) {
  return (i == 0 && h->l0_buf >= 0) ? buf_fence(h, h->l0_buf) : h->d_fence + h->fence_off[i];
}

// Orders `st` after the folds in flight on the internal stream.
cudaError_t join_side(const lsm_t* h, cudaStream_t st) {
  if (!h->side_pending) return cudaSuccess;
  return cudaStreamWaitEvent(st, h->ev_side, 0);
}

LevelSet full_levels(lsm_t* h) {
  LevelSet ls{};
  for (uint32_t i = 0; i < h->L; ++i) {
    if (!((h->r >> i) & 1u)) continue;
    ls.keys[ls.count] = level_keys(h, i);
    ls.vals[ls.count] = level_vals(h, i);
    ls.fence[ls.count] = level_fence(h, i);
    ls.fshift[ls.count] = h->fshift[i];
    ls.n[ls.count] = uint32_t(uint64_t(h->b) << i);
    ++ls.count;
  }
  return ls;
}

cudaError_t ensure_q(lsm_t* h, size_t bytes) {
  if (bytes <= h->q_bytes) return cudaSuccess;
  if (h->d_q) {
    cudaError_t e = cudaFree(h->d_q);
    h->d_q = nullptr;
    h->q_bytes = 0;
    if (e != cudaSuccess) return e;
  }
  const size_t want = round_up(bytes + bytes / 4, 1 << 20);
  cudaError_t e = alloc_gate();
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&h->d_q), want);
  if (e == cudaSuccess) h->q_bytes = want;
  return e;
}

// Stable sort of (keys[i], i) for i < n into the query scratch (grown on
// demand, `extra` more words kept after the four sort arrays); returns the
// sorted keys and positions.
cudaError_t sort_positions(lsm_t* h, const uint32_t* keys, uint64_t n, uint64_t extra, cudaStream_t st,
                           uint32_t** sk, uint32_t** sv) {
  const uint64_t tiles = (n + kSortTile - 1) / kSortTile;
  const uint64_t npad = round_up(n, kLevelAlign) + kSlack;
  cudaError_t e;
  if ((e = ensure_q(h, (4 * npad + extra) * sizeof(uint32_t))) != cudaSuccess) return e;
  if (!h->qsws.lookback || h->qsws.max_tiles < tiles) {
    if (h->qsws.lookback) cudaFree(h->qsws.lookback);
    h->qsws.lookback = nullptr;
    if ((e = dalloc(&h->qsws.lookback, uint64_t(kSortPasses) * tiles * 256)) != cudaSuccess) return e;
    if ((e = cudaMemset(h->qsws.lookback, 0, sizeof(uint64_t) * kSortPasses * tiles * 256)) != cudaSuccess)
      return e;
    h->qsws.max_tiles = uint32_t(tiles);
    h->qsws.epoch = 0;
  }
  if (!h->d_qctl) {
    if ((e = dalloc(&h->d_qctl, 2 * kSortCtlWords)) != cudaSuccess) return e;
    if ((e = cudaMemset(h->d_qctl, 0, sizeof(uint32_t) * 2 * kSortCtlWords)) != cudaSuccess) return e;
    h->qsws.flip = 0;
  }
  if (!h->qsws.tilecnt && (e = dalloc(&h->qsws.tilecnt, kMsdWsWords)) != cudaSuccess) return e;
  h->qsws.ctl = h->d_qctl;
  h->qsws.sticky = h->d_misc + kMiscSticky;
  uint32_t* base = reinterpret_cast<uint32_t*>(h->d_q);
  SortArgs a{};
  a.mode = kSortQueries;
  a.in_keys = keys;
  a.n_in = n;
  a.n = uint32_t(n);
  a.out_keys = base;
  a.out_vals = base + npad;
  a.tmp_keys = base + 2 * npad;
  a.tmp_vals = base + 3 * npad;
  *sk = a.out_keys;
  *sv = a.out_vals;
  return sort_launch(a, h->qsws, st, nullptr, nullptr);
}

// One batch of n_in <= b ops into level ffz(r).  With `checked`, the keys
// are checked on the device: by default the host waits for that check and
// leaves the dictionary alone if it failed (the batch only wrote a free
// sorted-batch buffer); with the deferred check (LSM_OPT_KEY_CHECK = 1, batch
// sizes of the bucket sort) nothing waits, and a failed batch is applied as
// placebos and recorded in the sticky error word.
lsm_status apply_batch(lsm_t* h, int mode, const uint32_t* keys, const uint32_t* vals, const uint8_t* del,
                       uint64_t n_in, cudaStream_t st, bool checked) {
  const bool deferred = checked && h->key_check_deferred && h->b <= kMsdMaxN;
  if (deferred) checked = false;
  const int k = ffz(h->r);
  if (k >= int(h->L)) return LSM_ERR_FULL;
  // next buffer in rotation that does not hold level 0; wait for the fold
  // that last read it
  int j = (h->last_buf + 1) % kBatchBufs;
  if (j == h->l0_buf) j = (j + 1) % kBatchBufs;
  LSM_TRY(cudaStreamWaitEvent(st, h->ev_free[j], 0));
  SortArgs a{};
  a.mode = mode;
  a.in_keys = keys;
  a.in_vals = vals;
  a.in_del = del;
  a.n_in = n_in;
  a.n = h->b;
  a.out_keys = buf_keys(h, j);
  a.out_vals = buf_vals(h, j);
  a.tmp_keys = h->d_tk;
  a.tmp_vals = h->d_tv;
  a.fence = buf_fence(h, j);
  a.fshift = h->fshift[0];
  a.defer_err = deferred ? h->d_misc + kMiscSticky : nullptr;
  {
    ProfScope ps(h, LSM_PROF_SORT, 16.0 * h->b, st);
    if (checked) *reinterpret_cast<volatile uint32_t*>(h->h_status) = 0u;
    LSM_TRY(sort_launch(a, h->sws, st, checked ? h->d_status_map : nullptr, h->ev));
  }
  if (checked) {
    LSM_TRY(cudaEventSynchronize(h->ev));
    if (*reinterpret_cast<volatile uint32_t*>(h->h_status) & kErrBadKey) return LSM_ERR_KEY_RANGE;
  }
  h->last_buf = j;
  if (k == 0) {
    h->l0_buf = j;  // the sorted batch is level 0
    h->r += 1;
    return LSM_OK;
  }
  LSM_TRY(cudaEventRecord(h->ev_sorted, st));
  cudaStream_t side = h->side;
  LSM_TRY(cudaStreamWaitEvent(side, h->ev_sorted, 0));
  FoldArgs f{};
  f.src.count = k + 1;
  f.src.keys[0] = buf_keys(h, j);
  f.src.vals[0] = buf_vals(h, j);
  f.src.fence[0] = buf_fence(h, j);
  f.src.fshift[0] = h->fshift[0];
  f.src.n[0] = h->b;
  for (int i = 0; i < k; ++i) {
    f.src.keys[i + 1] = level_keys(h, i);
    f.src.vals[i + 1] = level_vals(h, i);
    f.src.fence[i + 1] = level_fence(h, i);
    f.src.fshift[i + 1] = h->fshift[i];
    f.src.n[i + 1] = uint32_t(uint64_t(h->b) << i);
  }
  f.total = uint64_t(h->b) << k;
  f.out_keys = h->d_keys + h->level_off[k];
  f.out_vals = h->d_vals + h->level_off[k];
  f.out_fence = h->d_fence + h->fence_off[k];
  f.out_fshift = h->fshift[k];
  f.part = h->d_part;
  f.status = h->d_misc + kMiscSticky;
  f.cleanup = false;
  {
    ProfScope ps(h, LSM_PROF_PARTITION, 0.0, side);
    LSM_TRY(fold_partition_launch(f, side));
  }
  {
    ProfScope ps(h, LSM_PROF_MERGE, 16.0 * double(f.total), side);
    LSM_TRY(fold_merge_launch(f, side));
  }
  LSM_TRY(cudaEventRecord(h->ev_free[j], side));
  if (h->l0_buf >= 0) {
    LSM_TRY(cudaEventRecord(h->ev_free[h->l0_buf], side));
    h->l0_buf = -1;  // level 0 was consumed
  }
  LSM_TRY(cudaEventRecord(h->ev_side, side));
  h->side_pending = true;
  h->r += 1;
  return LSM_OK;
}

// insert / delete: ceil(n / b) batches.  One batch: the check is fused into
// the sort.  Several: all keys are checked first so that the call stays all
// or nothing.
lsm_status apply_call(lsm_t* h, int mode, const uint32_t* keys, const uint32_t* vals, uint64_t n,
                      cudaStream_t st) {
  if (!h || (n && !keys) || (n && mode == kSortInsert && !vals)) return LSM_ERR_ARG;
  if (n == 0) return LSM_OK;
  DeviceGuard g(h->device);
  const uint64_t nb = (n + h->b - 1) / h->b;
  const uint64_t limit = (h->L >= 64) ? ~0ull : ((1ull << h->L) - 1);
  if (h->r + nb > limit) return LSM_ERR_FULL;
  if (nb == 1) return apply_batch(h, mode, keys, vals, nullptr, n, st, true);
  if (h->key_check_deferred && h->b <= kMsdMaxN) {
    // deferred check: every batch checks its own keys on the device
    for (uint64_t c = 0; c < nb; ++c) {
      const uint64_t off = c * h->b;
      const uint64_t m = (n - off) < h->b ? (n - off) : h->b;
      lsm_status s = apply_batch(h, mode, keys + off, vals ? vals + off : nullptr, nullptr, m, st, true);
      if (s != LSM_OK) return s;
    }
    return LSM_OK;
  }
  LSM_TRY(cudaMemsetAsync(h->d_misc + kMiscCheck, 0, sizeof(uint32_t), st));
  LSM_TRY(check_keys_launch(keys, n, h->d_misc + kMiscCheck, st));
  LSM_TRY(cudaMemcpyAsync(h->h_status, h->d_misc + kMiscCheck, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  LSM_TRY(cudaStreamSynchronize(st));
  if (*h->h_status & kErrBadKey) return LSM_ERR_KEY_RANGE;
  for (uint64_t c = 0; c < nb; ++c) {
    const uint64_t off = c * h->b;
    const uint64_t m = (n - off) < h->b ? (n - off) : h->b;
    lsm_status s = apply_batch(h, mode, keys + off, vals ? vals + off : nullptr, nullptr, m, st, false);
    if (s != LSM_OK) return s;
  }
  return LSM_OK;
}

}  // namespace

// ------------------------------------------------ hooks for the serving engine
namespace gpulsm {

LevelSet dict_levels(lsm_t* h) { return full_levels(h); }

cudaError_t dict_join(lsm_t* h, cudaStream_t st) { return join_side(h, st); }

lsm_status dict_update_ordered(lsm_t* h, const uint32_t* keys, const uint32_t* vals, const uint8_t* del,
                               uint64_t n, cudaStream_t st, bool checked) {
  if (n == 0) return LSM_OK;
  const uint64_t npad = round_up(n, kLevelAlign) + kSlack;
  uint32_t* sk = nullptr;
  uint32_t* sv = nullptr;
  LSM_TRY(sort_positions(h, keys, n, 3 * npad, st, &sk, &sv));
  uint32_t* rk = reinterpret_cast<uint32_t*>(h->d_q) + 4 * npad;
  uint32_t* rv = rk + npad;
  uint8_t* rd = reinterpret_cast<uint8_t*>(rv + npad);
  LSM_TRY(resolve_last_launch(sk, sv, uint32_t(n), keys, vals, del, rk, rv, rd, st));
  return apply_batch(h, kSortUpdate, rk, rv, rd, n, st, checked);
}

cudaError_t dict_record_applied(lsm_t* h, cudaEvent_t ev, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaEventRecord(h->ev_sorted, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(h->side, h->ev_sorted, 0)) != cudaSuccess) return e;
  return cudaEventRecord(ev, h->side);
}

uint64_t dict_r(const lsm_t* h) { return h->r; }
uint32_t dict_L(const lsm_t* h) { return h->L; }
uint32_t* dict_status_word(lsm_t* h) { return h->d_misc + kMiscSticky; }

}  // namespace gpulsm

extern "C" {

const char* lsm_status_str(lsm_status s) {
  switch (s) {
    case LSM_OK: return "LSM_OK";
    case LSM_ERR_ARG: return "LSM_ERR_ARG";
    case LSM_ERR_KEY_RANGE: return "LSM_ERR_KEY_RANGE";
    case LSM_ERR_FULL: return "LSM_ERR_FULL";
    case LSM_ERR_OOM: return "LSM_ERR_OOM";
    case LSM_ERR_BUDGET: return "LSM_ERR_BUDGET";
    case LSM_ERR_CAPACITY: return "LSM_ERR_CAPACITY";
    case LSM_ERR_CUDA: return "LSM_ERR_CUDA";
    case LSM_ERR_TIMEOUT: return "LSM_ERR_TIMEOUT";
  }
  return "LSM_ERR_UNKNOWN";
}

lsm_status lsm_create(lsm_t** out, uint32_t b, uint64_t max_elements, int device) {
  if (!out || b == 0 || b > (1u << 26)) return LSM_ERR_ARG;
  *out = nullptr;
  uint32_t L = 1;
  while (L < uint32_t(kMaxLevels) && (uint64_t(b) * ((1ull << L) - 1)) < max_elements) ++L;
  if (uint64_t(b) * ((1ull << L) - 1) < max_elements) return LSM_ERR_ARG;
  uint64_t off[kMaxLevels + 1] = {};
  for (uint32_t i = 0; i < L; ++i) off[i + 1] = off[i] + round_up(uint64_t(b) << i, kLevelAlign);
  if (off[L] > (1ull << 31)) return LSM_ERR_ARG;

  DeviceGuard g(device);
  lsm_t* h = new (std::nothrow) lsm_t();
  if (!h) return LSM_ERR_OOM;
  h->device = device;
  h->b = b;
  h->L = L;
  memcpy(h->level_off, off, sizeof(off));
  h->capacity = off[L];
  const uint64_t bpad = round_up(b, kLevelAlign) + kSlack;
  const uint32_t sort_tiles = (b + kSortTile - 1) / kSortTile;
  h->part_words = (fold_tiles(h->capacity) + 2) * (L + 1);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&h->d_keys, h->capacity + kSlack);
  if (e == cudaSuccess) e = dalloc(&h->d_vals, h->capacity + kSlack);
  h->bpad = bpad;
  if (e == cudaSuccess) e = dalloc(&h->d_bk, kBatchBufs * bpad);
  if (e == cudaSuccess) e = dalloc(&h->d_bv, kBatchBufs * bpad);
  if (e == cudaSuccess) e = dalloc(&h->d_tk, bpad);
  if (e == cudaSuccess) e = dalloc(&h->d_tv, bpad);
  if (e == cudaSuccess) e = dalloc(&h->sws.ctl, 2 * kSortCtlWords);
  if (e == cudaSuccess) e = cudaMemset(h->sws.ctl, 0, sizeof(uint32_t) * 2 * kSortCtlWords);
  if (e == cudaSuccess) e = dalloc(&h->sws.lookback, uint64_t(kSortPasses) * sort_tiles * 256);
  if (e == cudaSuccess && b <= kMsdMaxN) e = dalloc(&h->sws.tilecnt, msd_ws_words(b));
  if (e == cudaSuccess) e = dalloc(&h->d_part, h->part_words);
  for (uint32_t i = 0; i < L + kBatchBufs; ++i) {
    h->fshift[i] = fence_shift_for(i < L ? (uint64_t(b) << i) : uint64_t(b));
    h->fence_off[i + 1] = h->fence_off[i] + round_up(fence_words(h->fshift[i]), 64);
  }
  if (e == cudaSuccess) e = dalloc(&h->d_fence, h->fence_off[L + kBatchBufs]);
  if (e == cudaSuccess) e = dalloc(&h->d_misc, kMiscWords);
  if (e == cudaSuccess) e = dalloc(&h->d_u64, 8);
  if (e == cudaSuccess) e = alloc_gate();
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&h->h_status), 64, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->d_status_map), h->h_status, 0);
  if (e == cudaSuccess) e = alloc_gate();
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&h->h_u64), 64, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(h->d_keys, 0, sizeof(uint32_t) * (h->capacity + kSlack));
  if (e == cudaSuccess) e = cudaMemset(h->d_vals, 0, sizeof(uint32_t) * (h->capacity + kSlack));
  if (e == cudaSuccess) e = cudaMemset(h->d_bk, 0, sizeof(uint32_t) * kBatchBufs * bpad);
  if (e == cudaSuccess) e = cudaMemset(h->d_bv, 0, sizeof(uint32_t) * kBatchBufs * bpad);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_sorted, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_side, cudaEventDisableTiming);
  for (int j = 0; j < kBatchBufs; ++j)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[j], cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemset(h->sws.lookback, 0, sizeof(uint64_t) * kSortPasses * uint64_t(sort_tiles) * 256);
  if (e == cudaSuccess) e = cudaMemset(h->d_misc, 0, sizeof(uint32_t) * kMiscWords);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_status(e);
  }
  h->sws.max_tiles = sort_tiles;
  h->sws.epoch = 0;
  h->sws.sticky = h->d_misc + kMiscSticky;
  *out = h;
  return LSM_OK;
}

void lsm_destroy(lsm_t* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

lsm_status lsm_insert_batch(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n,
                            void* stream) {
  return apply_call(h, kSortInsert, d_keys, d_vals, n, static_cast<cudaStream_t>(stream));
}

lsm_status lsm_delete_batch(lsm_t* h, const uint32_t* d_keys, uint64_t n, void* stream) {
  return apply_call(h, kSortDelete, d_keys, nullptr, n, static_cast<cudaStream_t>(stream));
}

lsm_status lsm_update_batch(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                            const uint8_t* d_is_delete, uint64_t n, void* stream) {
  if (!h || (n && (!d_keys || !d_vals || !d_is_delete)) || n > h->b) return LSM_ERR_ARG;
  if (n == 0) return LSM_OK;
  DeviceGuard g(h->device);
  return apply_batch(h, kSortUpdate, d_keys, d_vals, d_is_delete, n, static_cast<cudaStream_t>(stream), true);
}

lsm_status lsm_update_batch_ordered(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                                    const uint8_t* d_is_delete, uint64_t n, void* stream) {
  if (!h || (n && !d_keys) || n > h->b) return LSM_ERR_ARG;
  if (n == 0) return LSM_OK;
  DeviceGuard g(h->device);
  // Every op takes the content of the last op on its key (input order), so
  // the batch rules of §III-A see one kind of op per key.
  return dict_update_ordered(h, d_keys, d_vals, d_is_delete, n, static_cast<cudaStream_t>(stream), true);
}

lsm_status lsm_lookup(lsm_t* h, const uint32_t* d_q, uint64_t nq, uint32_t* d_val, uint8_t* d_found,
                      void* stream) {
  if (!h || (nq && (!d_q || !d_val || !d_found))) return LSM_ERR_ARG;
  if (nq == 0) return LSM_OK;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  const LevelSet ls = full_levels(h);
  if (ls.count == 0) {
    LSM_TRY(cudaMemsetAsync(d_val, 0, sizeof(uint32_t) * nq, st));
    LSM_TRY(cudaMemsetAsync(d_found, 0, nq, st));
    return LSM_OK;
  }
  const bool sorted = h->lookup_mode == 2 && nq <= 0xFFFFFFFFull;
  ProfScope ps(h, LSM_PROF_LOOKUP, double(nq) * (9.0 + 32.0 * ls.count), st);
  if (!sorted) return cuda_status(lookup_launch(ls, d_q, nq, d_val, d_found, st));
  // Sorted mode: radix sort (key, position), then warp-cooperative search.
  uint32_t* sk = nullptr;
  uint32_t* sv = nullptr;
  LSM_TRY(sort_positions(h, d_q, nq, 0, st, &sk, &sv));
  return cuda_status(lookup_sorted_launch(ls, sk, sv, nq, d_val, d_found, st));
}

static lsm_status neighbor_call(lsm_t* h, const uint32_t* d_q, uint64_t nq, bool successor, uint32_t* d_key,
                                uint32_t* d_val, uint8_t* d_found, void* stream) {
  if (!h || (nq && (!d_q || !d_key || !d_val || !d_found))) return LSM_ERR_ARG;
  if (nq == 0) return LSM_OK;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  const LevelSet ls = full_levels(h);
  if (ls.count == 0) {
    LSM_TRY(cudaMemsetAsync(d_key, 0, sizeof(uint32_t) * nq, st));
    LSM_TRY(cudaMemsetAsync(d_val, 0, sizeof(uint32_t) * nq, st));
    LSM_TRY(cudaMemsetAsync(d_found, 0, nq, st));
    return LSM_OK;
  }
  return cuda_status(neighbor_launch(ls, d_q, nq, successor, d_key, d_val, d_found, st));
}

lsm_status lsm_successor(lsm_t* h, const uint32_t* d_q, uint64_t nq, uint32_t* d_key, uint32_t* d_val,
                         uint8_t* d_found, void* stream) {
  return neighbor_call(h, d_q, nq, true, d_key, d_val, d_found, stream);
}

lsm_status lsm_predecessor(lsm_t* h, const uint32_t* d_q, uint64_t nq, uint32_t* d_key, uint32_t* d_val,
                           uint8_t* d_found, void* stream) {
  return neighbor_call(h, d_q, nq, false, d_key, d_val, d_found, stream);
}

lsm_status lsm_count(lsm_t* h, const uint32_t* d_k1, const uint32_t* d_k2, uint64_t nq, uint32_t* d_count,
                     void* stream) {
  if (!h || (nq && (!d_k1 || !d_k2 || !d_count))) return LSM_ERR_ARG;
  if (nq == 0) return LSM_OK;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  const LevelSet ls = full_levels(h);
  if (ls.count == 0) return cuda_status(cudaMemsetAsync(d_count, 0, sizeof(uint32_t) * nq, st));
  // scratch: the list of wide queries (counted by a warp each)
  LSM_TRY(ensure_q(h, (nq + 1) * 4));
  uint32_t* wide = reinterpret_cast<uint32_t*>(h->d_q);
  ProfScope ps(h, LSM_PROF_COUNT, double(nq) * (12.0 + 64.0 * ls.count), st);
  return cuda_status(count_launch(ls, d_k1, d_k2, nq, d_count, nullptr, st, nullptr, wide));
}

lsm_status lsm_range(lsm_t* h, const uint32_t* d_k1, const uint32_t* d_k2, uint64_t nq, uint64_t* d_offsets,
                     uint32_t* d_keys, uint32_t* d_vals, uint64_t capacity, uint64_t* total_out, void* stream) {
  if (!h || !d_offsets || !total_out || (nq && (!d_k1 || !d_k2))) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  const LevelSet ls = full_levels(h);
  if (nq == 0 || ls.count == 0) {
    LSM_TRY(cudaMemsetAsync(d_offsets, 0, sizeof(uint64_t) * (nq + 1), st));
    *total_out = 0;
    return LSM_OK;
  }
  // scratch: counts[nq] | bounds[nq * 2 * levels] | scan look-back[tiles] |
  // wide-query list[nq + 1]
  const uint64_t cnt_words = round_up(nq, 2);
  const uint64_t bnd_words = round_up(nq * 2 * ls.count, 2);
  const uint64_t lb_words = scan_tiles(nq);
  LSM_TRY(ensure_q(h, (cnt_words + bnd_words) * 4 + lb_words * 8 + (nq + 1) * 4));
  uint32_t* counts = reinterpret_cast<uint32_t*>(h->d_q);
  uint32_t* bounds = counts + cnt_words;
  uint64_t* lb = reinterpret_cast<uint64_t*>(bounds + bnd_words);
  uint32_t* wide = reinterpret_cast<uint32_t*>(lb + lb_words);
  {
    ProfScope ps(h, LSM_PROF_COUNT, double(nq) * (12.0 + 64.0 * ls.count), st);
    LSM_TRY(count_launch(ls, d_k1, d_k2, nq, counts, bounds, st, nullptr, wide));
    LSM_TRY(scan_launch(counts, nq, d_offsets, lb, h->d_misc + kMiscCtrB, h->d_misc + kMiscSticky, st));
  }
  LSM_TRY(cudaMemcpyAsync(h->h_u64, d_offsets + nq, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  LSM_TRY(cudaStreamSynchronize(st));
  const uint64_t total = *h->h_u64;
  *total_out = total;
  if (total > capacity) return LSM_ERR_CAPACITY;
  if (total && (!d_keys || !d_vals)) return LSM_ERR_ARG;
  ProfScope ps(h, LSM_PROF_EMIT, 8.0 * double(total) + 8.0 * double(nq), st);
  return cuda_status(range_emit_launch(ls, nq, bounds, d_offsets, d_keys, d_vals, st, nullptr, d_k1, d_k2, wide));
}

// Rebuild of the levels from sorted sources (rank order: newest first): the
// fold keeps the first element of every key when it is regular and compacts
// the survivors; the n' live pairs then fill the set bits of r' = ceil(n'/b)
// in ascending level order, with placebo tombstones after the last one
// (§IV-E).  Synchronises with `st` (the host must learn n').
static lsm_status rebuild(lsm_t* h, const FoldSources& src, uint64_t total, cudaStream_t st) {
  if (h->clean_cap < total) {
    if (h->d_ck) cudaFree(h->d_ck);
    if (h->d_cv) cudaFree(h->d_cv);
    if (h->d_clb) cudaFree(h->d_clb);
    h->d_ck = h->d_cv = nullptr;
    h->d_clb = nullptr;
    h->clean_cap = 0;
    const uint64_t cap = h->capacity;  // enough for any later cleanup too
    LSM_TRY(dalloc(&h->d_ck, cap + kSlack));
    LSM_TRY(dalloc(&h->d_cv, cap + kSlack));
    LSM_TRY(dalloc(&h->d_clb, fold_tiles(cap) + 1));
    h->clean_cap = cap;
  }
  FoldArgs f{};
  f.src = src;
  f.total = total;
  f.out_keys = h->d_ck;
  f.out_vals = h->d_cv;
  f.part = h->d_part;
  f.status = h->d_misc + kMiscSticky;
  f.cleanup = true;
  f.lookback = h->d_clb;
  f.tile_ctr = h->d_misc + kMiscCtrA;
  f.out_count = h->d_u64;
  {
    ProfScope ps(h, LSM_PROF_CLEANUP, 8.0 * double(total), st);
    LSM_TRY(fold_launch(f, st));
  }
  LSM_TRY(cudaMemcpyAsync(h->h_u64, h->d_u64, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  LSM_TRY(cudaStreamSynchronize(st));
  const uint64_t n_live = *h->h_u64;
  if (n_live > total) return LSM_ERR_CUDA;
  const uint64_t r2 = (n_live + h->b - 1) / h->b;
  h->l0_buf = -1;  // every level is rewritten in the level array
  DistributeArgs d{};
  d.src_keys = h->d_ck;
  d.src_vals = h->d_cv;
  d.n_live = n_live;
  d.keys = h->d_keys;
  d.vals = h->d_vals;
  d.total = r2 * h->b;
  for (uint32_t i = 0; i < h->L; ++i) {
    if (!((r2 >> i) & 1u)) continue;
    d.level_off[d.nlevels] = h->level_off[i];
    d.level_start[d.nlevels] = uint64_t(h->b) * (r2 & ((1ull << i) - 1));
    d.level_size[d.nlevels] = uint64_t(h->b) << i;
    ++d.nlevels;
  }
  {
    ProfScope ps(h, LSM_PROF_CLEANUP, 8.0 * double(d.total), st);
    LSM_TRY(distribute_launch(d, st));
    for (uint32_t i = 0; i < h->L; ++i)
      if ((r2 >> i) & 1u)
        LSM_TRY(build_fence_launch(level_keys(h, i), h->b << i, level_fence(h, i), h->fshift[i], st));
  }
  h->r = r2;
  return LSM_OK;
}

lsm_status lsm_cleanup(lsm_t* h, void* stream) {
  if (!h) return LSM_ERR_ARG;
  if (h->r == 0) return LSM_OK;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  const LevelSet ls = full_levels(h);
  FoldSources src{};
  src.count = ls.count;
  for (int i = 0; i < ls.count; ++i) {
    src.keys[i] = ls.keys[i];
    src.vals[i] = ls.vals[i];
    src.fence[i] = ls.fence[i];
    src.fshift[i] = ls.fshift[i];
    src.n[i] = ls.n[i];
  }
  return rebuild(h, src, h->r * h->b, st);
}

lsm_status lsm_bulk_build(lsm_t* h, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n, void* stream) {
  if (!h || (n && (!d_keys || !d_vals))) return LSM_ERR_ARG;
  if (h->r != 0) return LSM_ERR_ARG;
  if (n == 0) return LSM_OK;
  if (n > h->capacity || n > 0xFFFFFFFFull) return LSM_ERR_FULL;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  // one stable sort of the whole reversed input (the last occurrence of a key
  // first), with its prefix index, into temporary buffers
  const uint64_t npad = round_up(n, kLevelAlign) + kSlack;
  const uint64_t tiles = (n + kSortTile - 1) / kSortTile;
  const int fs = fence_shift_for(n);
  uint32_t *buf = nullptr, *ctl = nullptr, *tilecnt = nullptr;
  uint64_t* lookback = nullptr;
  lsm_status result = LSM_OK;
  cudaError_t e = dalloc(&buf, 4 * npad + fence_words(fs));
  if (e == cudaSuccess) e = dalloc(&ctl, 2 * kSortCtlWords);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 4ull * 2 * kSortCtlWords, st);
  if (e == cudaSuccess) e = dalloc(&tilecnt, msd_ws_words(n < kMsdMaxN ? n : kMsdMaxN));
  if (e == cudaSuccess) e = dalloc(&lookback, uint64_t(kSortPasses) * tiles * 256);
  if (e == cudaSuccess) e = cudaMemsetAsync(lookback, 0, 8ull * kSortPasses * tiles * 256, st);
  if (e == cudaSuccess) {
    SortWorkspace ws{};
    ws.ctl = ctl;
    ws.flip = 0;
    ws.lookback = lookback;
    ws.max_tiles = uint32_t(tiles);
    ws.epoch = 0;
    ws.sticky = h->d_misc + kMiscSticky;
    ws.tilecnt = tilecnt;
    SortArgs a{};
    a.mode = kSortInsert;
    a.in_keys = d_keys;
    a.in_vals = d_vals;
    a.n_in = n;
    a.n = uint32_t(n);
    a.out_keys = buf;
    a.out_vals = buf + npad;
    a.tmp_keys = buf + 2 * npad;
    a.tmp_vals = buf + 3 * npad;
    a.fence = buf + 4 * npad;
    a.fshift = fs;
    *reinterpret_cast<volatile uint32_t*>(h->h_status) = 0u;
    e = sort_launch(a, ws, st, h->d_status_map, h->ev);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && (*reinterpret_cast<volatile uint32_t*>(h->h_status) & kErrBadKey)) {
      result = LSM_ERR_KEY_RANGE;
    } else if (e == cudaSuccess) {
      FoldSources src{};
      src.count = 1;
      src.keys[0] = a.out_keys;
      src.vals[0] = a.out_vals;
      src.fence[0] = a.fence;
      src.fshift[0] = fs;
      src.n[0] = uint32_t(n);
      result = rebuild(h, src, n, st);
    }
  }
  cudaStreamSynchronize(st);
  if (buf) cudaFree(buf);
  if (ctl) cudaFree(ctl);
  if (tilecnt) cudaFree(tilecnt);
  if (lookback) cudaFree(lookback);
  if (e != cudaSuccess) return cuda_status(e);
  return result;
}

lsm_status lsm_stats(const lsm_t* h, uint64_t* r, uint64_t* resident, uint32_t* b, uint32_t* levels) {
  if (!h) return LSM_ERR_ARG;
  if (r) *r = h->r;
  if (resident) *resident = h->r * h->b;
  if (b) *b = h->b;
  if (levels) *levels = h->L;
  return LSM_OK;
}

lsm_status lsm_level_offset(const lsm_t* h, uint32_t i, uint64_t* offset, uint64_t* size) {
  if (!h || !offset || !size) return LSM_ERR_ARG;
  if (i >= h->L) {
    *offset = h->capacity;
    *size = 0;
    return LSM_OK;
  }
  *offset = h->level_off[i];
  *size = uint64_t(h->b) << i;
  return LSM_OK;
}

uint64_t lsm_capacity(const lsm_t* h) { return h ? h->capacity : 0; }

lsm_status lsm_reset(lsm_t* h) {
  if (!h) return LSM_ERR_ARG;
  h->r = 0;
  h->l0_buf = -1;
  return LSM_OK;
}

lsm_status lsm_stream_wait(lsm_t* h, void* stream) {
  if (!h) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  return cuda_status(join_side(h, static_cast<cudaStream_t>(stream)));
}

lsm_status lsm_profile(lsm_t* h, int enable) {
  if (!h || enable < 0 || enable >= 2 + LSM_PROF_COUNT_) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  LSM_TRY(cudaDeviceSynchronize());
  for (auto& p : h->prof_pending) {
    h->prof_pool.push_back(p.a);
    h->prof_pool.push_back(p.b);
  }
  h->prof_pending.clear();
  memset(h->prof_acc, 0, sizeof(h->prof_acc));
  h->prof = enable == 0 ? 0u : (enable == 1 ? (1u << LSM_PROF_COUNT_) - 1u : 1u << (enable - 2));
  return LSM_OK;
}

lsm_status lsm_profile_read(lsm_t* h, lsm_profile_entry* out) {
  if (!h || !out) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  LSM_TRY(cudaDeviceSynchronize());
  for (auto& p : h->prof_pending) {
    float ms = 0.f;
    LSM_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
    lsm_profile_entry& e = h->prof_acc[p.group];
    e.launches += 1;
    e.ms += ms;
    e.bytes += p.bytes;
    h->prof_pool.push_back(p.a);
    h->prof_pool.push_back(p.b);
  }
  h->prof_pending.clear();
  memcpy(out, h->prof_acc, sizeof(h->prof_acc));
  return LSM_OK;
}

lsm_status lsm_dump_levels(const lsm_t* h, uint32_t* h_keys, uint32_t* h_vals, void* stream) {
  if (!h || !h_keys || !h_vals) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  for (uint32_t i = 0; i < h->L; ++i) {
    if (!((h->r >> i) & 1u)) continue;
    const uint64_t off = h->level_off[i], n = uint64_t(h->b) << i;
    LSM_TRY(cudaMemcpyAsync(h_keys + off, level_keys(h, int(i)), n * 4, cudaMemcpyDeviceToHost, st));
    LSM_TRY(cudaMemcpyAsync(h_vals + off, level_vals(h, int(i)), n * 4, cudaMemcpyDeviceToHost, st));
  }
  return cuda_status(cudaStreamSynchronize(st));
}

lsm_status lsm_save(lsm_t* h, uint32_t* h_keys, uint32_t* h_vals, uint64_t capacity, uint64_t* r_out,
                    void* stream) {
  if (!h || !r_out || (h->r && (!h_keys || !h_vals))) return LSM_ERR_ARG;
  if (h->r * h->b > capacity) return LSM_ERR_CAPACITY;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  uint64_t pos = 0;
  for (uint32_t i = 0; i < h->L; ++i) {
    if (!((h->r >> i) & 1u)) continue;
    const uint64_t n = uint64_t(h->b) << i;
    LSM_TRY(cudaMemcpyAsync(h_keys + pos, level_keys(h, int(i)), n * 4, cudaMemcpyDeviceToHost, st));
    LSM_TRY(cudaMemcpyAsync(h_vals + pos, level_vals(h, int(i)), n * 4, cudaMemcpyDeviceToHost, st));
    pos += n;
  }
  LSM_TRY(cudaStreamSynchronize(st));
  *r_out = h->r;
  return LSM_OK;
}

lsm_status lsm_load(lsm_t* h, const uint32_t* h_keys, const uint32_t* h_vals, uint64_t r, uint32_t b,
                    void* stream) {
  if (!h || b != h->b || h->r != 0 || (r && (!h_keys || !h_vals))) return LSM_ERR_ARG;
  if (r == 0) return LSM_OK;
  if (r >> h->L) return LSM_ERR_FULL;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(join_side(h, st));
  h->l0_buf = -1;  // every level lives in the level array
  uint64_t pos = 0;
  for (uint32_t i = 0; i < h->L; ++i) {
    if (!((r >> i) & 1u)) continue;
    const uint64_t n = uint64_t(h->b) << i;
    LSM_TRY(cudaMemcpyAsync(h->d_keys + h->level_off[i], h_keys + pos, n * 4, cudaMemcpyHostToDevice, st));
    LSM_TRY(cudaMemcpyAsync(h->d_vals + h->level_off[i], h_vals + pos, n * 4, cudaMemcpyHostToDevice, st));
    LSM_TRY(build_fence_launch(h->d_keys + h->level_off[i], uint32_t(n), h->d_fence + h->fence_off[i], h->fshift[i],
                               st));
    pos += n;
  }
  h->r = r;
  return LSM_OK;
}

lsm_status lsm_sort_pairs(lsm_t* h, const uint32_t* d_keys_in, const uint32_t* d_vals_in, uint32_t* d_keys_out,
                          uint32_t* d_vals_out, uint64_t n, void* stream) {
  if (!h || n > h->b || (n && (!d_keys_in || !d_vals_in || !d_keys_out || !d_vals_out))) return LSM_ERR_ARG;
  if (n == 0) return LSM_OK;
  DeviceGuard g(h->device);
  SortArgs a{};
  a.mode = kSortPairs;
  a.in_keys = d_keys_in;
  a.in_vals = d_vals_in;
  a.n_in = n;
  a.n = uint32_t(n);
  a.out_keys = d_keys_out;
  a.out_vals = d_vals_out;
  a.tmp_keys = h->d_tk;
  a.tmp_vals = h->d_tv;
  return cuda_status(sort_launch(a, h->sws, static_cast<cudaStream_t>(stream), nullptr, nullptr));
}

lsm_status lsm_set_option(lsm_t* h, lsm_option opt, int64_t value) {
  if (!h) return LSM_ERR_ARG;
  if (opt == LSM_OPT_LOOKUP_MODE) {
    if (value < 0 || value > 2) return LSM_ERR_ARG;
    h->lookup_mode = int(value);
    return LSM_OK;
  }
  if (opt == LSM_OPT_KEY_CHECK) {
    if (value < 0 || value > 1) return LSM_ERR_ARG;
    h->key_check_deferred = value == 1;
    return LSM_OK;
  }
  return LSM_ERR_ARG;
}

lsm_status lsm_get_option(lsm_t* h, lsm_option opt, int64_t* value) {
  if (value && opt == LSM_OPT_KERNEL_LAUNCHES) {  // process-wide, no handle needed
    *value = int64_t(launches_so_far());
    return LSM_OK;
  }
  if (!h || !value) return LSM_ERR_ARG;
  if (opt == LSM_OPT_LOOKUP_MODE) {
    *value = h->lookup_mode;
    return LSM_OK;
  }
  if (opt == LSM_OPT_KEY_CHECK) {
    *value = h->key_check_deferred ? 1 : 0;
    return LSM_OK;
  }
  if (opt == LSM_OPT_DEVICE_ERROR) {
    DeviceGuard g(h->device);
    uint32_t w = 0;
    LSM_TRY(cudaDeviceSynchronize());
    LSM_TRY(cudaMemcpy(&w, h->d_misc + kMiscSticky, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    LSM_TRY(cudaMemset(h->d_misc + kMiscSticky, 0, sizeof(uint32_t)));
    *value = w;
    return LSM_OK;
  }
  return LSM_ERR_ARG;
}

}  // extern "C"
