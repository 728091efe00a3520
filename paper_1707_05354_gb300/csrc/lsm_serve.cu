// Serving engine of the GPU LSM (include/gpulsm.h, lsm_server_*): a
// continuous-batching loop over one dictionary that replays a trace of
// requests (insert / delete / lookup / count / range of 1 .. thousands of
// keys each) in real time and records each request's completion.
//
// Requests become visible at their arrival times and wait in two queues,
// updates and retrievals, in arrival order.  The loop admits them as
// GROUPS into a few in-flight slots:
//   update group     whole update requests, up to b ops, applied as ONE
//                    ordered batch (lsm_update_batch_ordered: the last op
//                    on a key decides, so coalescing requests keeps the
//                    meaning of applying them one after another); admitted
//                    when b ops are pending, when b/2 are pending and no
//                    update group is in flight, when its oldest request has
//                    waited flush_us, or when no more requests will arrive.
//   retrieval group  every pending retrieval up to group_keys keys, admitted
//                    as soon as a slot is free: one lookup, one count and one
//                    range launch for all of them.
// Update groups run in admission order on the server's stream (the
// dictionary's folds on its own stream); each retrieval group runs on its
// slot's stream after an event that follows every update group admitted
// before it, and beside the other retrieval groups; an update group first
// waits for the retrieval groups in flight, whose levels its fold or a
// cleanup may rewrite.  So a request sees exactly the updates admitted
// before its group: requests are linearised in admission order.  A request
// only waits with others that were pending at the same time, so the order
// respects real time.  Groups complete in any order.  The work of several
// groups overlaps on the device (retrieval groups with each other, a fold
// with the next batch's sort, copies with kernels); the host keeps admitting
// while the device works, bounded by the slots.  Range groups take two steps
// (counts and offsets, then the emit once the host knows the total); no
// update group is admitted between them, so the emit reads the state the
// counts saw.
//
// Device memory is admitted against a budget: the dictionary's levels and
// cleanup scratch, its batch scratch, and every slot's buffers (payload
// staging, results, range output).  The dictionary gets the largest number
// of levels that fits; when an update group would need a level beyond it,
// the engine runs a cleanup (§III-F) first, and refuses the group
// (LSM_ERR_BUDGET per request) if the live data still fills every level.
//
// Payloads live in device pools registered with lsm_server_set_pool; a
// request names a window of them.  The policy LSM_SERVE_FIXED is the
// comparison point: requests wait until b ops are pending (or the trace has
// ended), then everything pending runs to completion before the next
// admission.
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "lsm_internal.h"

using namespace gpulsm;

namespace {

uint64_t rup(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

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
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LSM_ERR_OOM : LSM_ERR_CUDA;
}

#define LSM_TRY(expr)                  \
  do {                                 \
    lsm_status _s = cuda_status(expr); \
    if (_s != LSM_OK) return _s;       \
  } while (0)
#define LSM_TRY_S(expr)          \
  do {                           \
    lsm_status _s = (expr);      \
    if (_s != LSM_OK) return _s; \
  } while (0)

bool is_update(uint8_t k) { return k == LSM_REQ_INSERT || k == LSM_REQ_DELETE; }

// Payload windows of the requests of one kind inside a group.
struct Section {
  uint32_t first = 0, count = 0;  // descriptor range
  uint64_t keys = 0;              // keys in the section
};

struct Slot {
  // device staging and results
  uint32_t *uk = nullptr, *uv = nullptr;
  uint8_t* ud = nullptr;
  uint32_t *q = nullptr, *val = nullptr;
  uint8_t* found = nullptr;
  uint32_t *c1 = nullptr, *c2 = nullptr, *cnt = nullptr;
  uint32_t *r1 = nullptr, *r2 = nullptr, *rcnt = nullptr, *bounds = nullptr;
  uint64_t *roff = nullptr, *lb = nullptr;
  uint32_t *rk = nullptr, *rv = nullptr;
  uint32_t* ctr = nullptr;
  uint64_t* d_start = nullptr;
  uint64_t* d_dst = nullptr;
  uint8_t* d_flag = nullptr;
  // pinned host mirrors
  uint64_t* h_start = nullptr;
  uint64_t* h_dst = nullptr;
  uint8_t* h_flag = nullptr;
  uint32_t *h_val = nullptr, *h_cnt = nullptr;
  uint8_t* h_found = nullptr;
  uint64_t* h_roff = nullptr;
  uint32_t *h_rk = nullptr, *h_rv = nullptr;
  uint64_t* h_total = nullptr;
  cudaStream_t st = nullptr;  // the slot's retrieval groups (update groups use the server's stream)
  cudaEvent_t ev_done = nullptr, ev_total = nullptr, ev_start = nullptr;
  cudaEvent_t ev_ph[6] = {};  // retrieval phases: after gathers+sorts ... before the emit
  // sorting the queries of a large group (by key, with their positions):
  // set A for lookups and counts, set B for ranges (its positions are read
  // again by the emit)
  SortWorkspace sws{};
  uint32_t *sort_ctl = nullptr, *sort_tilecnt = nullptr;
  uint32_t* sa[4] = {};  // sorted keys, positions, two scratch arrays
  uint32_t* sb[4] = {};
};

// Groups of at least this many keys of one kind are processed in key order
// (a sort first): neighbouring threads then search neighbouring parts of
// every level, which matters once the levels span many gigabytes.
constexpr uint64_t kSortQueriesFrom = 1u << 15;

enum Stage { kFree = 0, kRunning = 1, kRangePending = 2 };

struct Group {
  bool update = false;
  int slot = -1;
  int stage = kFree;
  uint64_t seq = 0;
  std::vector<uint64_t> reqs;  // trace indices, admission order
  Section look, count, range;
  uint64_t range_total = 0;
  LevelSet ls{};               // the state the range counts saw
  bool refused = false;
  bool range_sorted = false;   // the range intervals were processed in key order
  // range output larger than the slot's buffer: a buffer of its own
  uint32_t *big_k = nullptr, *big_v = nullptr, *h_big_k = nullptr, *h_big_v = nullptr;
};

}  // namespace

struct lsm_server_t {
  lsm_server_config cfg{};
  lsm_t* dict = nullptr;
  cudaStream_t st = nullptr;  // update groups (and cleanups)
  cudaEvent_t ev_applied = nullptr;  // after the latest admitted update group's sort and fold
  uint32_t L = 0;             // dictionary levels
  uint32_t max_levels = 0;    // bound on full levels (bounds scratch)
  uint32_t max_req = 0;       // descriptors per group
  uint64_t device_bytes = 0;  // slots + dictionary estimate
  const uint32_t *pool_a = nullptr, *pool_b = nullptr, *pool_c = nullptr;
  uint64_t pool_n = 0;
  std::vector<Slot> slots;
};

namespace {

template <typename T>
cudaError_t dalloc(T** p, uint64_t count) {
  const cudaError_t g = alloc_gate();
  if (g != cudaSuccess) return g;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}
template <typename T>
cudaError_t halloc(T** p, uint64_t count) {
  const cudaError_t g = alloc_gate();
  if (g != cudaSuccess) return g;
  return cudaHostAlloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1), cudaHostAllocDefault);
}

// Device bytes of one slot.
uint64_t slot_bytes(const lsm_server_config& c, uint32_t max_levels, uint32_t max_req) {
  const uint64_t b = rup(c.b, 32) + 32, G = rup(c.group_keys, 32) + 32;
  return b * 9 + G * (4 + 4 + 1) + G * 12 + G * (4 + 4 + 4 + 8ull * max_levels) + (G + 1) * 8 +
         (G / 2048 + 2) * 8 + uint64_t(c.range_cap) * 8 + uint64_t(max_req) * (8 + 8 + 1) + 8 * 4 * G +
         4ull * msd_ws_words(G < kMsdMaxN ? G : kMsdMaxN) + 64;
}

// Device bytes of a dictionary with L levels of batch size b, as lsm_create
// and a cleanup allocate them (levels, cleanup scratch, the sorted-batch
// buffers, sort scratch, prefix indexes, co-rank table, query scratch).
uint64_t dict_bytes(uint32_t b, uint32_t L) {
  const uint64_t cap = uint64_t(b) * ((1ull << L) - 1);
  const uint64_t bp = rup(b, 32) + 32;
  return 8 * cap + 8 * cap + 8 * (cap / kFoldTile + 2) + (kBatchBufs + 2) * 8 * bp + cap / 2 + 16 * bp +
         4 * (cap / kFoldTile + 2) * (L + 1) +
         (64ull << 20);
}

void free_slot(Slot& s) {
  void* d[] = {s.uk, s.uv, s.ud, s.q,  s.val, s.found, s.c1, s.c2, s.cnt, s.r1, s.r2, s.rcnt, s.bounds,
               s.roff, s.lb, s.rk, s.rv, s.ctr, s.d_start, s.d_dst, s.d_flag};
  for (void* p : d)
    if (p) cudaFree(p);
  void* h[] = {s.h_start, s.h_dst, s.h_flag, s.h_val, s.h_cnt, s.h_found, s.h_roff, s.h_rk, s.h_rv,
               s.h_total};
  for (void* p : h)
    if (p) cudaFreeHost(p);
  if (s.st) cudaStreamDestroy(s.st);
  if (s.ev_done) cudaEventDestroy(s.ev_done);
  if (s.ev_total) cudaEventDestroy(s.ev_total);
  if (s.ev_start) cudaEventDestroy(s.ev_start);
  for (cudaEvent_t e : s.ev_ph)
    if (e) cudaEventDestroy(e);
  if (s.sort_ctl) cudaFree(s.sort_ctl);
  if (s.sort_tilecnt) cudaFree(s.sort_tilecnt);
  for (int i = 0; i < 4; ++i) {
    if (s.sa[i]) cudaFree(s.sa[i]);
    if (s.sb[i]) cudaFree(s.sb[i]);
  }
  s = Slot{};
}

cudaError_t alloc_slot(Slot& s, const lsm_server_config& c, uint32_t max_levels, uint32_t max_req) {
  const uint64_t b = rup(c.b, 32) + 32, G = rup(c.group_keys, 32) + 32, R = uint64_t(c.range_cap) + 32;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&s.uk, b);
  if (e == cudaSuccess) e = dalloc(&s.uv, b);
  if (e == cudaSuccess) e = dalloc(&s.ud, b);
  if (e == cudaSuccess) e = dalloc(&s.q, G);
  if (e == cudaSuccess) e = dalloc(&s.val, G);
  if (e == cudaSuccess) e = dalloc(&s.found, G);
  if (e == cudaSuccess) e = dalloc(&s.c1, G);
  if (e == cudaSuccess) e = dalloc(&s.c2, G);
  if (e == cudaSuccess) e = dalloc(&s.cnt, G);
  if (e == cudaSuccess) e = dalloc(&s.r1, G);
  if (e == cudaSuccess) e = dalloc(&s.r2, G);
  if (e == cudaSuccess) e = dalloc(&s.rcnt, G);
  if (e == cudaSuccess) e = dalloc(&s.bounds, G * 2 * max_levels);
  if (e == cudaSuccess) e = dalloc(&s.roff, G + 1);
  if (e == cudaSuccess) e = dalloc(&s.lb, scan_tiles(G) + 2);
  if (e == cudaSuccess) e = dalloc(&s.rk, R);
  if (e == cudaSuccess) e = dalloc(&s.rv, R);
  if (e == cudaSuccess) e = dalloc(&s.ctr, 16);
  if (e == cudaSuccess) e = dalloc(&s.d_start, max_req);
  if (e == cudaSuccess) e = dalloc(&s.d_dst, max_req);
  if (e == cudaSuccess) e = dalloc(&s.d_flag, max_req);
  if (e == cudaSuccess) e = halloc(&s.h_start, max_req);
  if (e == cudaSuccess) e = halloc(&s.h_dst, max_req);
  if (e == cudaSuccess) e = halloc(&s.h_flag, max_req);
  if (e == cudaSuccess) e = halloc(&s.h_val, G);
  if (e == cudaSuccess) e = halloc(&s.h_cnt, G);
  if (e == cudaSuccess) e = halloc(&s.h_found, G);
  if (e == cudaSuccess) e = halloc(&s.h_roff, G + 1);
  if (e == cudaSuccess) e = halloc(&s.h_rk, R);
  if (e == cudaSuccess) e = halloc(&s.h_rv, R);
  if (e == cudaSuccess) e = halloc(&s.h_total, 8);
  if (e == cudaSuccess) e = cudaMemset(s.ctr, 0, 64);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&s.ev_done);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_total, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&s.ev_start);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreate(&s.ev_ph[i]);
  if (e == cudaSuccess) e = dalloc(&s.sort_ctl, 2 * kSortCtlWords);
  if (e == cudaSuccess) e = cudaMemset(s.sort_ctl, 0, 4ull * 2 * kSortCtlWords);
  if (e == cudaSuccess) e = dalloc(&s.sort_tilecnt, msd_ws_words(G < kMsdMaxN ? G : kMsdMaxN));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    e = dalloc(&s.sa[i], G);
    if (e == cudaSuccess) e = dalloc(&s.sb[i], G);
  }
  s.sws.ctl = s.sort_ctl;
  s.sws.flip = 0;
  s.sws.tilecnt = s.sort_tilecnt;
  return e;
}

double now_us(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

// The run of one trace.
struct Run {
  lsm_server_t* s;
  const lsm_trace* t;
  lsm_trace_result* res;
  std::chrono::steady_clock::time_point t0;
  std::deque<uint64_t> upd, ret;  // pending requests
  uint64_t upd_ops = 0, ret_keys = 0;
  uint64_t next = 0, done = 0, seq = 0;
  std::vector<Group> inflight;    // in admission order
  std::vector<int> free_slots;
  int pending_ranges = 0;         // range groups awaiting their totals (no update admitted meanwhile)
  uint64_t range_pos = 0;         // next free entry of the caller's range output

  // Update groups admitted and not yet completed.
  int updates_in_flight() const {
    int c = 0;
    for (const Group& g : inflight) c += g.update ? 1 : 0;
    return c;
  }

  // The update queue is ready for a group (ignoring range groups in flight):
  // a full batch, the end of the trace, a request that has waited flush_us,
  // or -- continuous batching -- half a batch while no update group is on
  // the device (the device would otherwise idle on updates until the batch
  // fills or times out).
  bool updates_ready(double now) const {
    if (upd.empty()) return false;
    if (upd_ops >= s->cfg.b || next >= t->n) return true;
    if (s->cfg.policy == LSM_SERVE_CONTINUOUS && 2 * upd_ops >= s->cfg.b && updates_in_flight() == 0) return true;
    return now - t->arrival_us[upd.front()] >= s->cfg.flush_us;
  }
  bool want_updates(double now) const { return pending_ranges == 0 && updates_ready(now); }

  // Writes the descriptors of requests [a, b) of `reqs` into the slot's
  // pinned arrays from index `first`; returns the keys.
  uint64_t describe(Slot& sl, const std::vector<uint64_t>& reqs, size_t a, size_t b, uint32_t first) {
    uint64_t keys = 0;
    for (size_t j = a; j < b; ++j) {
      const uint64_t i = reqs[j];
      const uint32_t d = first + uint32_t(j - a);
      sl.h_start[d] = t->start[i];
      sl.h_dst[d] = keys;
      sl.h_flag[d] = t->kind[i] == LSM_REQ_DELETE ? 1 : 0;
      keys += t->size[i];
    }
    return keys;
  }

  lsm_status admit_updates(int slot_id) {
    Slot& sl = s->slots[slot_id];
    Group g;
    g.update = true;
    g.slot = slot_id;
    g.seq = seq++;
    uint64_t ops = 0;
    while (!upd.empty() && g.reqs.size() < s->max_req) {
      const uint64_t i = upd.front();
      if (ops + t->size[i] > s->cfg.b) break;
      ops += t->size[i];
      g.reqs.push_back(i);
      upd.pop_front();
    }
    upd_ops -= ops;
    if (g.reqs.empty()) return LSM_ERR_ARG;  // cannot happen: sizes are <= b
    // retrieval groups still reading the levels finish before this group's
    // sort and fold (and a cleanup) may rewrite level memory
    for (const Group& o : inflight)
      if (!o.update) LSM_TRY(cudaStreamWaitEvent(s->st, s->slots[o.slot].ev_done, 0));
    // budget: a full dictionary is cleaned first; refused if still full
    const uint32_t L = dict_L(s->dict);
    uint64_t r = dict_r(s->dict);
    auto full = [&](uint64_t rr) {
      int k = 0;
      while ((rr >> k) & 1u) ++k;
      return k >= int(L);
    };
    if (full(r)) {
      const double c0 = now_us(t0);
      LSM_TRY_S(lsm_cleanup(s->dict, s->st));
      res->host_cleanup_us += now_us(t0) - c0;
      res->cleanups += 1;
      r = dict_r(s->dict);
    }
    LSM_TRY(cudaEventRecord(sl.ev_start, s->st));
    if (full(r)) {
      g.refused = true;
      res->refused += g.reqs.size();
      LSM_TRY(cudaEventRecord(sl.ev_done, s->st));
    } else {
      const uint64_t n = describe(sl, g.reqs, 0, g.reqs.size(), 0);
      const uint32_t nd = uint32_t(g.reqs.size());
      LSM_TRY(cudaMemcpyAsync(sl.d_start, sl.h_start, 8ull * nd, cudaMemcpyHostToDevice, s->st));
      LSM_TRY(cudaMemcpyAsync(sl.d_dst, sl.h_dst, 8ull * nd, cudaMemcpyHostToDevice, s->st));
      LSM_TRY(cudaMemcpyAsync(sl.d_flag, sl.h_flag, nd, cudaMemcpyHostToDevice, s->st));
      LSM_TRY(gather_update_launch(s->pool_a, s->pool_b, sl.d_start, sl.d_dst, sl.d_flag, nd, n, sl.uk, sl.uv,
                                   sl.ud, s->st));
      LSM_TRY_S(dict_update_ordered(s->dict, sl.uk, sl.uv, sl.ud, n, s->st, false));
      LSM_TRY(dict_record_applied(s->dict, sl.ev_done, s->st));
      LSM_TRY(dict_record_applied(s->dict, s->ev_applied, s->st));
      res->update_batches += 1;
      res->padded_ops += s->cfg.b - n;
    }
    g.stage = kRunning;
    inflight.push_back(std::move(g));
    return LSM_OK;
  }

  lsm_status admit_retrievals(int slot_id) {
    Slot& sl = s->slots[slot_id];
    cudaStream_t rs = sl.st;
    Group g;
    g.update = false;
    g.slot = slot_id;
    g.seq = seq++;
    // take requests in arrival order up to the key and descriptor caps;
    // then lay them out by kind
    uint64_t keys = 0;
    std::vector<uint64_t> take;
    while (!ret.empty() && take.size() < s->max_req) {
      const uint64_t i = ret.front();
      if (!take.empty() && keys + t->size[i] > s->cfg.group_keys) break;
      keys += t->size[i];
      take.push_back(i);
      ret.pop_front();
    }
    ret_keys -= keys;
    for (int kind : {int(LSM_REQ_LOOKUP), int(LSM_REQ_COUNT), int(LSM_REQ_RANGE)})
      for (uint64_t i : take)
        if (t->kind[i] == kind) g.reqs.push_back(i);
    size_t pos = 0;
    Section* secs[3] = {&g.look, &g.count, &g.range};
    for (int k = 0; k < 3; ++k) {
      Section& sec = *secs[k];
      sec.first = uint32_t(pos);
      size_t e = pos;
      while (e < g.reqs.size() && t->kind[g.reqs[e]] == uint8_t(LSM_REQ_LOOKUP + k)) ++e;
      sec.count = uint32_t(e - pos);
      sec.keys = describe(sl, g.reqs, pos, e, sec.first);
      pos = e;
    }
    const uint32_t nd = uint32_t(g.reqs.size());
    LSM_TRY(cudaEventRecord(sl.ev_start, rs));
    LSM_TRY(cudaMemcpyAsync(sl.d_start, sl.h_start, 8ull * nd, cudaMemcpyHostToDevice, rs));
    LSM_TRY(cudaMemcpyAsync(sl.d_dst, sl.h_dst, 8ull * nd, cudaMemcpyHostToDevice, rs));
    // the group sees every update group admitted before it (their sorts
    // and folds), and runs beside other retrieval groups
    LSM_TRY(cudaStreamWaitEvent(rs, s->ev_applied, 0));
    LSM_TRY(dict_join(s->dict, rs));
    g.ls = dict_levels(s->dict);
    const LevelSet& ls = g.ls;
    LSM_TRY(cudaEventRecord(sl.ev_ph[0], rs));
    if (g.look.count) {
      const uint32_t f = g.look.first;
      LSM_TRY(gather_windows_launch(s->pool_a, nullptr, sl.d_start + f, sl.d_dst + f, g.look.count, g.look.keys,
                                    sl.q, nullptr, rs));
      lsm_status err = LSM_OK;
      if (ls.count && sort_queries(sl, sl.sa, sl.q, g.look.keys, err)) {
        LSM_TRY(lookup_sorted_launch(ls, sl.sa[0], sl.sa[1], g.look.keys, sl.val, sl.found, rs));
      } else if (err != LSM_OK) {
        return err;
      } else if (ls.count) {
        LSM_TRY(lookup_launch(ls, sl.q, g.look.keys, sl.val, sl.found, rs));
      } else {
        LSM_TRY(cudaMemsetAsync(sl.val, 0, 4 * g.look.keys, rs));
        LSM_TRY(cudaMemsetAsync(sl.found, 0, g.look.keys, rs));
      }
      LSM_TRY(cudaMemcpyAsync(sl.h_val, sl.val, 4 * g.look.keys, cudaMemcpyDeviceToHost, rs));
      LSM_TRY(cudaMemcpyAsync(sl.h_found, sl.found, g.look.keys, cudaMemcpyDeviceToHost, rs));
    }
    LSM_TRY(cudaEventRecord(sl.ev_ph[1], rs));
    if (g.count.count) {
      const uint32_t f = g.count.first;
      LSM_TRY(gather_windows_launch(s->pool_a, s->pool_c, sl.d_start + f, sl.d_dst + f, g.count.count,
                                    g.count.keys, sl.c1, sl.c2, rs));
      lsm_status err = LSM_OK;
      if (ls.count && sort_queries(sl, sl.sa, sl.c1, g.count.keys, err))
        LSM_TRY(count_launch(ls, sl.sa[0], sl.c2, g.count.keys, sl.cnt, nullptr, rs, sl.sa[1]));
      else if (err != LSM_OK)
        return err;
      else if (ls.count)
        LSM_TRY(count_launch(ls, sl.c1, sl.c2, g.count.keys, sl.cnt, nullptr, rs));
      else
        LSM_TRY(cudaMemsetAsync(sl.cnt, 0, 4 * g.count.keys, rs));
      LSM_TRY(cudaMemcpyAsync(sl.h_cnt, sl.cnt, 4 * g.count.keys, cudaMemcpyDeviceToHost, rs));
    }
    LSM_TRY(cudaEventRecord(sl.ev_ph[2], rs));
    if (g.range.count) {
      const uint32_t f = g.range.first;
      const uint64_t nr = g.range.keys;
      LSM_TRY(gather_windows_launch(s->pool_a, s->pool_c, sl.d_start + f, sl.d_dst + f, g.range.count,
                                    g.range.keys, sl.r1, sl.r2, rs));
      if (ls.count) {
        lsm_status err = LSM_OK;
        g.range_sorted = sort_queries(sl, sl.sb, sl.r1, nr, err);
        if (err != LSM_OK) return err;
        if (g.range_sorted)
          LSM_TRY(count_launch(ls, sl.sb[0], sl.r2, nr, sl.rcnt, sl.bounds, rs, sl.sb[1]));
        else
          LSM_TRY(count_launch(ls, sl.r1, sl.r2, nr, sl.rcnt, sl.bounds, rs));
        LSM_TRY(scan_launch(sl.rcnt, nr, sl.roff, sl.lb, sl.ctr, dict_status_word(s->dict), rs));
      } else {
        LSM_TRY(cudaMemsetAsync(sl.roff, 0, 8 * (nr + 1), rs));
      }
      LSM_TRY(cudaEventRecord(sl.ev_ph[3], rs));
      LSM_TRY(cudaMemcpyAsync(sl.h_total, sl.roff + nr, 8, cudaMemcpyDeviceToHost, rs));
      LSM_TRY(cudaEventRecord(sl.ev_total, rs));
      g.stage = kRangePending;
      pending_ranges += 1;
    } else {
      LSM_TRY(cudaEventRecord(sl.ev_ph[3], rs));
      LSM_TRY(cudaEventRecord(sl.ev_done, rs));
      g.stage = kRunning;
    }
    res->retrieval_groups += 1;
    inflight.push_back(std::move(g));
    return LSM_OK;
  }

  // Sorts n query keys with their positions into set[0] (keys) / set[1]
  // (positions), when the group is large enough to profit.
  bool sort_queries(Slot& sl, uint32_t* const* set, const uint32_t* keys, uint64_t n, lsm_status& err) {
    cudaStream_t rs = sl.st;
    if (n < kSortQueriesFrom || n > kMsdMaxN) return false;
    SortArgs a{};
    a.mode = kSortQueries;
    a.in_keys = keys;
    a.n_in = n;
    a.n = uint32_t(n);
    a.out_keys = set[0];
    a.out_vals = set[1];
    a.tmp_keys = set[2];
    a.tmp_vals = set[3];
    sl.sws.sticky = dict_status_word(s->dict);
    err = cuda_status(sort_launch(a, sl.sws, rs, nullptr, nullptr));
    return err == LSM_OK;
  }

  // Second step of a range group: the emit (the state has not changed since
  // the counts: no update group was admitted in between).
  lsm_status finish_range(Group& g) {
    Slot& sl = s->slots[g.slot];
    cudaStream_t rs = sl.st;
    const uint64_t nr = g.range.keys;
    const uint64_t total = *sl.h_total;
    g.range_total = total;
    uint32_t *dk = sl.rk, *dv = sl.rv, *hk = sl.h_rk, *hv = sl.h_rv;
    if (total > s->cfg.range_cap) {
      // rare: more results than the slot holds; buffers for this group only
      LSM_TRY(alloc_gate());
      LSM_TRY(cudaMallocAsync(reinterpret_cast<void**>(&g.big_k), 4 * total, rs));
      LSM_TRY(cudaMallocAsync(reinterpret_cast<void**>(&g.big_v), 4 * total, rs));
      LSM_TRY(cudaHostAlloc(reinterpret_cast<void**>(&g.h_big_k), 4 * total, cudaHostAllocDefault));
      LSM_TRY(cudaHostAlloc(reinterpret_cast<void**>(&g.h_big_v), 4 * total, cudaHostAllocDefault));
      dk = g.big_k;
      dv = g.big_v;
      hk = g.h_big_k;
      hv = g.h_big_v;
    }
    LSM_TRY(cudaEventRecord(sl.ev_ph[4], rs));
    if (total && g.ls.count)
      LSM_TRY(range_emit_launch(g.ls, nr, sl.bounds, sl.roff, dk, dv, rs, g.range_sorted ? sl.sb[1] : nullptr));
    LSM_TRY(cudaEventRecord(sl.ev_ph[5], rs));
    LSM_TRY(cudaMemcpyAsync(sl.h_roff, sl.roff, 8 * (nr + 1), cudaMemcpyDeviceToHost, rs));
    if (total) {
      LSM_TRY(cudaMemcpyAsync(hk, dk, 4 * total, cudaMemcpyDeviceToHost, rs));
      LSM_TRY(cudaMemcpyAsync(hv, dv, 4 * total, cudaMemcpyDeviceToHost, rs));
    }
    if (g.big_k) {
      LSM_TRY(cudaFreeAsync(g.big_k, rs));
      LSM_TRY(cudaFreeAsync(g.big_v, rs));
      g.big_k = g.big_v = nullptr;
    }
    LSM_TRY(cudaEventRecord(sl.ev_done, rs));
    g.stage = kRunning;
    pending_ranges -= 1;
    return LSM_OK;
  }

  // Results of a finished group to the caller's arrays; completion times.
  void complete(Group& g, double now) {
    Slot& sl = s->slots[g.slot];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sl.ev_start, sl.ev_done) == cudaSuccess) {
      if (g.update) res->gpu_update_ms += ms;
      else res->gpu_retrieval_ms += ms;
    }
    if (!g.update) {
      // the phases (the lookups include their gathers and sort, and so on)
      auto el = [&](cudaEvent_t a, cudaEvent_t b) {
        float x = 0.f;
        return cudaEventElapsedTime(&x, a, b) == cudaSuccess ? double(x) : 0.0;
      };
      res->gpu_prep_ms += el(sl.ev_start, sl.ev_ph[0]);
      res->gpu_lookup_ms += el(sl.ev_ph[0], sl.ev_ph[1]);
      res->gpu_count_ms += el(sl.ev_ph[1], sl.ev_ph[2]);
      res->gpu_range_ms += el(sl.ev_ph[2], sl.ev_ph[3]);
      if (g.range.count) res->gpu_emit_ms += el(sl.ev_ph[4], sl.ev_ph[5]);
    }
    const double h0 = now_us(t0);
    for (uint64_t i : g.reqs) {
      res->done_us[i] = now;
      res->status[i] = g.refused ? LSM_ERR_BUDGET : LSM_OK;
      if (res->order) res->order[i] = g.seq;
    }
    if (!g.update && res->res_off) {
      auto copy_section = [&](const Section& sec, int kind) {
        uint64_t pos = 0;
        for (uint32_t d = 0; d < sec.count; ++d) {
          const uint64_t i = g.reqs[sec.first + d];
          const uint64_t o = res->res_off[i];
          const uint32_t m = t->size[i];
          if (kind == LSM_REQ_LOOKUP) {
            if (res->val) memcpy(res->val + o, sl.h_val + pos, 4ull * m);
            if (res->found) memcpy(res->found + o, sl.h_found + pos, m);
          } else if (kind == LSM_REQ_COUNT) {
            if (res->val) memcpy(res->val + o, sl.h_cnt + pos, 4ull * m);
          } else {
            const uint32_t* hk = g.h_big_k ? g.h_big_k : sl.h_rk;
            const uint32_t* hv = g.h_big_v ? g.h_big_v : sl.h_rv;
            for (uint32_t k = 0; k < m; ++k) {
              const uint64_t a = sl.h_roff[pos + k], z = sl.h_roff[pos + k + 1];
              if (res->val) res->val[o + k] = uint32_t(z - a);
              if (res->range_start) res->range_start[o + k] = range_pos;
              if (res->rk && res->rv && range_pos + (z - a) <= res->range_cap) {
                memcpy(res->rk + range_pos, hk + a, 4 * (z - a));
                memcpy(res->rv + range_pos, hv + a, 4 * (z - a));
              }
              range_pos += z - a;
            }
          }
          pos += m;
        }
      };
      copy_section(g.look, LSM_REQ_LOOKUP);
      copy_section(g.count, LSM_REQ_COUNT);
      copy_section(g.range, LSM_REQ_RANGE);
    }
    if (g.h_big_k) cudaFreeHost(g.h_big_k);
    if (g.h_big_v) cudaFreeHost(g.h_big_v);
    g.h_big_k = g.h_big_v = nullptr;
    res->range_total += g.range_total;
    done += g.reqs.size();
    free_slots.push_back(g.slot);
    res->host_complete_us += now_us(t0) - h0;
  }

  lsm_status poll(double now) {
    // range groups whose totals arrived get their emit (in admission order:
    // no update group is admitted while one waits)
    for (size_t j = 0; j < inflight.size(); ++j) {
      Group& g = inflight[j];
      Slot& sl = s->slots[g.slot];
      if (g.stage == kRangePending) {
        const cudaError_t e = cudaEventQuery(sl.ev_total);
        if (e == cudaErrorNotReady) continue;
        LSM_TRY(e);
        const double f0 = now_us(t0);
        LSM_TRY_S(finish_range(g));
        res->host_range_us += now_us(t0) - f0;
      }
    }
    // groups on different streams complete in any order
    for (size_t j = 0; j < inflight.size();) {
      Group& g = inflight[j];
      if (g.stage != kRunning) {
        ++j;
        continue;
      }
      const cudaError_t e = cudaEventQuery(s->slots[g.slot].ev_done);
      if (e == cudaErrorNotReady) {
        ++j;
        continue;
      }
      LSM_TRY(e);
      complete(g, now);
      inflight.erase(inflight.begin() + long(j));
    }
    return LSM_OK;
  }

  void arrive(double now) {
    while (next < t->n && t->arrival_us[next] <= now) {
      if (is_update(t->kind[next])) {
        upd.push_back(next);
        upd_ops += t->size[next];
      } else {
        ret.push_back(next);
        ret_keys += t->size[next];
      }
      ++next;
    }
  }

  lsm_status run_continuous() {
    while (done < t->n) {
      const double now = now_us(t0);
      arrive(now);
      LSM_TRY_S(poll(now));
      while (!free_slots.empty()) {
        const bool wu = want_updates(now);
        bool wr = !ret.empty();
        // a ready update group held back only by range groups in flight goes
        // before retrievals that arrived after it (else a steady stream of
        // range groups would keep the barrier up and starve the updates)
        if (!wu && wr && updates_ready(now) && t->arrival_us[upd.front()] <= t->arrival_us[ret.front()]) wr = false;
        if (!wu && !wr) break;
        const int sl = free_slots.back();
        free_slots.pop_back();
        // the older front goes first
        const double a0 = now_us(t0);
        if (wu && (!wr || t->arrival_us[upd.front()] <= t->arrival_us[ret.front()])) {
          LSM_TRY_S(admit_updates(sl));
          res->host_admit_update_us += now_us(t0) - a0;
        } else {
          LSM_TRY_S(admit_retrievals(sl));
          res->host_admit_retrieval_us += now_us(t0) - a0;
        }
      }
      if (inflight.empty() && next < t->n && upd.empty() && ret.empty()) {
        // idle until the next arrival
        const double wait = t->arrival_us[next] - now_us(t0);
        if (wait > 50.0) {
          std::this_thread::sleep_for(std::chrono::microseconds(int64_t(wait - 20.0)));
          res->host_sleep_us += wait - 20.0;
        }
      }
    }
    return LSM_OK;
  }

  lsm_status drain_all() {
    while (!inflight.empty()) {
      LSM_TRY(cudaStreamSynchronize(s->st));
      for (const Slot& sl : s->slots) LSM_TRY(cudaStreamSynchronize(sl.st));
      LSM_TRY_S(poll(now_us(t0)));
    }
    return LSM_OK;
  }

  lsm_status run_fixed() {
    while (done < t->n) {
      double now = now_us(t0);
      arrive(now);
      if (upd_ops + ret_keys < s->cfg.b && next < t->n) {
        const double wait = t->arrival_us[next] - now_us(t0);
        if (wait > 50.0) std::this_thread::sleep_for(std::chrono::microseconds(int64_t(wait - 20.0)));
        continue;
      }
      // everything pending, updates first (in arrival order), then the
      // retrievals, each group run to completion
      while (!upd.empty()) {
        const int sl = free_slots.back();
        free_slots.pop_back();
        LSM_TRY_S(admit_updates(sl));
        LSM_TRY_S(drain_all());
      }
      while (!ret.empty()) {
        const int sl = free_slots.back();
        free_slots.pop_back();
        LSM_TRY_S(admit_retrievals(sl));
        LSM_TRY_S(drain_all());
      }
    }
    return LSM_OK;
  }
};

}  // namespace

extern "C" {

lsm_status lsm_server_create(lsm_server_t** out, const lsm_server_config* cfg) {
  if (!out || !cfg || cfg->b == 0 || cfg->b > kMsdMaxN || cfg->group_keys == 0 || cfg->slots == 0 ||
      cfg->slots > 16 || cfg->flush_us < 0 || (cfg->policy != LSM_SERVE_CONTINUOUS && cfg->policy != LSM_SERVE_FIXED))
    return LSM_ERR_ARG;
  *out = nullptr;
  lsm_server_t* s = new (std::nothrow) lsm_server_t();
  if (!s) return LSM_ERR_OOM;
  s->cfg = *cfg;
  s->max_req = cfg->group_keys < 65536u ? cfg->group_keys : 65536u;
  // levels: the largest count whose dictionary fits the budget beside the slots
  const uint32_t nslots = cfg->policy == LSM_SERVE_FIXED ? 1u : cfg->slots;
  uint32_t L = 0;
  for (uint32_t l = 1; l <= 24; ++l) {
    const uint64_t need = dict_bytes(cfg->b, l) + nslots * slot_bytes(*cfg, l, s->max_req);
    if (need <= cfg->hbm_budget && (uint64_t(cfg->b) * ((1ull << l) - 1)) <= (1ull << 31)) L = l;
  }
  if (L == 0) {
    delete s;
    return LSM_ERR_BUDGET;
  }
  s->L = L;
  s->max_levels = L;
  s->device_bytes = dict_bytes(cfg->b, L) + nslots * slot_bytes(*cfg, L, s->max_req);
  DeviceGuard g(cfg->device);
  lsm_status st = lsm_create(&s->dict, cfg->b, uint64_t(cfg->b) * ((1ull << L) - 1), cfg->device);
  if (st != LSM_OK) {
    delete s;
    return st;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_applied, cudaEventDisableTiming);
  s->slots.resize(nslots);
  for (uint32_t i = 0; i < nslots && e == cudaSuccess; ++i) e = alloc_slot(s->slots[i], *cfg, L, s->max_req);
  if (e != cudaSuccess) {
    lsm_server_destroy(s);
    return cuda_status(e);
  }
  *out = s;
  return LSM_OK;
}

void lsm_server_destroy(lsm_server_t* s) {
  if (!s) return;
  DeviceGuard g(s->cfg.device);
  cudaDeviceSynchronize();
  for (Slot& sl : s->slots) free_slot(sl);
  if (s->st) cudaStreamDestroy(s->st);
  if (s->ev_applied) cudaEventDestroy(s->ev_applied);
  if (s->dict) lsm_destroy(s->dict);
  delete s;
}

lsm_status lsm_server_set_pool(lsm_server_t* s, const uint32_t* d_a, const uint32_t* d_b, const uint32_t* d_c,
                               uint64_t n) {
  if (!s || !d_a || !d_b || !d_c || n == 0) return LSM_ERR_ARG;
  DeviceGuard g(s->cfg.device);
  LSM_TRY(cudaDeviceSynchronize());  // the pools were written on other streams
  // update keys come from pool a: check them once here, so that batches need
  // no per-batch key check
  uint32_t* flag = nullptr;
  LSM_TRY(dalloc(&flag, 1));
  cudaError_t e = cudaMemsetAsync(flag, 0, 4, s->st);
  if (e == cudaSuccess) e = check_keys_launch(d_a, n, flag, s->st);
  uint32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(flag);
  LSM_TRY(e);
  if (h & kErrBadKey) return LSM_ERR_KEY_RANGE;
  s->pool_a = d_a;
  s->pool_b = d_b;
  s->pool_c = d_c;
  s->pool_n = n;
  return LSM_OK;
}

lsm_status lsm_server_preload(lsm_server_t* s, const uint32_t* d_keys, const uint32_t* d_vals, uint64_t n) {
  if (!s) return LSM_ERR_ARG;
  DeviceGuard g(s->cfg.device);
  LSM_TRY(cudaDeviceSynchronize());  // the pairs were written on other streams
  LSM_TRY_S(lsm_insert_batch(s->dict, d_keys, d_vals, n, s->st));
  LSM_TRY(cudaDeviceSynchronize());
  return LSM_OK;
}

lsm_status lsm_server_run(lsm_server_t* s, const lsm_trace* t, lsm_trace_result* r) {
  if (!s || !t || !r || !r->done_us || !r->status || !s->pool_a) return LSM_ERR_ARG;
  for (uint64_t i = 0; i < t->n; ++i) {
    if (t->kind[i] > LSM_REQ_RANGE || t->size[i] == 0 || t->size[i] > s->cfg.group_keys ||
        (is_update(t->kind[i]) && t->size[i] > s->cfg.b) || t->start[i] + t->size[i] > s->pool_n ||
        (i && t->arrival_us[i] < t->arrival_us[i - 1]))
      return LSM_ERR_ARG;
  }
  DeviceGuard g(s->cfg.device);
  r->range_total = 0;
  r->update_batches = r->padded_ops = r->retrieval_groups = r->cleanups = r->refused = 0;
  r->host_admit_update_us = r->host_admit_retrieval_us = r->host_range_us = r->host_complete_us = 0;
  r->host_cleanup_us = r->host_sleep_us = r->gpu_update_ms = r->gpu_retrieval_ms = 0;
  r->gpu_prep_ms = r->gpu_lookup_ms = r->gpu_count_ms = r->gpu_range_ms = r->gpu_emit_ms = 0;
  Run run;
  run.s = s;
  run.t = t;
  run.res = r;
  for (int i = int(s->slots.size()) - 1; i >= 0; --i) run.free_slots.push_back(i);
  run.t0 = std::chrono::steady_clock::now();
  lsm_status st = s->cfg.policy == LSM_SERVE_FIXED ? run.run_fixed() : run.run_continuous();
  r->wall_us = now_us(run.t0);
  if (st == LSM_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_status(e);
  }
  return st;
}

lsm_status lsm_server_stats(const lsm_server_t* s, uint64_t* r, uint64_t* resident, uint32_t* levels,
                            uint64_t* device_bytes) {
  if (!s) return LSM_ERR_ARG;
  uint64_t rr = 0, res = 0;
  lsm_stats(s->dict, &rr, &res, nullptr, nullptr);
  if (r) *r = rr;
  if (resident) *resident = res;
  if (levels) *levels = s->L;
  if (device_bytes) *device_bytes = s->device_bytes;
  return LSM_OK;
}

lsm_t* lsm_server_dict(lsm_server_t* s) { return s ? s->dict : nullptr; }

}  // extern "C"
