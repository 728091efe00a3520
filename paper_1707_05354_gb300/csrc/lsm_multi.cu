// Host side of the batched form (include/gpulsm.h, lsm_multi_*): many
// independent GPU LSMs (§III) with their own batch sizes, advanced together
// one round at a time.
//
// Every instance keeps its own binary counter r_i on the device; a round's
// kernels read it, so the host never needs to know which level a fold fills
// and one captured CUDA graph replays every round.  The launch shapes depend
// only on the instances' sizes (fixed at creation): sort tiles and buckets
// are counted statically, the partition and the merge are persistent and
// take their work counts from the prep kernel.
#include <cstring>
#include <new>
#include <vector>

#include "gpulsm.h"
#include "lsm_kernels.h"

using namespace gpulsm;

namespace {

uint64_t rup(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  uint64_t kernels = 0;  // kernel nodes per replay
  uint64_t used = 0;     // last use (LRU)
  // arguments the graph was captured with
  const void* args[9] = {};
  uint64_t nq = 0;
};
constexpr size_t kMaxGraphs = 64;  // captured rounds kept (one per distinct argument set)

}  // namespace

struct lsm_multi_t {
  int device = 0;
  uint32_t n = 0;
  std::vector<MultiInst> inst;
  MultiArena ar{};
  // allocations
  MultiInst* d_inst = nullptr;
  uint64_t* d_prefix = nullptr;  // stile_prefix, bucket_prefix, tile_prefix, part_prefix (n + 1 each)
  uint32_t *d_keys = nullptr, *d_vals = nullptr, *d_bk = nullptr, *d_bv = nullptr, *d_tk = nullptr,
           *d_tv = nullptr, *d_fence = nullptr, *d_tilecnt = nullptr, *d_bucket = nullptr, *d_part = nullptr,
           *d_state = nullptr;  // r, k, badkey, flags (n each), work_ctr, status
  uint64_t level_words = 0, batch_words = 0;
  bool use_graph = true;
  uint64_t device_bytes = 0;
  cudaStream_t cap = nullptr;  // private capture stream
  std::vector<GraphSlot> graphs;  // LRU cache of captured rounds
  uint64_t graph_clock = 0;
  uint64_t last_kernels = 0;
};

namespace {

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

template <typename T>
cudaError_t dalloc(T** p, uint64_t count) {
  const cudaError_t g = alloc_gate();
  if (g != cudaSuccess) return g;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

void drop_graph(GraphSlot& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g = GraphSlot{};
}

void free_all(lsm_multi_t* h) {
  for (auto& g : h->graphs) drop_graph(g);
  h->graphs.clear();
  void* p[] = {h->d_inst, h->d_prefix, h->d_keys, h->d_vals, h->d_bk,      h->d_bv,   h->d_tk,
               h->d_tv,   h->d_fence,  h->d_tilecnt, h->d_bucket, h->d_part, h->d_state};
  for (void* q : p)
    if (q) cudaFree(q);
  if (h->cap) cudaStreamDestroy(h->cap);
}

int ceil_log2(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

// Everything a round enqueues: the update kernels and, when nq > 0, the
// lookups (which see the round's batches).
cudaError_t enqueue_round(lsm_multi_t* h, const MultiBatch& in, const uint32_t* q, const uint64_t* qoff,
                          uint64_t nq, uint32_t* val, uint8_t* found, cudaStream_t st) {
  cudaError_t e = multi_update_launch(h->ar, in, st);
  if (e != cudaSuccess || nq == 0) return e;
  return multi_lookup_launch(h->ar, q, qoff, nq, val, found, st);
}

// Runs a round through a graph captured on the private stream with these
// exact arguments (one cached graph per distinct argument set, least
// recently used dropped beyond kMaxGraphs), ordered after the work already on
// `st` and before whatever follows it there.
lsm_status run_round(lsm_multi_t* h, int kind, const MultiBatch& in, const uint32_t* q, const uint64_t* qoff,
                     uint64_t nq, uint32_t* val, uint8_t* found, cudaStream_t st) {
  if (!h->use_graph) return cuda_status(enqueue_round(h, in, q, qoff, nq, val, found, st));
  const void* args[9] = {in.keys, in.vals, in.del, in.counts, q, qoff, val, found,
                         reinterpret_cast<const void*>(uintptr_t(kind))};
  GraphSlot* g = nullptr;
  for (auto& s : h->graphs)
    if (s.nq == nq && memcmp(args, s.args, sizeof(args)) == 0) g = &s;
  if (!g) {
    if (h->graphs.size() >= kMaxGraphs) {
      size_t lru = 0;
      for (size_t j = 1; j < h->graphs.size(); ++j)
        if (h->graphs[j].used < h->graphs[lru].used) lru = j;
      drop_graph(h->graphs[lru]);
      h->graphs.erase(h->graphs.begin() + lru);
    }
    GraphSlot ns;
    const uint64_t before = launches_so_far();
    LSM_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_round(h, in, q, qoff, nq, val, found, h->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ns.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    ns.kernels = launches_so_far() - before;
    count_launches(0ull - ns.kernels);  // captured, not launched
    if (e != cudaSuccess) return cuda_status(e);
    memcpy(ns.args, args, sizeof(args));
    ns.nq = nq;
    h->graphs.push_back(ns);
    g = &h->graphs.back();
  }
  g->used = ++h->graph_clock;
  h->last_kernels = g->kernels;
  count_launches(g->kernels);
  return cuda_status(cudaGraphLaunch(g->exec, st));
}

}  // namespace

extern "C" {

lsm_status lsm_multi_create(lsm_multi_t** out, uint32_t n_inst, const uint32_t* h_b, uint32_t max_batches,
                            const lsm_multi_tuning* h_tuning, int device) {
  if (!out || n_inst == 0 || !h_b || max_batches == 0) return LSM_ERR_ARG;
  *out = nullptr;
  int L = 0;
  while ((1ull << L) <= max_batches) ++L;  // r <= max_batches needs bits 0 .. L - 1
  if (L > kMultiMaxLevels) return LSM_ERR_ARG;
  std::vector<MultiInst> inst(n_inst);
  std::vector<uint64_t> stp(n_inst + 1, 0), bkp(n_inst + 1, 0);
  uint64_t in_off = 0, boff = 0, loff = 0, foff = 0, part_words = 0;
  for (uint32_t i = 0; i < n_inst; ++i) {
    const uint32_t b = h_b[i];
    if (b == 0 || b > kMultiMaxB || (uint64_t(b) << (L - 1)) >= (1ull << 31)) return LSM_ERR_ARG;
    uint32_t tile = kFoldTile, e = 3;
    if (h_tuning) {
      tile = h_tuning[i].tile;
      e = h_tuning[i].bin_log2;
      if ((tile != 1024 && tile != 2048) || e < 1 || e > 6) return LSM_ERR_ARG;
    }
    MultiInst& d = inst[i];
    memset(&d, 0, sizeof(d));
    d.in_off = in_off;
    in_off += b;
    d.boff = boff;
    boff += rup(uint64_t(b) + kSlack, kLevelAlign);
    d.b = b;
    d.levels = uint32_t(L);
    int msd = ceil_log2((uint64_t(b) + kMultiSortTile - 1) / kMultiSortTile);
    d.msd_bits = uint32_t(msd < 1 ? 1 : (msd > 8 ? 8 : msd));
    d.tile = tile;
    d.stile0 = uint32_t(stp[i]);
    stp[i + 1] = stp[i] + (b + kMultiSortTile - 1) / kMultiSortTile;
    d.bucket0 = uint32_t(bkp[i]);
    bkp[i + 1] = bkp[i] + (1ull << d.msd_bits);
    for (int l = 0; l < L; ++l) {
      const uint64_t nl = uint64_t(b) << l;
      d.lvl_off[l] = loff;
      loff += rup(nl + kSlack, kLevelAlign);
      d.lvl_fshift[l] = fence_shift_for(nl, int(e), 8);
      d.lvl_fence[l] = foff;
      foff += rup(fence_words(d.lvl_fshift[l]), 64);
    }
    d.fshift0 = d.lvl_fshift[0];
    if (32 - int(d.msd_bits) < d.fshift0) return LSM_ERR_ARG;  // a bucket spans whole bins
    d.batch_fence = foff;
    foff += rup(fence_words(d.fshift0), 64);
    part_words += ((uint64_t(b) << (L - 1)) + tile - 1) / tile + 1;
  }
  if (stp[n_inst] >= (1ull << 31) || bkp[n_inst] >= (1ull << 31)) return LSM_ERR_ARG;

  DeviceGuard g(device);
  lsm_multi_t* h = new (std::nothrow) lsm_multi_t();
  if (!h) return LSM_ERR_OOM;
  h->device = device;
  h->n = n_inst;
  h->inst = inst;
  h->level_words = loff;
  h->batch_words = boff;
  const uint64_t stiles = stp[n_inst], buckets = bkp[n_inst];
  const uint64_t state_words = 4ull * n_inst + 8;
  h->device_bytes = sizeof(MultiInst) * n_inst + 32ull * (n_inst + 1) + 8 * loff + 16 * boff + 4 * foff +
                    4 * stiles * 512 + 8 * buckets + 4 * part_words * kMultiPartStride + 4 * state_words;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&h->d_inst, n_inst);
  if (e == cudaSuccess) e = dalloc(&h->d_prefix, 4ull * (n_inst + 1));
  if (e == cudaSuccess) e = dalloc(&h->d_keys, loff);
  if (e == cudaSuccess) e = dalloc(&h->d_vals, loff);
  if (e == cudaSuccess) e = dalloc(&h->d_bk, boff);
  if (e == cudaSuccess) e = dalloc(&h->d_bv, boff);
  if (e == cudaSuccess) e = dalloc(&h->d_tk, boff);
  if (e == cudaSuccess) e = dalloc(&h->d_tv, boff);
  if (e == cudaSuccess) e = dalloc(&h->d_fence, foff);
  if (e == cudaSuccess) e = dalloc(&h->d_tilecnt, stiles * 512);
  if (e == cudaSuccess) e = dalloc(&h->d_bucket, 2 * buckets);
  if (e == cudaSuccess) e = dalloc(&h->d_part, part_words * kMultiPartStride);
  if (e == cudaSuccess) e = dalloc(&h->d_state, state_words);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_inst, inst.data(), sizeof(MultiInst) * n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->d_prefix, stp.data(), 8 * (n_inst + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_prefix + (n_inst + 1), bkp.data(), 8 * (n_inst + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_prefix + 2 * (n_inst + 1), 0, 16 * (n_inst + 1));
  if (e == cudaSuccess) e = cudaMemset(h->d_keys, 0, 4 * loff);
  if (e == cudaSuccess) e = cudaMemset(h->d_vals, 0, 4 * loff);
  if (e == cudaSuccess) e = cudaMemset(h->d_bk, 0, 4 * boff);
  if (e == cudaSuccess) e = cudaMemset(h->d_bv, 0, 4 * boff);
  if (e == cudaSuccess) e = cudaMemset(h->d_state, 0, 4 * state_words);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = multi_prepare_kernels();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return cuda_status(e);
  }
  MultiArena& a = h->ar;
  a.inst = h->d_inst;
  a.n = n_inst;
  a.keys = h->d_keys;
  a.vals = h->d_vals;
  a.bkeys = h->d_bk;
  a.bvals = h->d_bv;
  a.tkeys = h->d_tk;
  a.tvals = h->d_tv;
  a.fence = h->d_fence;
  a.stile_prefix = h->d_prefix;
  a.bucket_prefix = h->d_prefix + (n_inst + 1);
  a.tile_prefix = h->d_prefix + 2 * (n_inst + 1);
  a.part_prefix = h->d_prefix + 3 * (n_inst + 1);
  a.total_stiles = stiles;
  a.total_buckets = buckets;
  a.tilecnt = h->d_tilecnt;
  a.bstart = h->d_bucket;
  a.bcnt = h->d_bucket + buckets;
  a.r = h->d_state;
  a.k = reinterpret_cast<int32_t*>(h->d_state + n_inst);
  a.badkey = h->d_state + 2 * n_inst;
  a.flags = h->d_state + 3 * n_inst;
  a.work_ctr = h->d_state + 4 * n_inst;
  a.status = h->d_state + 4 * n_inst + 1;
  a.part = h->d_part;
  *out = h;
  return LSM_OK;
}

void lsm_multi_destroy(lsm_multi_t* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

lsm_status lsm_multi_update(lsm_multi_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                            const uint8_t* d_is_delete, const uint32_t* d_counts, void* stream) {
  if (!h || !d_keys) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  const MultiBatch in{d_keys, d_vals, d_is_delete, d_counts};
  return run_round(h, 0, in, nullptr, nullptr, 0, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

lsm_status lsm_multi_lookup(lsm_multi_t* h, const uint32_t* d_q, const uint64_t* d_qoff, uint64_t nq,
                            uint32_t* d_val, uint8_t* d_found, void* stream) {
  if (!h || (nq && (!d_q || !d_qoff || !d_val || !d_found))) return LSM_ERR_ARG;
  if (nq == 0) return LSM_OK;
  DeviceGuard g(h->device);
  return cuda_status(multi_lookup_launch(h->ar, d_q, d_qoff, nq, d_val, d_found, static_cast<cudaStream_t>(stream)));
}

lsm_status lsm_multi_round(lsm_multi_t* h, const uint32_t* d_keys, const uint32_t* d_vals,
                           const uint8_t* d_is_delete, const uint32_t* d_counts, const uint32_t* d_q,
                           const uint64_t* d_qoff, uint64_t nq, uint32_t* d_val, uint8_t* d_found, void* stream) {
  if (!h || !d_keys) return LSM_ERR_ARG;
  if (nq && (!d_q || !d_qoff || !d_val || !d_found)) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  const MultiBatch in{d_keys, d_vals, d_is_delete, d_counts};
  return run_round(h, 1, in, d_q, d_qoff, nq, d_val, d_found, static_cast<cudaStream_t>(stream));
}

lsm_status lsm_multi_sync(lsm_multi_t* h, void* stream, uint32_t* h_flags) {
  if (!h) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LSM_TRY(cudaStreamSynchronize(st));
  uint32_t status = 0;
  LSM_TRY(cudaMemcpy(&status, h->ar.status, 4, cudaMemcpyDeviceToHost));
  if (h_flags) LSM_TRY(cudaMemcpy(h_flags, h->ar.flags, 4ull * h->n, cudaMemcpyDeviceToHost));
  if (status) LSM_TRY(cudaMemset(h->ar.status, 0, 4));
  if (status & kErrTimeout) return LSM_ERR_TIMEOUT;
  if (status & kErrAlign) return LSM_ERR_CUDA;
  if (status & kErrBadKey) return LSM_ERR_KEY_RANGE;
  if (status & kErrArg) return LSM_ERR_ARG;
  if (status & kErrFull) return LSM_ERR_FULL;
  return LSM_OK;
}

lsm_status lsm_multi_stats(const lsm_multi_t* h, uint32_t i, uint64_t* r, uint32_t* b, uint64_t* resident) {
  if (!h || i >= h->n) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  uint32_t rr = 0;
  LSM_TRY(cudaMemcpy(&rr, h->ar.r + i, 4, cudaMemcpyDeviceToHost));
  if (r) *r = rr;
  if (b) *b = h->inst[i].b;
  if (resident) *resident = uint64_t(rr) * h->inst[i].b;
  return LSM_OK;
}

lsm_status lsm_multi_layout(const lsm_multi_t* h, uint32_t i, uint64_t* in_off, uint32_t* tile,
                            int32_t* fence_shift0, uint32_t* levels) {
  if (!h || i >= h->n) return LSM_ERR_ARG;
  const MultiInst& d = h->inst[i];
  if (in_off) *in_off = d.in_off;
  if (tile) *tile = d.tile;
  if (fence_shift0) *fence_shift0 = d.fshift0;
  if (levels) *levels = d.levels;
  return LSM_OK;
}

lsm_status lsm_multi_dump_levels(const lsm_multi_t* h, uint32_t i, uint32_t* h_keys, uint32_t* h_vals) {
  if (!h || i >= h->n || !h_keys || !h_vals) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  uint32_t rr = 0;
  LSM_TRY(cudaDeviceSynchronize());
  LSM_TRY(cudaMemcpy(&rr, h->ar.r + i, 4, cudaMemcpyDeviceToHost));
  const MultiInst& d = h->inst[i];
  uint64_t pos = 0;
  for (uint32_t l = 0; l < d.levels; ++l) {
    if (!((rr >> l) & 1u)) continue;
    const uint64_t nl = uint64_t(d.b) << l;
    LSM_TRY(cudaMemcpy(h_keys + pos, h->d_keys + d.lvl_off[l], 4 * nl, cudaMemcpyDeviceToHost));
    LSM_TRY(cudaMemcpy(h_vals + pos, h->d_vals + d.lvl_off[l], 4 * nl, cudaMemcpyDeviceToHost));
    pos += nl;
  }
  return LSM_OK;
}

lsm_status lsm_multi_reset(lsm_multi_t* h, void* stream) {
  if (!h) return LSM_ERR_ARG;
  DeviceGuard g(h->device);
  // r = 0 empties every level; flags and the bad-key marks start clean
  return cuda_status(cudaMemsetAsync(h->d_state, 0, 4ull * 4 * h->n, static_cast<cudaStream_t>(stream)));
}

lsm_status lsm_multi_set_option(lsm_multi_t* h, int opt, int64_t value) {
  if (!h) return LSM_ERR_ARG;
  if (opt == LSM_MULTI_OPT_GRAPH) {
    h->use_graph = value != 0;
    return LSM_OK;
  }
  return LSM_ERR_ARG;
}

lsm_status lsm_multi_get_option(const lsm_multi_t* h, int opt, int64_t* value) {
  if (!h || !value) return LSM_ERR_ARG;
  if (opt == LSM_MULTI_OPT_GRAPH) {
    *value = h->use_graph ? 1 : 0;
    return LSM_OK;
  }
  if (opt == LSM_MULTI_OPT_GRAPH_KERNELS) {
    *value = int64_t(h->last_kernels);
    return LSM_OK;
  }
  if (opt == LSM_MULTI_OPT_DEVICE_BYTES) {
    *value = int64_t(h->device_bytes);
    return LSM_OK;
  }
  return LSM_ERR_ARG;
}

}  // extern "C"
