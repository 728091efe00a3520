// Batch sort of the GPU LSM: a stable least-significant-digit radix sort of
// (key variable, value) pairs over all 32 bits, 8 bits per pass (§IV-A sorts
// every batch with a radix sort over the whole key variable, status bit
// included, so a tombstone precedes a regular element of the same key).
//
// Structure (one histogram kernel, then one kernel per digit):
//   * sort_histogram reads the input once and counts all four digits; in the
//     batch modes it also encodes each op as (key << 1) | status and checks
//     that keys are below 2^31 - 1.
//   * sort_pass ranks a tile of 4096 elements per CTA in shared memory, gets
//     the tile's global offset per digit from the tiles before it by
//     decoupled look-back (tile order comes from an atomic ticket, so a CTA
//     only ever waits on CTAs that already started), and scatters.
// In the batch modes the first pass reads the input back to front, padded at
// the logical end with copies of the last op; a stable sort of that sequence
// puts the last of several equal key variables first (the "last insert wins"
// reading of §III-A rule 4).
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIPT = kSortTile / kThreads;  // 16 items per thread
constexpr int kRadix = 256;
constexpr uint32_t kNoDigit = 256;
static_assert(kThreads == kRadix, "one thread per digit in the look-back");

// Look-back word: [epoch:30][flag:2][value:32].
constexpr uint64_t kFlagAgg = 1, kFlagIncl = 2;
__device__ __forceinline__ uint64_t lb_pack(uint32_t epoch, uint64_t flag, uint32_t v) {
  return (uint64_t(epoch) << 34) | (flag << 32) | v;
}

struct Loader {
  int mode;
  const uint32_t* keys;
  const uint32_t* vals;
  const uint8_t* del;
  uint64_t n_in;
  uint32_t n;

  // Element p of the logical sequence.  Batch modes: position p of the
  // reversed padded batch, i.e. op min(n - 1 - p, n_in - 1).
  __device__ __forceinline__ void load(uint32_t p, uint32_t& kv, uint32_t& v, bool& bad) const {
    bad = false;
    if (mode == kSortPairs) {
      kv = __ldg(keys + p);
      v = __ldg(vals + p);
      return;
    }
    if (mode == kSortQueries) {
      kv = __ldg(keys + p);
      v = p;
      return;
    }
    uint64_t s = uint64_t(n) - 1 - p;
    if (s >= n_in) s = n_in - 1;
    const uint32_t k = __ldg(keys + s);
    const bool is_del = (mode == kSortDelete) || (mode == kSortUpdate && __ldg(del + s) != 0);
    bad = k > kMaxUserKey;
    kv = bad ? kPlaceboKv : ((k << 1) | (is_del ? 0u : 1u));
    v = (is_del || bad) ? 0u : __ldg(vals + s);
  }

  // Key variable only (the histogram needs no values).
  __device__ __forceinline__ uint32_t load_key(uint32_t p, bool& bad) const {
    bad = false;
    if (mode == kSortPairs || mode == kSortQueries) return __ldg(keys + p);
    uint64_t s = uint64_t(n) - 1 - p;
    if (s >= n_in) s = n_in - 1;
    const uint32_t k = __ldg(keys + s);
    const bool is_del = (mode == kSortDelete) || (mode == kSortUpdate && __ldg(del + s) != 0);
    bad = k > kMaxUserKey;
    return bad ? kPlaceboKv : ((k << 1) | (is_del ? 0u : 1u));
  }
};

__global__ void __launch_bounds__(kThreads) sort_histogram(Loader ld, uint32_t* __restrict__ ctl) {
  __shared__ uint32_t s_h[kSortPasses * kRadix];
  for (int i = threadIdx.x; i < kSortPasses * kRadix; i += kThreads) s_h[i] = 0;
  __syncthreads();
  bool bad_any = false;
  for (uint32_t p = blockIdx.x * kThreads + threadIdx.x; p < ld.n; p += gridDim.x * kThreads) {
    bool bad;
    const uint32_t kv = ld.load_key(p, bad);
    bad_any |= bad;
#pragma unroll
    for (int d = 0; d < kSortPasses; ++d) atomicAdd(&s_h[d * kRadix + ((kv >> (8 * d)) & 255u)], 1u);
  }
  const int any_bad = __syncthreads_or(bad_any);
  for (int i = threadIdx.x; i < kSortPasses * kRadix; i += kThreads) {
    const uint32_t c = s_h[i];
    if (c) atomicAdd(ctl + i, c);
  }
  if (any_bad && threadIdx.x == 0) atomicOr(ctl + kSortCtlStatus, kErrBadKey);
}

template <bool kFirst>
__global__ void __launch_bounds__(kThreads) sort_pass(Loader ld, const uint32_t* __restrict__ in_k,
                                                      const uint32_t* __restrict__ in_v,
                                                      uint32_t* __restrict__ out_k,
                                                      uint32_t* __restrict__ out_v,
                                                      uint32_t* __restrict__ ctl, uint64_t* lookback,
                                                      int pass, uint32_t epoch, uint32_t* sticky) {
  __shared__ __align__(16) uint32_t s_keys[kSortTile];
  __shared__ __align__(16) uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_whist[kWarps][kRadix];
  __shared__ uint32_t s_excl[kRadix];   // tile-local start of each digit
  __shared__ uint32_t s_gbase[kRadix];  // global start of this tile's run of each digit
  __shared__ uint32_t s_scan[kWarps];
  __shared__ uint32_t s_tile;

  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t n = ld.n;
  const int shift = 8 * pass;
  if (tid == 0) s_tile = atomicAdd(ctl + kSortPasses * kRadix + pass, 1u);
  for (uint32_t i = lane; i < kRadix; i += 32) s_whist[warp][i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t base = tile * kSortTile + warp * (32 * kIPT);

  uint32_t kv[kIPT], v[kIPT], rank[kIPT];
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    kv[j] = 0;
    v[j] = 0;
    if (p < n) {
      if (kFirst) {
        bool bad;
        ld.load(p, kv[j], v[j], bad);
      } else {
        kv[j] = __ldg(in_k + p);
        v[j] = __ldg(in_v + p);
      }
    }
  }

  // Rank within the warp, items in (j, lane) order = input order.
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    const uint32_t d = (p < n) ? ((kv[j] >> shift) & 255u) : kNoDigit;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & lt);
    const uint32_t cnt = (d != kNoDigit) ? s_whist[warp][d] : 0u;
    __syncwarp();
    if (d != kNoDigit && before == 0) s_whist[warp][d] = cnt + __popc(peers);
    __syncwarp();
    rank[j] = cnt + before;
  }
  __syncthreads();

  // Per digit: warp prefix inside the tile and the tile total.
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_whist[w][tid];
    s_whist[w][tid] = total;
    total += c;
  }
  uint32_t tile_sum;
  const uint32_t excl = block_excl_scan<kThreads>(total, s_scan, tile_sum);
  s_excl[tid] = excl;
  // Global start of the digit (exclusive scan of the pass histogram).
  uint32_t hsum;
  const uint32_t hbase = block_excl_scan<kThreads>(ctl[pass * kRadix + tid], s_scan, hsum);

  // Decoupled look-back over the tiles before this one, one digit per thread.
  uint64_t* my = lookback + uint64_t(tile) * kRadix + tid;
  uint32_t prefix = 0;
  if (tile == 0) {
    st_relaxed_u64(my, lb_pack(epoch, kFlagIncl, total));
  } else {
    st_relaxed_u64(my, lb_pack(epoch, kFlagAgg, total));
    int64_t t = int64_t(tile) - 1;
    uint64_t t0 = 0;
    while (t >= 0) {
      const uint64_t w = ld_relaxed_u64(lookback + uint64_t(t) * kRadix + tid);
      const uint64_t flag = (w >> 32) & 3u;
      if (uint32_t(w >> 34) != epoch || flag == 0) {
        if (t0 == 0) t0 = globaltimer_ns();
        else if (globaltimer_ns() - t0 > kWaitLimitNs) {
          atomicOr(sticky, kErrTimeout);
          break;
        }
        continue;
      }
      prefix += uint32_t(w);
      if (flag == kFlagIncl) break;
      --t;
    }
    st_relaxed_u64(my, lb_pack(epoch, kFlagIncl, prefix + total));
  }
  s_gbase[tid] = hbase + prefix;
  __syncthreads();

  // Scatter into shared memory in digit order (stable), then write out.
#pragma unroll
  for (int j = 0; j < kIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    if (p < n) {
      const uint32_t d = (kv[j] >> shift) & 255u;
      const uint32_t pos = s_excl[d] + s_whist[warp][d] + rank[j];
      s_keys[pos] = kv[j];
      s_vals[pos] = v[j];
    }
  }
  __syncthreads();
  const uint32_t tile_start = tile * kSortTile;
  const uint32_t tile_n = (n - tile_start) < uint32_t(kSortTile) ? (n - tile_start) : uint32_t(kSortTile);
  for (uint32_t i = tid; i < tile_n; i += kThreads) {
    const uint32_t k = s_keys[i];
    const uint32_t d = (k >> shift) & 255u;
    const uint32_t dst = s_gbase[d] + (i - s_excl[d]);
    if (dst < n) {
      out_k[dst] = k;
      out_v[dst] = s_vals[i];
    }
  }
}

__global__ void __launch_bounds__(256) check_keys(const uint32_t* __restrict__ keys, uint64_t n,
                                                  uint32_t* status) {
  bool bad = false;
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += uint64_t(gridDim.x) * 256ull)
    bad |= __ldg(keys + i) > kMaxUserKey;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kErrBadKey);
}

}  // namespace

cudaError_t sort_launch(const SortArgs& a, SortWorkspace& ws, cudaStream_t st, uint32_t* h_status,
                        cudaEvent_t ev) {
  if (a.n == 0) return cudaSuccess;
  const uint32_t ntiles = (a.n + kSortTile - 1) / kSortTile;
  if (ntiles > ws.max_tiles) return cudaErrorInvalidValue;
  cudaError_t e;
  if (++ws.epoch >= (1u << 30)) {
    ws.epoch = 1;
    e = cudaMemsetAsync(ws.lookback, 0, sizeof(uint64_t) * kSortPasses * ws.max_tiles * kRadix, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(ws.ctl, 0, sizeof(uint32_t) * kSortCtlWords, st);
  if (e != cudaSuccess) return e;
  Loader ld{a.mode, a.in_keys, a.in_vals, a.in_del, a.n_in, a.n};
  uint32_t hblocks = (a.n + 255) / 256;
  if (hblocks > 4 * 152) hblocks = 4 * 152;
  count_launches(1);
  sort_histogram<<<hblocks, 256, 0, st>>>(ld, ws.ctl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (h_status) {
    e = cudaMemcpyAsync(h_status, ws.ctl + kSortCtlStatus, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev, st)) != cudaSuccess) return e;
  }
  // in -> tmp -> out -> tmp -> out
  uint32_t* bk[2] = {a.tmp_keys, a.out_keys};
  uint32_t* bv[2] = {a.tmp_vals, a.out_vals};
  const size_t lb_stride = size_t(ws.max_tiles) * kRadix;
  count_launches(1);
  sort_pass<true><<<ntiles, kThreads, 0, st>>>(ld, nullptr, nullptr, bk[0], bv[0], ws.ctl, ws.lookback,
                                                0, ws.epoch, ws.sticky);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int p = 1; p < kSortPasses; ++p) {
    count_launches(1);
    sort_pass<false><<<ntiles, kThreads, 0, st>>>(ld, bk[(p - 1) & 1], bv[(p - 1) & 1], bk[p & 1],
                                                   bv[p & 1], ws.ctl, ws.lookback + p * lb_stride, p,
                                                   ws.epoch, ws.sticky);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t check_keys_launch(const uint32_t* keys, uint64_t n, uint32_t* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 8 * 152) blocks = 8 * 152;
  count_launches(1);
  check_keys<<<unsigned(blocks), 256, 0, st>>>(keys, n, status);
  return cudaGetLastError();
}

}  // namespace gpulsm

// ---------------------------------------------------------------------------
// Allocation-free batch sort (lsm_sort_pairs_noalloc in gpulsm.h).
//
// Some callers may not allocate device memory once they are running: a
// process whose memory is handed out by its own pool allocator and forbids
// raw cudaMalloc, or a latency-bound loop that cannot afford the implicit
// device-wide synchronisation and the unbounded time a cudaMalloc/cudaFree
// may take.  For them the sort below takes all of its scratch (ping-pong
// buffers, histograms, look-back words) from one fixed array with static
// storage in this file, which every GPU that loads the library holds until
// the process exits.  Its size is set by kNoAllocMaxPairs.
// ---------------------------------------------------------------------------
#include <mutex>

#include "gpulsm.h"

namespace gpulsm {
namespace {

constexpr uint32_t kNoAllocMaxPairs = LSM_SORT_NOALLOC_MAX_PAIRS;
constexpr uint32_t kNoAllocTiles = (kNoAllocMaxPairs + kSortTile - 1) / kSortTile;
constexpr size_t kNoAllocCtl = 1088;                    // >= kSortCtlWords, multiple of 64
constexpr size_t kNoAllocSticky = kNoAllocCtl - 1;      // last ctl word: wait timeouts
constexpr size_t kNoAllocTmpK = kNoAllocCtl;
constexpr size_t kNoAllocTmpV = kNoAllocTmpK + kNoAllocMaxPairs;
constexpr size_t kNoAllocLookback = kNoAllocTmpV + kNoAllocMaxPairs;   // u64 words from here
constexpr size_t kNoAllocLookbackWords = size_t(kSortPasses) * kNoAllocTiles * 256;
constexpr size_t kNoAllocWords = kNoAllocLookback + 2 * kNoAllocLookbackWords;
static_assert(kNoAllocCtl > size_t(kSortCtlWords), "control block fits");
static_assert(kNoAllocLookback % 2 == 0, "look-back words 8-byte aligned");

// The scratch itself: about 10.5 MB for kNoAllocMaxPairs = 2^20.
static __device__ __align__(256) uint32_t g_sort_scratch[kNoAllocWords];

constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
  uint32_t* base = nullptr;  // device address of g_sort_scratch on this device
  SortWorkspace ws{};
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[kNoAllocMaxDevices];

}  // namespace
}  // namespace gpulsm

extern "C" lsm_status lsm_sort_pairs_noalloc(const uint32_t* d_keys_in, const uint32_t* d_vals_in,
                                             uint32_t* d_keys_out, uint32_t* d_vals_out, uint64_t n,
                                             void* stream) {
  using namespace gpulsm;
  if (n > kNoAllocMaxPairs) return LSM_ERR_CAPACITY;
  if (n && (!d_keys_in || !d_vals_in || !d_keys_out || !d_vals_out)) return LSM_ERR_ARG;
  if (n == 0) return LSM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return LSM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc[dev];
  if (!d.base) {
    // Once per device, with that device current: the host needs the array's
    // device address (its name in host code is only a host-side stand-in),
    // and the look-back words must start at zero.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LSM_ERR_CUDA;
    }
    uint32_t* base = static_cast<uint32_t*>(p);
    if (cudaMemsetAsync(base, 0, kNoAllocWords * sizeof(uint32_t), st) != cudaSuccess) {
      cudaGetLastError();
      return LSM_ERR_CUDA;
    }
    d.ws.ctl = base;
    d.ws.lookback = reinterpret_cast<uint64_t*>(base + kNoAllocLookback);
    d.ws.max_tiles = kNoAllocTiles;
    d.ws.epoch = 0;
    d.ws.sticky = base + kNoAllocSticky;
    d.base = base;
  }
  SortArgs a{};
  a.mode = kSortPairs;
  a.in_keys = d_keys_in;
  a.in_vals = d_vals_in;
  a.n_in = n;
  a.n = uint32_t(n);
  a.out_keys = d_keys_out;
  a.out_vals = d_vals_out;
  a.tmp_keys = d.base + kNoAllocTmpK;
  a.tmp_vals = d.base + kNoAllocTmpV;
  // sort_launch clears the histogram/counter block itself on every call and
  // tags look-back words with a per-call epoch, so nothing else needs zeroing.
  cudaError_t e = sort_launch(a, d.ws, st, nullptr, nullptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LSM_ERR_CUDA;
  }
  return LSM_OK;
}
