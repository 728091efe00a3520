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
constexpr int kLookbackWindow = LSM_SORT_LBW;
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
    // the key, delete flag and value loads are independent (insert and
    // update calls always pass values), so they are in flight together
    const uint32_t k = __ldg(keys + s);
    const uint32_t v0 = mode != kSortDelete ? __ldg(vals + s) : 0u;
    const bool is_del = (mode == kSortDelete) || (mode == kSortUpdate && __ldg(del + s) != 0);
    bad = k > kMaxUserKey;
    kv = bad ? kPlaceboKv : ((k << 1) | (is_del ? 0u : 1u));
    v = (is_del || bad) ? 0u : v0;
  }

  // Leading positions of the reversed padded batch that are padding (copies
  // of op n_in - 1); 0 outside the batch modes.
  __device__ __forceinline__ uint32_t npad() const {
    if (mode == kSortPairs || mode == kSortQueries) return 0u;
    return uint64_t(n) > n_in ? uint32_t(uint64_t(n) - n_in) : 0u;
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

__global__ void __launch_bounds__(kThreads) sort_histogram(Loader ld, uint32_t* __restrict__ ctl,
                                                           uint32_t* status) {
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
  if (any_bad && threadIdx.x == 0 && status) *reinterpret_cast<volatile uint32_t*>(status) = kErrBadKey;
}

template <bool kFirst>
__global__ void __launch_bounds__(kThreads, LSM_SORT_MINB) sort_pass(Loader ld, const uint32_t* __restrict__ in_k,
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
    const uint32_t peers = warp_peers<9>(d);  // d <= kNoDigit = 256
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

  // Scatter into shared memory in digit order (stable) while the look-back
  // below is still to come: the item registers are free afterwards.
  __syncthreads();
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

  // Decoupled look-back over the tiles before this one, one digit per
  // thread, reading kLookbackWindow predecessors per step: the words are
  // consumed from the nearest tile down until an inclusive prefix is found;
  // a word not yet published stops the step, which is then retried from
  // there (bounded in time).
  uint64_t* my = lookback + uint64_t(tile) * kRadix + tid;
  uint32_t prefix = 0;
  if (tile == 0) {
    st_relaxed_u64(my, lb_pack(epoch, kFlagIncl, total));
  } else {
    st_relaxed_u64(my, lb_pack(epoch, kFlagAgg, total));
    int64_t t = int64_t(tile) - 1;
    uint64_t t0 = 0;
    bool done = false;
    while (!done) {
      uint64_t w[kLookbackWindow];
#pragma unroll
      for (int i = 0; i < kLookbackWindow; ++i)
        w[i] = (t - i >= 0) ? ld_relaxed_u64(lookback + uint64_t(t - i) * kRadix + tid) : 0ull;
      int consumed = 0;
      bool stall = false;
#pragma unroll
      for (int i = 0; i < kLookbackWindow; ++i) {
        if (done || stall) continue;
        if (t - i < 0) {  // ran past tile 0: the prefix is complete
          done = true;
          continue;
        }
        const uint64_t flag = (w[i] >> 32) & 3u;
        if (uint32_t(w[i] >> 34) != epoch || flag == 0) {
          stall = true;
          continue;
        }
        prefix += uint32_t(w[i]);
        ++consumed;
        if (flag == kFlagIncl) done = true;
      }
      t -= consumed;
      if (!done && consumed == 0 && !spin_continue(t0, kWaitLimitNs, sticky)) break;
    }
    st_relaxed_u64(my, lb_pack(epoch, kFlagIncl, prefix + total));
  }
  s_gbase[tid] = hbase + prefix;
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

// ---------------------------------------------------------------------------
// Bucket sort for n <= kMsdMaxN (the batch sizes of the plain form): the top
// byte of the key variable first, then the low 24 bits inside each bucket.
// Two kernels, so that a batch sort is one dependent launch after another:
//   msd_tile     per 4096-element tile of the (encoded, reversed) input: the
//                tile stably sorted by its top byte in shared memory and
//                written back to the scratch at the tile's own place (one
//                coalesced write), so bucket d's elements of tile t form the
//                run runs[d][t] = (start, count) there; the grand total of
//                each bucket (global atomics) and the key check.
//   bucket_sort  per bucket, one CTA: the bucket's runs, in tile order (the
//                stable order), gathered into shared memory -- the start of
//                the bucket in the output is the sum of the totals before
//                it, so no tile waits for another -- then sorted on bits
//                0..23 and written out with the prefix index entries of its
//                256 bins.  A bucket above kBucketCap elements (heavy
//                duplicate keys) is gathered into the spill area and sorted
//                by the same CTA in chunks through global memory, still
//                stably.
// ---------------------------------------------------------------------------
constexpr int kBucketThreads = 512;
constexpr int kBucketWarps = kBucketThreads / 32;
constexpr int kBucketIPT = 10;
constexpr uint32_t kBucketCap = kBucketThreads * kBucketIPT;  // 5120
constexpr uint32_t kSubBins = 4096;      // counting pass of the bucket fast path
constexpr uint32_t kSubBinMax = 48;      // larger sub-bins take the pass-by-pass path

// The tile kernel runs 512 threads of 8 elements per 4096-element tile:
// many warps to keep loads in flight, and a short ranking chain per warp.
constexpr int kScatterThreads = 512;
constexpr int kScatterWarps = kScatterThreads / 32;
constexpr int kScatterIPT = int(kMsdTile) / kScatterThreads;  // 8
static_assert(kScatterIPT * kScatterThreads == int(kMsdTile), "tile");
static_assert(kMsdMaxTiles <= uint32_t(kBucketThreads), "one thread per tile run in the bucket kernel");

// Start of bucket d in the output: the sum of the totals of the buckets
// before it (every thread of the block gets it).
template <int NT>
__device__ __forceinline__ uint32_t bucket_start(const uint32_t* ctl, uint32_t d, uint32_t* s_scan) {
  uint32_t x = 0;
  for (uint32_t i = threadIdx.x; i < kRadix; i += NT)
    if (i < d) x += ctl[3 * kRadix + i];
  uint32_t tot;
  block_excl_scan<NT>(x, s_scan, tot);
  return tot;
}

// Stable in-shared-memory rank of up to IPT items per thread of a warp-striped
// block (item j of lane l of warp w is element w*32*IPT + j*32 + l): on return
// s_whist[w][d] holds warp w's start inside digit d's run, s_excl[d] the run's
// start, and rank[j] the item's position among its warp's items of its digit.
template <int NT, int IPT>
__device__ __forceinline__ void rank_block(const uint32_t (&kv)[IPT], uint32_t m, uint32_t base, int shift,
                                           uint32_t (&rank)[IPT], uint32_t (*s_whist)[kRadix],
                                           uint32_t* s_excl, uint32_t* s_scan, uint32_t* digit_total,
                                           uint32_t lo = 0) {
  constexpr int NW = NT / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  for (uint32_t i = lane; i < kRadix; i += 32) s_whist[warp][i] = 0;
  __syncwarp();
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    const uint32_t d = (p < m && p >= lo) ? ((kv[j] >> shift) & 255u) : kNoDigit;
    const uint32_t peers = warp_peers<9>(d);  // d <= kNoDigit = 256
    const uint32_t before = __popc(peers & lt);
    const uint32_t cnt = (d != kNoDigit) ? s_whist[warp][d] : 0u;
    __syncwarp();
    if (d != kNoDigit && before == 0) s_whist[warp][d] = cnt + __popc(peers);
    __syncwarp();
    rank[j] = cnt + before;
  }
  __syncthreads();
  uint32_t total = 0;
  if (tid < kRadix) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = s_whist[w][tid];
      s_whist[w][tid] = total;
      total += c;
    }
  }
  uint32_t all;
  const uint32_t excl = block_excl_scan<NT>(tid < kRadix ? total : 0u, s_scan, all);
  if (tid < kRadix) {
    s_excl[tid] = excl;
    if (digit_total) digit_total[tid] = total;
  }
  __syncthreads();
}

// The padding of a short batch (copies of its last op, the leading
// positions of the reversed sequence) is neither ranked nor written: it is
// one run of equal elements, added to its bucket's total here and written by
// that bucket's sort at its sorted place.  A tile of padding only still
// writes its (empty) runs.
__global__ void __launch_bounds__(kScatterThreads) msd_tile(Loader ld, uint32_t* __restrict__ tmp_k,
                                                     uint32_t* __restrict__ tmp_v, uint2* __restrict__ runs,
                                                     uint32_t* __restrict__ ctl, uint32_t* status) {
  __shared__ __align__(16) uint32_t s_keys[kMsdTile];
  __shared__ __align__(16) uint32_t s_vals[kMsdTile];
  __shared__ uint32_t s_whist[kScatterWarps][kRadix];
  __shared__ uint32_t s_excl[kRadix], s_cnt[kRadix], s_scan[kScatterWarps];
  pdl_trigger();
  pdl_wait();
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, tile = blockIdx.x;
  const uint32_t n = ld.n, npad = ld.npad();
  const uint32_t t0 = tile * kMsdTile;
  const uint32_t base = t0 + warp * (32 * kScatterIPT);
  uint32_t kv[kScatterIPT], v[kScatterIPT], rank[kScatterIPT];
  bool bad_any = false;
#pragma unroll
  for (int j = 0; j < kScatterIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    kv[j] = 0;
    v[j] = 0;
    if (p < n && p >= npad) {
      bool bad;
      ld.load(p, kv[j], v[j], bad);
      bad_any |= bad;
    }
  }
  rank_block<kScatterThreads, kScatterIPT>(kv, n, base, 24, rank, s_whist, s_excl, s_scan, s_cnt, npad);
#pragma unroll
  for (int j = 0; j < kScatterIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    if (p < n && p >= npad) {
      const uint32_t d = kv[j] >> 24;
      const uint32_t pos = s_excl[d] + s_whist[warp][d] + rank[j];
      s_keys[pos] = kv[j];
      s_vals[pos] = v[j];
    }
  }
  const int any_bad = __syncthreads_or(bad_any);  // also orders the writes above before the reads below
  const uint32_t lo_t = t0 > npad ? t0 : npad, hi_t = (n - t0) < kMsdTile ? n : t0 + kMsdTile;
  const uint32_t tile_n = hi_t > lo_t ? hi_t - lo_t : 0u;  // real elements of the tile
  for (uint32_t i = tid; i < tile_n; i += kScatterThreads) {
    tmp_k[t0 + i] = s_keys[i];
    tmp_v[t0 + i] = s_vals[i];
  }
  if (tid < kRadix) {
    const uint32_t c = s_cnt[tid];
    runs[tid * kMsdMaxTiles + tile] = make_uint2(t0 + s_excl[tid], c);
    if (c) atomicAdd(ctl + 3 * kRadix + tid, c);
  }
  if (tile == 0 && tid == 0 && npad) {
    bool bad;
    atomicAdd(ctl + 3 * kRadix + (ld.load_key(0, bad) >> 24), npad);
  }
  if (any_bad && tid == 0 && status) *reinterpret_cast<volatile uint32_t*>(status) = kErrBadKey;
}

// First position i in [0, m) with (a[i] >> fshift) >= bin, a sorted.
__device__ __forceinline__ uint32_t lower_bound_bin(const uint32_t* a, uint32_t m, uint32_t bin, int fshift) {
  uint32_t lo = 0, hi = m;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((a[mid] >> fshift) < bin) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Prefix-index entries of bins [bin0, bin0 + nbins) from the sorted run
// a[0, m) that starts at position start and holds exactly those bins.
__device__ __forceinline__ void bucket_fence(const uint32_t* a, uint32_t m, uint32_t start, uint32_t bin0,
                                             uint32_t nbins, uint32_t* fence, int fshift) {
  for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x)
    fence[bin0 + i] = start + lower_bound_bin(a, m, bin0 + i, fshift);
}

// Writes the sorted run a/av[0, m) (shared memory) to out[start ..) with
// the padding run inserted before the first element >= pad_kv, and the
// prefix-index entries of bins [bin0, bin0 + nbins) of the result.
__device__ __forceinline__ void bucket_write(const uint32_t* a, const uint32_t* av, uint32_t m, uint32_t* out_k,
                                             uint32_t* out_v, uint32_t start, uint32_t pad, uint32_t pad_kv,
                                             uint32_t pad_v, uint32_t* fence, int fshift, uint32_t bin0,
                                             uint32_t nbins) {
  uint32_t L = m;
  if (pad) {
    uint32_t lo = 0, hi = m;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a[mid] < pad_kv) lo = mid + 1; else hi = mid;
    }
    L = lo;
  }
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const uint32_t dst = start + i + (i >= L ? pad : 0u);
    out_k[dst] = a[i];
    out_v[dst] = av[i];
  }
  for (uint32_t j = threadIdx.x; j < pad; j += blockDim.x) {
    out_k[start + L + j] = pad_kv;
    out_v[start + L + j] = pad_v;
  }
  if (fence) {
    const uint32_t pad_bin = pad ? fence_bin(pad_kv, fshift) : 0xFFFFFFFFu;
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) {
      const uint32_t bin = bin0 + i;
      fence[bin] = start + lower_bound_bin(a, m, bin, fshift) + (bin > pad_bin ? pad : 0u);
    }
  }
}

// Where element i of a bucket lives in the scratch its sort reads.
// ContigSrc: elements start .. start + m - 1 (the batched form's scatter
// writes every bucket contiguously).  RunSrc: the bucket's runs over the
// tiles, in tile order (the stable order); rstart[t] is the first bucket
// position of run t (an exclusive scan of the run lengths) and run t's
// element i - rstart[t] sits at rbase[t] + i (both in shared memory).
struct ContigSrc {
  uint32_t start;
  __device__ __forceinline__ uint32_t at(uint32_t i) const { return start + i; }
};
struct RunSrc {
  const uint32_t* rstart;  // nruns + 1 entries, rstart[nruns] = the bucket's size
  const uint32_t* rbase;
  const uint8_t* chunk;    // run holding element 16 c, per 16-element chunk c (buckets in shared memory), or null
  uint32_t nruns;          // >= 1
  // the largest t with rstart[t] <= i: the run holding i (empty runs share
  // their start with the next run, so they are never the largest)
  __device__ __forceinline__ uint32_t at(uint32_t i) const {
    if (chunk) {  // from the run of the chunk's first element, forward (runs of ~16 elements)
      uint32_t t = chunk[i >> 4];
      while (rstart[t + 1] <= i) ++t;
      return rbase[t] + i;
    }
    uint32_t lo = 0, hi = nruns - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (rstart[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return rbase[lo] + i;
  }
};
static_assert(kMsdMaxTiles <= 256u, "a run index fits in a byte");

// One bucket, one CTA of kBucketThreads: sorts the m elements src.at(0 ..
// m - 1) of (src_k, src_v) stably by the low `rest` bits of the key variable
// (the bits above are the bucket's and equal) into out[start, start + m),
// and writes the prefix-index entries of the bucket's bins [bin0, bin0 +
// nbins) when fence is given.
//   Fast path (bucket in shared memory, no sub-bin above kSubBinMax): one
//   counting pass on the top 12 of the `rest` bits places every element in
//   its sub-bin (about one element each for spread keys), at an arbitrary
//   slot; every element then goes to its sub-bin's start plus its rank in
//   the sub-bin by (key variable, index in the bucket), the stable order.
//   Otherwise: ceil(rest / 8) stable 8-bit passes in shared memory, or, for
//   a bucket above kBucketCap (heavy duplicate keys), the same passes in
//   chunks through global memory, alternating between out and spill (both
//   indexed like out: [start, start + m) belongs to this bucket alone).
// A run of `pad` copies of (pad_kv, pad_v) (a short batch's padding, which
// comes first among equal key variables in the stable order) is written at
// its sorted place: the output holds m + pad elements.
// bsm holds 4 kBucketCap words plus kBucketCap 16-bit indexes.
template <class Src>
__device__ __forceinline__ void bucket_body(const uint32_t* src_k, const uint32_t* src_v, const Src& src,
                                            uint32_t* spill_k, uint32_t* spill_v, uint32_t* out_k, uint32_t* out_v,
                                            uint32_t start, uint32_t m, int rest, uint32_t* __restrict__ fence,
                                            int fshift, uint32_t bin0, uint32_t nbins, uint32_t* bsm,
                                            uint32_t* s_scan, uint32_t pad, uint32_t pad_kv, uint32_t pad_v) {
  __shared__ uint32_t s_whist[kBucketWarps][kRadix];
  __shared__ uint32_t s_excl[kRadix], s_run[kRadix], s_tot[kRadix];
  __shared__ uint32_t s_max;
  uint32_t* ak = bsm;
  uint32_t* av = bsm + kBucketCap;
  uint32_t* bk = bsm + 2 * kBucketCap;
  uint32_t* bv = bsm + 3 * kBucketCap;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t wbase = warp * (32 * kBucketIPT);
  const int npass = (rest + 7) / 8;
  uint32_t kv[kBucketIPT], v[kBucketIPT], rank[kBucketIPT];
  static_assert(kSubBins == kBucketWarps * kRadix, "the counters reuse the per-warp histograms");

  if (m <= kBucketCap && rest >= 12) {
    uint32_t* cnt = &s_whist[0][0];
    uint16_t* bi = reinterpret_cast<uint16_t*>(bsm + 4 * kBucketCap);
    const int sh = rest - 12;
    for (uint32_t i = tid; i < kSubBins; i += kBucketThreads) cnt[i] = 0u;
    if (tid == 0) s_max = 0u;
    __syncthreads();
    uint32_t slot[kBucketIPT];
#pragma unroll
    for (int j = 0; j < kBucketIPT; ++j) {
      const uint32_t i = tid + j * kBucketThreads;
      if (i < m) {
        const uint32_t at = src.at(i);
        const uint32_t k = src_k[at];
        ak[i] = k;
        av[i] = src_v[at];
        slot[j] = atomicAdd(&cnt[(k >> sh) & (kSubBins - 1)], 1u);
      }
    }
    __syncthreads();
    // sub-bin starts: thread t owns counters [8 t, 8 t + 8)
    constexpr int kPer = int(kSubBins) / kBucketThreads;
    uint32_t c[kPer], sum = 0, mx = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      c[e] = cnt[tid * kPer + e];
      sum += c[e];
      mx = max(mx, c[e]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > kSubBinMax) atomicMax(&s_max, mx);
    uint32_t all;
    uint32_t run = block_excl_scan<kBucketThreads>(sum, s_scan, all);
    if (s_max <= kSubBinMax) {  // uniform: s_max settled before the scan's barriers
#pragma unroll
      for (int e = 0; e < kPer; ++e) {
        cnt[tid * kPer + e] = run;
        run += c[e];
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kBucketIPT; ++j) {
        const uint32_t i = tid + j * kBucketThreads;
        if (i < m) {
          const uint32_t k = ak[i];
          const uint32_t pos = cnt[(k >> sh) & (kSubBins - 1)] + slot[j];
          bk[pos] = k;
          bv[pos] = av[i];
          bi[pos] = uint16_t(i);
        }
      }
      __syncthreads();
      // Every element's place: its sub-bin's start plus its rank there by
      // (key variable, index), the stable order.  Each element counts the
      // members of its sub-bin that precede it (independent loads, about
      // two a sub-bin for spread keys) rather than a per-sub-bin insertion
      // sort, whose shifting chain made a warp wait for its fullest sub-bin.
#pragma unroll 2
      for (int j = 0; j < kBucketIPT; ++j) {
        const uint32_t x = tid + j * kBucketThreads;
        if (x < m) {
          const uint32_t k = bk[x], vv = bv[x];
          const uint16_t ix = bi[x];
          const uint32_t b = (k >> sh) & (kSubBins - 1);
          const uint32_t s0 = cnt[b], s1 = b + 1 < kSubBins ? cnt[b + 1] : m;
          // The first four members without a branch (a sub-bin rarely holds
          // more for spread keys, and a loop made each warp run as long as
          // its fullest sub-bin), then the rest.
          uint32_t r = 0;
#pragma unroll
          for (uint32_t u = 0; u < 4; ++u) {
            if (s0 + u < s1) {
              const uint32_t ky = bk[s0 + u];
              r += (ky < k || (ky == k && bi[s0 + u] < ix)) ? 1u : 0u;
            }
          }
          for (uint32_t y = s0 + 4; y < s1; ++y) {
            const uint32_t ky = bk[y];
            r += (ky < k || (ky == k && bi[y] < ix)) ? 1u : 0u;
          }
          ak[s0 + r] = k;
          av[s0 + r] = vv;
        }
      }
      __syncthreads();
      // The prefix-index entries come from the sub-bin starts when a bin is
      // a whole number of sub-bins (fshift >= sh): entry bin0 + j is the
      // start of sub-bin j << (fshift - sh), after the padding run when the
      // bin lies above the padding's bin.
      const bool direct_fence = fence && fshift >= sh;
      bucket_write(ak, av, m, out_k, out_v, start, pad, pad_kv, pad_v, direct_fence ? nullptr : fence, fshift, bin0,
                   nbins);
      if (direct_fence) {
        const uint32_t pad_bin = pad ? fence_bin(pad_kv, fshift) : 0xFFFFFFFFu;
        for (uint32_t j = tid; j < nbins; j += kBucketThreads) {
          const uint32_t sb = j << (fshift - sh);
          fence[bin0 + j] = start + (sb < kSubBins ? cnt[sb] : m) + (bin0 + j > pad_bin ? pad : 0u);
        }
      }
      return;
    }
    __syncthreads();  // skewed bucket: the pass-by-pass path below reloads it
  }

  if (m <= kBucketCap) {
    if (rest < 12) {  // otherwise the fast path above has loaded the bucket already
      for (uint32_t i = tid; i < m; i += kBucketThreads) {
        const uint32_t at = src.at(i);
        ak[i] = src_k[at];
        av[i] = src_v[at];
      }
      __syncthreads();
    }
    uint32_t *sk = ak, *sv = av, *dk = bk, *dv = bv;
    for (int pass = 0; pass < npass; ++pass) {
      const int shift = 8 * pass;
#pragma unroll
      for (int j = 0; j < kBucketIPT; ++j) {
        const uint32_t p = wbase + j * 32 + lane;
        kv[j] = p < m ? sk[p] : 0u;
        v[j] = p < m ? sv[p] : 0u;
      }
      rank_block<kBucketThreads, kBucketIPT>(kv, m, wbase, shift, rank, s_whist, s_excl, s_scan, nullptr);
#pragma unroll
      for (int j = 0; j < kBucketIPT; ++j) {
        const uint32_t p = wbase + j * 32 + lane;
        if (p < m) {
          const uint32_t dg = (kv[j] >> shift) & 255u;
          const uint32_t pos = s_excl[dg] + s_whist[warp][dg] + rank[j];
          dk[pos] = kv[j];
          dv[pos] = v[j];
        }
      }
      __syncthreads();
      uint32_t* t;
      t = sk; sk = dk; dk = t;
      t = sv; sv = dv; dv = t;
    }
    bucket_write(sk, sv, m, out_k, out_v, start, pad, pad_kv, pad_v, fence, fshift, bin0, nbins);
    return;
  }
  // Chunked: npass stable passes through global memory, kBucketCap elements
  // at a time in order: pass 0 from the source to out, then alternating
  // out -> spill -> out ...; an even pass count ends in spill and is copied
  // to out.
  const uint32_t* curk = out_k;
  const uint32_t* curv = out_v;
  uint32_t* dstk = out_k;
  uint32_t* dstv = out_v;
  for (int pass = 0; pass < npass; ++pass) {
    const int shift = 8 * pass;
    if (tid < kRadix) s_tot[tid] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < m; i += kBucketThreads) {
      const uint32_t k = pass == 0 ? src_k[src.at(i)] : curk[start + i];
      atomicAdd(&s_tot[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t all;
    const uint32_t ex = block_excl_scan<kBucketThreads>(tid < kRadix ? s_tot[tid] : 0u, s_scan, all);
    if (tid < kRadix) s_run[tid] = ex;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < m; c0 += kBucketCap) {
      const uint32_t cm = (m - c0) < kBucketCap ? (m - c0) : kBucketCap;
#pragma unroll
      for (int j = 0; j < kBucketIPT; ++j) {
        const uint32_t p = wbase + j * 32 + lane;
        kv[j] = 0u;
        v[j] = 0u;
        if (p < cm) {
          if (pass == 0) {
            const uint32_t at = src.at(c0 + p);
            kv[j] = src_k[at];
            v[j] = src_v[at];
          } else {
            kv[j] = curk[start + c0 + p];
            v[j] = curv[start + c0 + p];
          }
        }
      }
      rank_block<kBucketThreads, kBucketIPT>(kv, cm, wbase, shift, rank, s_whist, s_excl, s_scan, s_tot);
#pragma unroll
      for (int j = 0; j < kBucketIPT; ++j) {
        const uint32_t p = wbase + j * 32 + lane;
        if (p < cm) {
          const uint32_t dg = (kv[j] >> shift) & 255u;
          const uint32_t pos = s_run[dg] + s_whist[warp][dg] + rank[j];
          dstk[start + pos] = kv[j];
          dstv[start + pos] = v[j];
        }
      }
      __syncthreads();
      if (tid < kRadix) s_run[tid] += s_tot[tid];
      __syncthreads();
    }
    curk = dstk;
    curv = dstv;
    dstk = (dstk == out_k) ? spill_k : out_k;
    dstv = (dstv == out_v) ? spill_v : out_v;
  }
  if (curk != out_k) {
    for (uint32_t i = tid; i < m; i += kBucketThreads) {
      out_k[start + i] = curk[start + i];
      out_v[start + i] = curv[start + i];
    }
    __syncthreads();
  }
  if (pad) {
    // open a gap of `pad` before the first element >= pad_kv: move the tail
    // up, a block at a time from the end (each block read before written)
    __shared__ uint32_t s_L;
    if (tid == 0) {
      uint32_t lo = 0, hi = m;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (out_k[start + mid] < pad_kv) lo = mid + 1; else hi = mid;
      }
      s_L = lo;
    }
    __syncthreads();
    const uint32_t L = s_L;
    for (uint32_t e = m; e > L;) {
      const uint32_t c = (e - L) < kBucketThreads ? (e - L) : kBucketThreads;
      uint32_t k = 0, x = 0;
      if (tid < c) {
        k = out_k[start + e - c + tid];
        x = out_v[start + e - c + tid];
      }
      __syncthreads();
      if (tid < c) {
        out_k[start + e - c + tid + pad] = k;
        out_v[start + e - c + tid + pad] = x;
      }
      __syncthreads();
      e -= c;
    }
    for (uint32_t j = tid; j < pad; j += kBucketThreads) {
      out_k[start + L + j] = pad_kv;
      out_v[start + L + j] = pad_v;
    }
    __syncthreads();
  }
  if (fence) bucket_fence(out_k + start, m + pad, start, bin0, nbins, fence, fshift);
}

__global__ void __launch_bounds__(kBucketThreads, 2) bucket_sort(Loader ld, const uint32_t* __restrict__ tmp_k,
                                                              const uint32_t* __restrict__ tmp_v,
                                                              const uint2* __restrict__ runs, uint32_t* spill_k,
                                                              uint32_t* spill_v, uint32_t* __restrict__ out_k,
                                                              uint32_t* __restrict__ out_v,
                                                              const uint32_t* __restrict__ ctl, uint32_t n,
                                                              uint32_t* __restrict__ fence, int fshift,
                                                              uint32_t* __restrict__ next_ctl,
                                                              uint32_t* defer_err) {
  extern __shared__ __align__(16) uint32_t bsm[];
  __shared__ uint32_t s_scan[kBucketWarps];
  __shared__ uint32_t s_rstart[kMsdMaxTiles + 1], s_rbase[kMsdMaxTiles];
  __shared__ uint8_t s_chunk[kBucketCap / 16];
  pdl_trigger();
  pdl_wait();
  const uint32_t tid = threadIdx.x, d = blockIdx.x;
  const uint32_t ntiles = (n + kMsdTile - 1) / kMsdTile;
  // the control block of the next sort starts zeroed (it is idle now)
  if (d == 0)
    for (uint32_t i = tid; i < uint32_t(kSortCtlWords); i += kBucketThreads) next_ctl[i] = 0u;
  if (defer_err && ctl[kSortCtlStatus]) {
    // Deferred key check failed: the batch becomes n placebo tombstones (the
    // key 2^31 - 1 that no query sees), all in the last bin.
    const uint32_t chunk = (n + kRadix - 1) / kRadix;
    const uint32_t lo = d * chunk, hi = (lo + chunk) < n ? lo + chunk : n;
    for (uint32_t i = lo + tid; i < hi; i += kBucketThreads) {
      out_k[i] = kPlaceboKv;
      out_v[i] = 0u;
    }
    if (fence) {
      const uint32_t per = 1u << (24 - fshift);
      for (uint32_t i = tid; i < per; i += kBucketThreads) fence[d * per + i] = 0u;
      if (d == kRadix - 1 && tid == 0) {
        fence[fence_bins(fshift)] = n;
        fence[fence_bins(fshift) + 2] = 0u;
        fence[fence_bins(fshift) + 3] = fence_bins(fshift) - 1;
      }
    }
    if (d == 0 && tid == 0) atomicOr(defer_err, kErrBadKey);
    return;
  }
  // this bucket's run in every tile, in tile order
  const uint2 run = tid < ntiles ? runs[d * kMsdMaxTiles + tid] : make_uint2(0u, 0u);
  uint32_t m;
  const uint32_t rs = block_excl_scan<kBucketThreads>(run.y, s_scan, m);
  if (tid < ntiles) {
    s_rstart[tid] = rs;
    s_rbase[tid] = run.x - rs;
    // the chunks (16 elements) whose first element lies in this run
    if (m <= kBucketCap)
      for (uint32_t c = (rs + 15) >> 4; c < ((rs + run.y + 15) >> 4); ++c) s_chunk[c] = uint8_t(tid);
  }
  if (tid == 0) s_rstart[ntiles] = m;
  const uint32_t start = bucket_start<kBucketThreads>(ctl, d, s_scan);  // its barriers publish the tables
  // a short batch's padding: one run in the bucket of its key variable
  uint32_t pad = ld.npad(), pad_kv = 0, pad_v = 0;
  if (pad) {
    bool bad;
    ld.load(0, pad_kv, pad_v, bad);
    if ((pad_kv >> 24) != d) pad = 0;
  }
  const uint32_t per = fence ? 1u << (24 - fshift) : 0u;  // bins per bucket
  const RunSrc src{s_rstart, s_rbase, m <= kBucketCap ? s_chunk : nullptr, ntiles};
  bucket_body(tmp_k, tmp_v, src, spill_k, spill_v, out_k, out_v, start, m, 24, fence, fshift, d * per, per, bsm,
              s_scan, pad, pad_kv, pad_v);
  // the bucket sort writes every entry: the populated range is all bins
  if (fence && d == kRadix - 1 && tid == 0) {
    fence[fence_bins(fshift)] = n;
    fence[fence_bins(fshift) + 2] = 0u;
    fence[fence_bins(fshift) + 3] = fence_bins(fshift) - 1;
  }
}

__global__ void __launch_bounds__(256) check_keys(const uint32_t* __restrict__ keys, uint64_t n,
                                                  uint32_t* status) {
  bool bad = false;
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += uint64_t(gridDim.x) * 256ull)
    bad |= __ldg(keys + i) > kMaxUserKey;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kErrBadKey);
}

// ---------------------------------------------------------------------------
// The batch sort of the batched form: the same bucket scheme on every
// instance's batch at once.  Instance i splits on the top d_i bits of the key
// variable (2^d_i buckets of about 4096 elements); its batch is cut into
// kMultiSortTile-element tiles; one launch per phase covers every tile or
// bucket of every instance.  Instances without a batch this round (count 0,
// or refused by the prep kernel) leave at once.
// ---------------------------------------------------------------------------
constexpr int kMultiIPT = int(kMultiSortTile) / kThreads;  // 16
static_assert(kMultiIPT * kThreads == int(kMultiSortTile), "tile");

__device__ __forceinline__ uint32_t multi_ops(const MultiBatch& in, const MultiInst& d, uint32_t i) {
  return in.counts ? __ldg(in.counts + i) : d.b;
}

// Element p (< b) of instance d's reversed padded batch: op min(b-1-p, n-1).
__device__ __forceinline__ uint32_t multi_load_key(const MultiBatch& in, const MultiInst& d, uint32_t nops,
                                                   uint32_t p, bool& bad) {
  uint64_t s = uint64_t(d.b) - 1 - p;
  if (s >= nops) s = nops - 1;
  s += d.in_off;
  const uint32_t k = __ldg(in.keys + s);
  const bool is_del = in.del && __ldg(in.del + s) != 0;
  bad = k > kMaxUserKey;
  return bad ? kPlaceboKv : ((k << 1) | (is_del ? 0u : 1u));
}
__device__ __forceinline__ void multi_load(const MultiBatch& in, const MultiInst& d, uint32_t nops, uint32_t p,
                                           uint32_t& kv, uint32_t& v) {
  uint64_t s = uint64_t(d.b) - 1 - p;
  if (s >= nops) s = nops - 1;
  s += d.in_off;
  const uint32_t k = __ldg(in.keys + s);
  const bool is_del = in.del && __ldg(in.del + s) != 0;
  const bool bad = k > kMaxUserKey;
  kv = bad ? kPlaceboKv : ((k << 1) | (is_del ? 0u : 1u));
  v = (is_del || bad || !in.vals) ? 0u : __ldg(in.vals + s);
}

__global__ void __launch_bounds__(kThreads) mseg_count(MultiArena ar, MultiBatch in) {
  __shared__ uint32_t s_h[kRadix];
  const uint32_t tid = threadIdx.x, gt = blockIdx.x;
  const uint32_t i = find_instance(ar.stile_prefix, ar.n, gt);
  const MultiInst& d = ar.inst[i];
  const uint32_t nops = multi_ops(in, d, i);
  if (nops == 0 || nops > d.b) return;  // whole CTA: no batch, or refused
  s_h[tid] = 0;
  __syncthreads();
  const uint32_t t0 = (gt - d.stile0) * kMultiSortTile;
  const uint32_t m = (d.b - t0) < kMultiSortTile ? (d.b - t0) : kMultiSortTile;
  const int shift = 32 - int(d.msd_bits);
  bool bad_any = false;
#pragma unroll 4
  for (int j = 0; j < kMultiIPT; ++j) {
    const uint32_t p = j * kThreads + tid;
    if (p < m) {
      bool bad;
      const uint32_t kv = multi_load_key(in, d, nops, t0 + p, bad);
      bad_any |= bad;
      atomicAdd(&s_h[kv >> shift], 1u);
    }
  }
  const int any_bad = __syncthreads_or(bad_any);
  ar.tilecnt[uint64_t(gt) * 512 + tid] = s_h[tid];
  if (any_bad && tid == 0) atomicOr(ar.badkey + i, 1u);
}

// Per instance (one CTA, thread = bucket): where each tile's run of each
// bucket goes, relative to the instance's batch start.
__global__ void __launch_bounds__(kThreads) mseg_offsets(MultiArena ar) {
  __shared__ uint32_t s_scan[kWarps];
  const uint32_t i = blockIdx.x, tid = threadIdx.x;
  if (ar.k[i] < 0) return;
  const MultiInst& d = ar.inst[i];
  const uint32_t nbk = 1u << d.msd_bits;
  const uint32_t ntiles = (d.b + kMultiSortTile - 1) / kMultiSortTile;
  uint32_t* tc = ar.tilecnt + uint64_t(d.stile0) * 512;
  uint32_t total = 0;
  if (tid < nbk)
    for (uint32_t t = 0; t < ntiles; ++t) total += tc[t * 512 + tid];
  uint32_t all;
  const uint32_t start = block_excl_scan<kThreads>(total, s_scan, all);
  if (tid < nbk) {
    uint32_t run = start;
    for (uint32_t t = 0; t < ntiles; ++t) {
      const uint32_t c = tc[t * 512 + tid];
      tc[t * 512 + 256 + tid] = run;
      run += c;
    }
    ar.bstart[d.bucket0 + tid] = start;
    ar.bcnt[d.bucket0 + tid] = total;
  }
}

__global__ void __launch_bounds__(kThreads) mseg_scatter(MultiArena ar, MultiBatch in) {
  __shared__ __align__(16) uint32_t s_keys[kMultiSortTile];
  __shared__ __align__(16) uint32_t s_vals[kMultiSortTile];
  __shared__ uint32_t s_whist[kWarps][kRadix];
  __shared__ uint32_t s_excl[kRadix], s_gbase[kRadix], s_scan[kWarps];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, gt = blockIdx.x;
  const uint32_t i = find_instance(ar.stile_prefix, ar.n, gt);
  if (ar.k[i] < 0) return;  // whole CTA
  const MultiInst& d = ar.inst[i];
  const uint32_t nops = multi_ops(in, d, i);
  const uint32_t t0 = (gt - d.stile0) * kMultiSortTile;
  const uint32_t m = (d.b - t0) < kMultiSortTile ? (d.b - t0) : kMultiSortTile;
  const int shift = 32 - int(d.msd_bits);
  const uint32_t base = warp * (32 * kMultiIPT);
  uint32_t kv[kMultiIPT], v[kMultiIPT], rank[kMultiIPT];
#pragma unroll
  for (int j = 0; j < kMultiIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    kv[j] = 0;
    v[j] = 0;
    if (p < m) multi_load(in, d, nops, t0 + p, kv[j], v[j]);
  }
  s_gbase[tid] = ar.tilecnt[uint64_t(gt) * 512 + 256 + tid];
  rank_block<kThreads, kMultiIPT>(kv, m, base, shift, rank, s_whist, s_excl, s_scan, nullptr);
#pragma unroll
  for (int j = 0; j < kMultiIPT; ++j) {
    const uint32_t p = base + j * 32 + lane;
    if (p < m) {
      const uint32_t dg = kv[j] >> shift;
      const uint32_t pos = s_excl[dg] + s_whist[warp][dg] + rank[j];
      s_keys[pos] = kv[j];
      s_vals[pos] = v[j];
    }
  }
  __syncthreads();
  uint32_t* tk = ar.tkeys + d.boff;
  uint32_t* tv = ar.tvals + d.boff;
  for (uint32_t e = tid; e < m; e += kThreads) {
    const uint32_t k = s_keys[e];
    const uint32_t dg = k >> shift;
    const uint32_t dst = s_gbase[dg] + (e - s_excl[dg]);
    if (dst < d.b) {
      tk[dst] = k;
      tv[dst] = s_vals[e];
    }
  }
}

// One bucket of one instance per CTA: sorted on the bits below the top d
// into level 0 (when the round's fold target is level 0) or the sorted-batch
// buffer, with that run's prefix-index entries.
__global__ void __launch_bounds__(kBucketThreads, 2) mseg_bucket(MultiArena ar) {
  extern __shared__ __align__(16) uint32_t bsm[];
  __shared__ uint32_t s_scan[kBucketWarps];
  const uint32_t gb = blockIdx.x;
  const uint32_t i = find_instance(ar.bucket_prefix, ar.n, gb);
  const int k = ar.k[i];
  if (k < 0) return;  // whole CTA
  const MultiInst& d = ar.inst[i];
  const uint32_t bucket = gb - d.bucket0;
  const uint32_t start = ar.bstart[gb], m = ar.bcnt[gb];
  uint32_t *ok, *ov, *of;
  if (k == 0) {
    ok = ar.keys + d.lvl_off[0];
    ov = ar.vals + d.lvl_off[0];
    of = ar.fence + d.lvl_fence[0];
  } else {
    ok = ar.bkeys + d.boff;
    ov = ar.bvals + d.boff;
    of = ar.fence + d.batch_fence;
  }
  const int fs = d.fshift0;
  const int rest = 32 - int(d.msd_bits);              // bits below the bucket bits
  const uint32_t per = 1u << (rest - fs);             // bins per bucket
  uint32_t* tk = ar.tkeys + d.boff;
  uint32_t* tv = ar.tvals + d.boff;
  bucket_body(tk, tv, ContigSrc{start}, tk, tv, ok, ov, start, m, rest, of, fs, bucket * per, per, bsm, s_scan, 0u,
              0u, 0u);
  if (bucket == (1u << d.msd_bits) - 1 && threadIdx.x == 0) {
    const uint32_t nb = fence_bins(fs);
    of[nb] = d.b;
    of[nb + 2] = 0u;
    of[nb + 3] = nb - 1;
  }
}

}  // namespace

constexpr size_t kBucketSmem = 4 * size_t(kBucketCap) * sizeof(uint32_t) + size_t(kBucketCap) * sizeof(uint16_t);
PerDeviceFlags g_bucket_attr;

cudaError_t bucket_sort_launch(const SortArgs& a, SortWorkspace& ws, cudaStream_t st, uint32_t* status,
                               cudaEvent_t ev) {
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = set_smem_attr_once(bucket_sort, kBucketSmem, dev, g_bucket_attr)) != cudaSuccess) return e;
  const uint32_t ntiles = (a.n + kMsdTile - 1) / kMsdTile;
  uint2* runs = reinterpret_cast<uint2*>(ws.tilecnt);
  uint32_t* spill_k = ws.tilecnt + kMsdRunWords;
  uint32_t* spill_v = spill_k + a.n;
  uint32_t* ctl = ws.ctl + ws.flip * kSortCtlWords;
  uint32_t* next = ws.ctl + (ws.flip ^ 1) * kSortCtlWords;
  Loader ld{a.mode, a.in_keys, a.in_vals, a.in_del, a.n_in, a.n};
  // a deferred check leaves its verdict in the sort's own control block
  uint32_t* check = a.defer_err ? ctl + kSortCtlStatus : status;
  count_launches(1);
  if ((e = launch_pdl(msd_tile, dim3(ntiles), dim3(kScatterThreads), 0, st, ld, a.tmp_keys, a.tmp_vals, runs, ctl,
                      check)) != cudaSuccess)
    return e;
  if (status && !a.defer_err && (e = cudaEventRecord(ev, st)) != cudaSuccess) return e;
  count_launches(1);
  if ((e = launch_pdl(bucket_sort, dim3(kRadix), dim3(kBucketThreads), kBucketSmem, st, ld,
                      static_cast<const uint32_t*>(a.tmp_keys), static_cast<const uint32_t*>(a.tmp_vals),
                      static_cast<const uint2*>(runs), spill_k, spill_v, a.out_keys, a.out_vals,
                      static_cast<const uint32_t*>(ctl), a.n, a.fence, a.fshift, next, a.defer_err)) != cudaSuccess)
    return e;
  ws.flip ^= 1;
  return cudaSuccess;
}

cudaError_t sort_launch(const SortArgs& a, SortWorkspace& ws, cudaStream_t st, uint32_t* status,
                        cudaEvent_t ev) {
  if (a.n == 0) return cudaSuccess;
  if (a.n <= kMsdMaxN && ws.tilecnt) return bucket_sort_launch(a, ws, st, status, ev);
  const uint32_t ntiles = (a.n + kSortTile - 1) / kSortTile;
  if (ntiles > ws.max_tiles) return cudaErrorInvalidValue;
  cudaError_t e;
  if (++ws.epoch >= (1u << 30)) {
    ws.epoch = 1;
    e = cudaMemsetAsync(ws.lookback, 0, sizeof(uint64_t) * kSortPasses * ws.max_tiles * kRadix, st);
    if (e != cudaSuccess) return e;
  }
  uint32_t* ctl = ws.ctl + ws.flip * kSortCtlWords;
  e = cudaMemsetAsync(ctl, 0, sizeof(uint32_t) * kSortCtlWords, st);
  if (e != cudaSuccess) return e;
  Loader ld{a.mode, a.in_keys, a.in_vals, a.in_del, a.n_in, a.n};
  uint32_t hblocks = (a.n + 255) / 256;
  if (hblocks > 4 * 152) hblocks = 4 * 152;
  count_launches(1);
  sort_histogram<<<hblocks, 256, 0, st>>>(ld, ctl, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (status && (e = cudaEventRecord(ev, st)) != cudaSuccess) return e;
  // in -> tmp -> out -> tmp -> out
  uint32_t* bk[2] = {a.tmp_keys, a.out_keys};
  uint32_t* bv[2] = {a.tmp_vals, a.out_vals};
  const size_t lb_stride = size_t(ws.max_tiles) * kRadix;
  count_launches(1);
  sort_pass<true><<<ntiles, kThreads, 0, st>>>(ld, nullptr, nullptr, bk[0], bv[0], ctl, ws.lookback,
                                                0, ws.epoch, ws.sticky);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  for (int p = 1; p < kSortPasses; ++p) {
    count_launches(1);
    sort_pass<false><<<ntiles, kThreads, 0, st>>>(ld, bk[(p - 1) & 1], bv[(p - 1) & 1], bk[p & 1],
                                                   bv[p & 1], ctl, ws.lookback + p * lb_stride, p,
                                                   ws.epoch, ws.sticky);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // leave the next half zeroed, as the bucket path does
  ws.flip ^= 1;
  e = cudaMemsetAsync(ws.ctl + ws.flip * kSortCtlWords, 0, sizeof(uint32_t) * kSortCtlWords, st);
  if (e != cudaSuccess) return e;
  if (a.fence) return build_fence_launch(a.out_keys, a.n, a.fence, a.fshift, st);
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


cudaError_t multi_sort_count_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st) {
  if (ar.total_stiles == 0) return cudaSuccess;
  count_launches(1);
  mseg_count<<<unsigned(ar.total_stiles), kThreads, 0, st>>>(ar, in);
  return cudaGetLastError();
}

cudaError_t multi_sort_prepare() {
  return cudaFuncSetAttribute(mseg_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBucketSmem));
}

cudaError_t multi_sort_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st) {
  cudaError_t e;
  if (ar.total_stiles == 0) return cudaSuccess;
  count_launches(1);
  mseg_offsets<<<ar.n, kThreads, 0, st>>>(ar);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  count_launches(1);
  mseg_scatter<<<unsigned(ar.total_stiles), kThreads, 0, st>>>(ar, in);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  count_launches(1);
  mseg_bucket<<<unsigned(ar.total_buckets), kBucketThreads, kBucketSmem, st>>>(ar);
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
// may take.  For them the sort below takes all of its scratch (the
// bucket sort's tile scratch, control words, run table and spill area) from
// one fixed array with static storage in this file, which every GPU that
// loads the library holds until the process exits.  Its size is set by
// kNoAllocMaxPairs.
// ---------------------------------------------------------------------------
#include <mutex>

#include "gpulsm.h"

namespace gpulsm {
namespace {

constexpr uint32_t kNoAllocMaxPairs = LSM_SORT_NOALLOC_MAX_PAIRS;
// Up to kMsdMaxN pairs the sort is the two-kernel bucket sort, which needs
// no look-back words; the array below holds only what that path uses.
static_assert(kNoAllocMaxPairs <= kMsdMaxN, "the allocation-free sort stays on the bucket path");
constexpr size_t kNoAllocCtl = 2112;                    // > 2 * kSortCtlWords, multiple of 64
constexpr size_t kNoAllocSticky = kNoAllocCtl - 1;      // last ctl word: device error bits
constexpr size_t kNoAllocTmpK = kNoAllocCtl;
constexpr size_t kNoAllocTmpV = kNoAllocTmpK + kNoAllocMaxPairs;
constexpr size_t kNoAllocRuns = kNoAllocTmpV + kNoAllocMaxPairs;  // run table + spill area
constexpr size_t kNoAllocWords = kNoAllocRuns + kMsdWsWords;
static_assert(kNoAllocCtl > 2 * size_t(kSortCtlWords), "both control halves and the error word fit");
static_assert(kNoAllocRuns % 2 == 0, "the run table holds 8-byte entries");

// The scratch itself: about 17 MB for kNoAllocMaxPairs = 2^20.
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
    // and the control words must start at zero.
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LSM_ERR_CUDA;
    }
    uint32_t* base = static_cast<uint32_t*>(p);
    if (cudaMemsetAsync(base, 0, kNoAllocCtl * sizeof(uint32_t), st) != cudaSuccess) {
      cudaGetLastError();
      return LSM_ERR_CUDA;
    }
    d.ws.ctl = base;
    d.ws.lookback = nullptr;
    d.ws.max_tiles = 0;
    d.ws.epoch = 0;
    d.ws.flip = 0;
    d.ws.sticky = base + kNoAllocSticky;
    d.ws.tilecnt = base + kNoAllocRuns;
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
  // Each sort leaves the control block of the next one zeroed; the run table
  // and the tile scratch are fully rewritten by every call before they are
  // read, so nothing else needs zeroing.
  cudaError_t e = sort_launch(a, d.ws, st, nullptr, nullptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LSM_ERR_CUDA;
  }
  return LSM_OK;
}
