// Retrieval paths of the GPU LSM: LOOKUP (§III-D, §IV-B, Fig. 2(b)), COUNT
// (§III-E, §IV-C, Fig. 2(c)) and RANGE (§III-E, §IV-D, Fig. 2(d)).
//
// LOOKUP  searches the full levels from the newest (smallest) to the oldest
//         for the first element whose key is >= q; if that element has key q
//         it decides: regular -> found with its value, tombstone -> absent
//         (and the search stops).  The top of each level's search tree is the
//         level's prefix index, a splitter table of 2^16 .. 2^24 entries
//         (about one per 8 elements): two adjacent loads narrow a search to
//         one bin of about one 32-byte sector, and a short binary search
//         finishes inside it.
//         lookup_direct takes the queries in input order (one thread each);
//         lookup_sorted takes them sorted by key (the "bulk" alternative of
//         §IV-B): the same search, but neighbouring threads read
//         neighbouring parts of each level, which keeps page and sector
//         reuse high when the levels span many gigabytes.
// COUNT   per query and level the window [lower_bound(k1), upper_bound(k2))
//         on the original key; the windows of all levels are then merged on
//         the key, newer level first among equal keys, and a key counts when
//         its first element in that order (its newest version) is regular.
//         This replaces the paper's gather + segmented sort + validation of
//         §IV-C by a per-query multi-way merge of windows that are already
//         sorted; the result is the same count.
// RANGE   the same windows (kept from the count pass), an exclusive scan of
//         the counts into offsets, and a second merge that writes each live
//         (key, value) at its offset, keys ascending within a query (§IV-D).
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

constexpr int kThreads = 256;

// lower_bound of key variable `target` in level l: the level's prefix index
// (a splitter table with about one entry per 8 elements) gives the run of the
// target's bin in two adjacent loads; a short binary search finishes inside.
__device__ __forceinline__ uint32_t level_lower_bound(const LevelSet& ls, int l, uint32_t target) {
  const uint32_t* f = ls.fence[l];
  const int fs = ls.fshift[l];
  const uint32_t bin = fence_bin(target, fs), n = ls.n[l];
  return lower_bound_kv(ls.keys[l], fence_at(f, fs, n, bin), fence_at(f, fs, n, bin + 1), target);
}

// Window [lower_bound(t1), lower_bound(t2)) of level l, t1 <= t2.  A narrow
// interval usually has both bounds in one prefix-index bin: the bin's two
// entries are then loaded once and the second search starts at the first
// bound.
__device__ __forceinline__ uint32_t bin_lower_bound(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t target,
                                                    uint32_t& kv);

__device__ __forceinline__ void level_window(const LevelSet& ls, int l, uint32_t t1, uint32_t t2, uint32_t& lo,
                                             uint32_t& hi) {
  const uint32_t* f = ls.fence[l];
  const int fs = ls.fshift[l];
  const uint32_t n = ls.n[l], b1 = fence_bin(t1, fs), b2 = fence_bin(t2, fs);
  const uint32_t s1 = fence_at(f, fs, n, b1), e1 = fence_at(f, fs, n, b1 + 1);
  const uint32_t s2 = b2 == b1 ? s1 : fence_at(f, fs, n, b2), e2 = b2 == b1 ? e1 : fence_at(f, fs, n, b2 + 1);
  uint32_t kv;
  // the two bounds' searches are independent (each bin read in one round trip)
  lo = bin_lower_bound(ls.keys[l], s1, e1, t1, kv);
  hi = bin_lower_bound(ls.keys[l], s2, e2, t2, kv);
}

// lower_bound of key variable `target` inside the bin [lo, hi) of a level's
// keys `a` (128-byte aligned, readable slack after the end), with the key
// variable at the result in kv when it is < hi.  A bin of up to eight
// elements from its 16-byte aligned start is read with two 16-byte loads and
// searched in registers, so the search and the key at the found position
// cost one round trip instead of a chain of dependent loads; longer bins are
// bisected.
__device__ __forceinline__ uint32_t bin_lower_bound(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t target,
                                                    uint32_t& kv) {
  const uint32_t a0 = lo & ~3u;
  kv = 0;
  if (hi <= a0 + 8) {
    const uint4 x = __ldg(reinterpret_cast<const uint4*>(a + a0));
    const uint4 y = __ldg(reinterpret_cast<const uint4*>(a + a0 + 4));
    const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) c += (a0 + j >= lo && a0 + j < hi && w[j] < target) ? 1u : 0u;
    const uint32_t pos = lo + c;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (a0 + j == pos) kv = w[j];
    return pos;
  }
  const uint32_t pos = lower_bound_kv(a, lo, hi, target);
  if (pos < hi) kv = __ldg(a + pos);
  return pos;
}

// Lookup of one key over the levels (newest first).  The elements of the
// key, if any, lie in the target's prefix-index bin [lo, hi) (both status
// bits of a key share its bin).
__device__ __forceinline__ void lookup_one(const LevelSet& ls, uint32_t key, uint32_t& val, uint8_t& found) {
  val = 0;
  found = 0;
  if (key > kMaxUserKey) return;
  const uint32_t target = key << 1;
  for (int l = 0; l < ls.count; ++l) {
    const uint32_t* f = ls.fence[l];
    const int fs = ls.fshift[l];
    const uint32_t n = ls.n[l], bin = fence_bin(target, fs);
    const uint32_t hi = fence_at(f, fs, n, bin + 1);
    uint32_t kv;
    const uint32_t pos = bin_lower_bound(ls.keys[l], fence_at(f, fs, n, bin), hi, target, kv);
    if (pos < hi && key_of(kv) == key) {
      if (kv & 1u) {
        found = 1;
        val = __ldg(ls.vals[l] + pos);
      }
      return;
    }
  }
}

__global__ void __launch_bounds__(kThreads) lookup_direct(LevelSet ls, const uint32_t* __restrict__ q, uint64_t nq,
                                                          uint32_t* __restrict__ out_v,
                                                          uint8_t* __restrict__ out_f) {
  for (uint64_t i = blockIdx.x * uint64_t(kThreads) + threadIdx.x; i < nq;
       i += uint64_t(gridDim.x) * kThreads) {
    uint32_t v;
    uint8_t f;
    lookup_one(ls, __ldg(q + i), v, f);
    out_v[i] = v;
    out_f[i] = f;
  }
}

// Queries sorted by key: the same per-query search as lookup_direct, in key
// order, so neighbouring threads read neighbouring parts of every level and
// prefix index (few pages and sectors per warp); results scattered back to
// positions idx[i].
__global__ void __launch_bounds__(kThreads) lookup_sorted(LevelSet ls, const uint32_t* __restrict__ sq,
                                                          const uint32_t* __restrict__ idx, uint64_t nq,
                                                          uint32_t* __restrict__ out_v,
                                                          uint8_t* __restrict__ out_f) {
  for (uint64_t i = blockIdx.x * uint64_t(kThreads) + threadIdx.x; i < nq;
       i += uint64_t(gridDim.x) * kThreads) {
    uint32_t v;
    uint8_t f;
    lookup_one(ls, __ldg(sq + i), v, f);
    const uint32_t o = __ldg(idx + i);
    if (o < nq) {  // a permutation of [0, nq) unless the sort gave up on a wait
      out_v[o] = v;
      out_f[o] = f;
    }
  }
}

// Per-query multi-way merge of the level windows on the key, newer level
// first among equal keys; visits the newest element of every key once.  L is
// a compile-time bound on the number of full levels (loops fully unrolled, so
// the cursors stay in registers); levels l >= ls.count are empty.  Once a
// key's newest element is taken, every level skips the whole run of that key
// (a binary search when the run is longer than one element), so keys stored
// many times (stale versions, a short batch's padding) cost O(L log run).
template <bool kEmit, int L>
__device__ __forceinline__ uint32_t merge_windows(const LevelSet& ls, const uint32_t (&lo)[L],
                                                  const uint32_t (&hi)[L], uint32_t* out_k, uint32_t* out_v,
                                                  uint64_t room) {
  if (L == 1 && ls.count == 1 && hi[0] - (lo[0] & ~3u) <= 16) {
    // One level and a short window: its keys (and values) from the 16-byte
    // aligned start in four 16-byte loads each, walked in registers; a key's
    // first element is its newest (level order), kept when regular.
    const uint32_t* a = ls.keys[0];
    const uint32_t a0 = lo[0] & ~3u;
    uint32_t w[16], v[16];
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
      const uint4 x = __ldg(reinterpret_cast<const uint4*>(a + a0) + c4);
      w[4 * c4] = x.x;
      w[4 * c4 + 1] = x.y;
      w[4 * c4 + 2] = x.z;
      w[4 * c4 + 3] = x.w;
      if (kEmit) {
        const uint4 y = __ldg(reinterpret_cast<const uint4*>(ls.vals[0] + a0) + c4);
        v[4 * c4] = y.x;
        v[4 * c4 + 1] = y.y;
        v[4 * c4 + 2] = y.z;
        v[4 * c4 + 3] = y.w;
      }
    }
    uint32_t c = 0, prev = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t pos = a0 + j;
      if (pos >= lo[0] && pos < hi[0]) {
        const uint32_t k = key_of(w[j]);
        if (k != prev && (w[j] & 1u)) {
          if (kEmit && c < room) {
            out_k[c] = k;
            out_v[c] = v[j];
          }
          ++c;
        }
        prev = k;
      }
    }
    return c;
  }
  uint32_t cur[L], head[L];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    cur[l] = lo[l];
    head[l] = (l < ls.count && cur[l] < hi[l]) ? key_of(__ldg(ls.keys[l] + cur[l])) : 0xFFFFFFFFu;
  }
  uint32_t c = 0;
  while (true) {
    uint32_t bk = 0xFFFFFFFFu, p = 0;
    int best = -1;
#pragma unroll
    for (int l = 0; l < L; ++l)
      if (head[l] < bk) {  // strict: the lowest (newest) level wins ties
        bk = head[l];
        best = l;
        p = cur[l];
      }
    if (best < 0) break;
    const uint32_t kv = __ldg(ls.keys[best] + p);
    if (kv & 1u) {
      if (kEmit && c < room) {
        out_k[c] = bk;
        out_v[c] = __ldg(ls.vals[best] + p);
      }
      ++c;
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
      if (head[l] == bk) {  // past every element of key bk in level l
        const uint32_t* a = ls.keys[l];
        uint32_t q = cur[l] + 1;
        uint32_t nk = q < hi[l] ? key_of(__ldg(a + q)) : 0xFFFFFFFFu;
        if (nk == bk) {
          q = upper_bound_key(a, q + 1, hi[l], bk);
          nk = q < hi[l] ? key_of(__ldg(a + q)) : 0xFFFFFFFFu;
        }
        cur[l] = q;
        head[l] = nk;
      }
    }
  }
  return c;
}

// With `perm` (queries sorted by k1: k1 holds the sorted lower bounds and
// perm their positions), thread i serves query perm[i] and stores its count
// and windows at that position; neighbouring threads then search
// neighbouring parts of every level.
// Queries whose windows hold more than kWideMin elements in all are wide:
// with a wide list, the count kernel appends them to it (their count and
// output are then written by the warp kernels below) instead of merging
// hundreds of elements in one thread.
constexpr uint32_t kWideMin = 40;

template <int L>
__device__ __forceinline__ uint32_t window_total(const uint32_t (&lo)[L], const uint32_t (&hi)[L]) {
  uint32_t t = 0;
#pragma unroll
  for (int l = 0; l < L; ++l) t += hi[l] - lo[l];
  return t;
}

template <int L>
__global__ void __launch_bounds__(kThreads) count_kernel(LevelSet ls, const uint32_t* __restrict__ k1,
                                                         const uint32_t* __restrict__ k2, uint64_t nq,
                                                         uint32_t* __restrict__ out_count,
                                                         uint32_t* __restrict__ bounds,
                                                         const uint32_t* __restrict__ perm,
                                                         uint32_t* __restrict__ wide) {
  for (uint64_t i0 = blockIdx.x * uint64_t(kThreads) + threadIdx.x; i0 < nq;
       i0 += uint64_t(gridDim.x) * kThreads) {
    const uint64_t i = perm ? __ldg(perm + i0) : i0;
    if (i >= nq) continue;  // a permutation of [0, nq) unless its sort gave up on a wait
    const uint32_t a = __ldg(k1 + i0);
    uint32_t z = __ldg(k2 + i);
    if (z > kMaxUserKey) z = kMaxUserKey;
    uint32_t lo[L], hi[L];
    const bool empty = a > z;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      lo[l] = hi[l] = 0;
      if (l < ls.count && !empty) level_window(ls, l, a << 1, (z + 1u) << 1, lo[l], hi[l]);
    }
    if (wide && window_total(lo, hi) > kWideMin) {
      wide[1 + atomicAdd(wide, 1u)] = uint32_t(i0);
    } else {
      out_count[i] = merge_windows<false, L>(ls, lo, hi, nullptr, nullptr, 0);
    }
    if (bounds) {
      uint32_t* b = bounds + i * 2 * ls.count;
#pragma unroll
      for (int l = 0; l < L; ++l)
        if (l < ls.count) {
          b[2 * l] = lo[l];
          b[2 * l + 1] = hi[l];
        }
    }
  }
}

template <int L>
__global__ void __launch_bounds__(kThreads) range_emit(LevelSet ls, uint64_t nq,
                                                       const uint32_t* __restrict__ bounds,
                                                       const uint64_t* __restrict__ offsets,
                                                       uint32_t* __restrict__ keys,
                                                       uint32_t* __restrict__ vals,
                                                       const uint32_t* __restrict__ perm, bool wide) {
  for (uint64_t i0 = blockIdx.x * uint64_t(kThreads) + threadIdx.x; i0 < nq;
       i0 += uint64_t(gridDim.x) * kThreads) {
    const uint64_t i = perm ? __ldg(perm + i0) : i0;
    if (i >= nq) continue;
    uint32_t lo[L], hi[L];
    const uint32_t* b = bounds + i * 2 * ls.count;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      lo[l] = l < ls.count ? b[2 * l] : 0u;
      hi[l] = l < ls.count ? b[2 * l + 1] : 0u;
    }
    if (wide && window_total(lo, hi) > kWideMin) continue;  // emitted by range_wide
    const uint64_t o = offsets[i];
    merge_windows<true, L>(ls, lo, hi, keys + o, vals + o, offsets[i + 1] - o);
  }
}

// Wide queries, one warp each: the key interval [k1, k2] is cut into 32
// equal key sub-intervals, one per lane; every lane takes its windows in
// each level and merges them as the one-thread path does (all versions of
// a key fall in one lane's sub-interval, so the lanes' results are
// disjoint).  The count is the warp's sum; the range output of a lane goes
// after the lanes before it (a warp scan of their counts).
template <int L>
__device__ __forceinline__ uint32_t lane_windows(const LevelSet& ls, uint32_t a, uint32_t z, uint32_t (&lo)[L],
                                                 uint32_t (&hi)[L]) {
  const uint64_t w = (uint64_t(z) - a + 32) / 32;  // ceil((z - a + 1) / 32)
  const uint64_t s0 = uint64_t(a) + lane_id() * w;
  const uint64_t s1 = s0 + w - 1 < z ? s0 + w - 1 : uint64_t(z);
  const bool empty = s0 > z;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    lo[l] = hi[l] = 0;
    if (l < ls.count && !empty) level_window(ls, l, uint32_t(s0) << 1, (uint32_t(s1) + 1u) << 1, lo[l], hi[l]);
  }
  return empty ? 0u : merge_windows<false, L>(ls, lo, hi, nullptr, nullptr, 0);
}

template <int L>
__global__ void __launch_bounds__(kThreads) count_wide(LevelSet ls, const uint32_t* __restrict__ k1,
                                                       const uint32_t* __restrict__ k2, uint64_t nq,
                                                       uint32_t* __restrict__ out_count,
                                                       const uint32_t* __restrict__ perm,
                                                       const uint32_t* __restrict__ wide) {
  const uint32_t nw = *reinterpret_cast<const volatile uint32_t*>(wide);
  const uint32_t lane = lane_id();
  for (uint32_t w = (blockIdx.x * kThreads + threadIdx.x) >> 5; w < nw; w += (gridDim.x * kThreads) >> 5) {
    const uint32_t i0 = wide[1 + w];
    const uint64_t i = perm ? __ldg(perm + i0) : i0;
    if (i >= nq) continue;  // whole warp
    const uint32_t a = __ldg(k1 + i0);
    uint32_t z = __ldg(k2 + i);
    if (z > kMaxUserKey) z = kMaxUserKey;
    uint32_t lo[L], hi[L];
    const uint32_t c = warp_sum(lane_windows<L>(ls, a, z, lo, hi));
    if (lane == 0) out_count[i] = c;
  }
}

template <int L>
__global__ void __launch_bounds__(kThreads) range_wide(LevelSet ls, const uint32_t* __restrict__ k1,
                                                       const uint32_t* __restrict__ k2, uint64_t nq,
                                                       const uint64_t* __restrict__ offsets,
                                                       uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                       const uint32_t* __restrict__ perm,
                                                       const uint32_t* __restrict__ wide) {
  const uint32_t nw = *reinterpret_cast<const volatile uint32_t*>(wide);
  for (uint32_t w = (blockIdx.x * kThreads + threadIdx.x) >> 5; w < nw; w += (gridDim.x * kThreads) >> 5) {
    const uint32_t i0 = wide[1 + w];
    const uint64_t i = perm ? __ldg(perm + i0) : i0;
    if (i >= nq) continue;  // whole warp
    const uint32_t a = __ldg(k1 + i0);
    uint32_t z = __ldg(k2 + i);
    if (z > kMaxUserKey) z = kMaxUserKey;
    uint32_t lo[L], hi[L];
    const uint32_t c = lane_windows<L>(ls, a, z, lo, hi);
    const uint32_t before = warp_incl_scan(c) - c;
    const uint64_t o = offsets[i], room = offsets[i + 1] - o;
    if (c && before < room)
      merge_windows<true, L>(ls, lo, hi, keys + o + before, vals + o + before, room - before);
  }
}

// SUCCESSOR / PREDECESSOR (the order-based queries the problem statement's
// footnote names beside the three retrievals, read inclusively): the live
// pair with the smallest key >= q, or the largest key <= q.  Each level's
// cursor starts at q's position; the levels are merged on the key from q
// outwards (ascending for the successor, descending for the predecessor),
// newest level first among equal keys; the first key whose newest element is
// regular is the answer, every other key is skipped in all levels at once.
// Within a level a key's newest element is the first of its run, so the
// descending merge looks up each run's start.
template <int L, bool kSucc>
__global__ void __launch_bounds__(kThreads) neighbor_kernel(LevelSet ls, const uint32_t* __restrict__ q,
                                                            uint64_t nq, uint32_t* __restrict__ out_k,
                                                            uint32_t* __restrict__ out_v,
                                                            uint8_t* __restrict__ out_f) {
  for (uint64_t i = blockIdx.x * uint64_t(kThreads) + threadIdx.x; i < nq; i += uint64_t(gridDim.x) * kThreads) {
    const uint32_t key = __ldg(q + i);
    uint32_t rk = 0, rv = 0;
    uint8_t rf = 0;
    uint32_t cur[L], head[L];
    bool live[L];  // the level still has a candidate on the search side
#pragma unroll
    for (int l = 0; l < L; ++l) {
      cur[l] = 0;
      head[l] = 0;
      live[l] = false;
      if (l < ls.count) {
        if (kSucc) {
          if (key <= kMaxUserKey) {
            cur[l] = level_lower_bound(ls, l, key << 1);
            live[l] = cur[l] < ls.n[l];
          }
        } else {
          const uint32_t kq = key < kMaxUserKey ? key : kMaxUserKey;
          const uint32_t e = level_lower_bound(ls, l, (kq + 1u) << 1);  // first key > kq
          live[l] = e > 0;
          cur[l] = live[l] ? e - 1 : 0u;
        }
        if (live[l]) head[l] = key_of(__ldg(ls.keys[l] + cur[l]));
      }
    }
    while (true) {
      int best = -1;
      uint32_t bk = 0;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        if (!live[l]) continue;
        const bool better = best < 0 || (kSucc ? head[l] < bk : head[l] > bk);  // strict: newest level wins ties
        if (better) {
          bk = head[l];
          best = l;
        }
      }
      if (best < 0) break;
      // newest element of key bk: the run start in the newest level holding it
      uint32_t p = cur[best];
      if (!kSucc) p = lower_bound_kv(ls.keys[best], 0, cur[best] + 1, bk << 1);
      const uint32_t kv = __ldg(ls.keys[best] + p);
      if (kv & 1u) {
        rk = bk;
        rv = __ldg(ls.vals[best] + p);
        rf = 1;
        break;
      }
      // skip key bk in every level
#pragma unroll
      for (int l = 0; l < L; ++l) {
        if (!live[l] || head[l] != bk) continue;
        const uint32_t* a = ls.keys[l];
        if (kSucc) {
          uint32_t nx = cur[l] + 1;
          if (nx < ls.n[l] && key_of(__ldg(a + nx)) == bk) nx = upper_bound_key(a, nx + 1, ls.n[l], bk);
          cur[l] = nx;
          live[l] = nx < ls.n[l];
          if (live[l]) head[l] = key_of(__ldg(a + nx));
        } else {
          const uint32_t st = lower_bound_kv(a, 0, cur[l] + 1, bk << 1);  // run start of bk
          live[l] = st > 0;
          if (live[l]) {
            cur[l] = st - 1;
            head[l] = key_of(__ldg(a + cur[l]));
          }
        }
      }
    }
    out_k[i] = rk;
    out_v[i] = rv;
    out_f[i] = rf;
  }
}

constexpr int kScanIPT = 8;
constexpr int kScanTile = kThreads * kScanIPT;  // 2048
constexpr uint64_t kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbMask = (1ull << 62) - 1;

__global__ void __launch_bounds__(kThreads) scan_kernel(const uint32_t* __restrict__ in, uint64_t n,
                                                        uint64_t* __restrict__ out, uint64_t* lookback,
                                                        uint32_t* tile_ctr, uint32_t* status,
                                                        uint64_t ntiles) {
  __shared__ uint64_t s_scan[kThreads / 32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_tile;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint64_t tile = s_tile;
  const uint64_t base = tile * kScanTile + uint64_t(tid) * kScanIPT;
  uint32_t v[kScanIPT];
  uint64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kScanIPT; ++j) {
    v[j] = base + j < n ? __ldg(in + base + j) : 0u;
    sum += v[j];
  }
  uint64_t tile_sum;
  const uint64_t before = block_excl_scan<kThreads, uint64_t>(sum, s_scan, tile_sum);
  if (tid == 0) {
    uint64_t prefix = 0;
    if (tile == 0) {
      st_relaxed_u64(lookback, kLbIncl | tile_sum);
    } else {
      st_relaxed_u64(lookback + tile, kLbAgg | tile_sum);
      int64_t t = int64_t(tile) - 1;
      uint64_t t0 = 0;
      while (t >= 0) {
        const uint64_t w = ld_relaxed_u64(lookback + t);
        if (!(w & (kLbAgg | kLbIncl))) {
          if (!spin_continue(t0, kWaitLimitNs, status)) break;
          continue;
        }
        prefix += w & kLbMask;
        if (w & kLbIncl) break;
        --t;
      }
      st_relaxed_u64(lookback + tile, kLbIncl | (prefix + tile_sum));
    }
    s_prefix = prefix;
    if (tile == ntiles - 1) out[n] = prefix + tile_sum;
  }
  __syncthreads();
  uint64_t run = s_prefix + before;
#pragma unroll
  for (int j = 0; j < kScanIPT; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
}

unsigned persistent_grid(uint64_t work, int per_block, unsigned cap) {
  uint64_t b = (work + per_block - 1) / per_block;
  if (b > cap) b = cap;
  return unsigned(b ? b : 1);
}

// Lookup in the batched form: query g belongs to instance i with
// qoff[i] <= g < qoff[i + 1] and searches that instance's full levels (the
// set bits of r_i), newest first, exactly as lookup_one does.
__global__ void __launch_bounds__(kThreads) multi_lookup(MultiArena ar, const uint32_t* __restrict__ q,
                                                         const uint64_t* __restrict__ qoff, uint64_t nq,
                                                         uint32_t* __restrict__ out_v,
                                                         uint8_t* __restrict__ out_f) {
  for (uint64_t g = blockIdx.x * uint64_t(kThreads) + threadIdx.x; g < nq; g += uint64_t(gridDim.x) * kThreads) {
    const uint32_t i = find_instance(qoff, ar.n, g);
    const MultiInst& d = ar.inst[i];
    const uint32_t key = __ldg(q + g);
    uint32_t val = 0;
    uint8_t found = 0;
    if (key <= kMaxUserKey) {
      const uint32_t target = key << 1;
      uint32_t r = ar.r[i];
      while (r) {
        const int l = __ffs(r) - 1;
        r &= r - 1;
        const uint32_t* keys = ar.keys + d.lvl_off[l];
        const uint32_t* f = ar.fence + d.lvl_fence[l];
        const int fs = d.lvl_fshift[l];
        const uint32_t n = d.b << l, bin = fence_bin(target, fs);
        const uint32_t hi = fence_at(f, fs, n, bin + 1);
        uint32_t kv;
        const uint32_t pos = bin_lower_bound(keys, fence_at(f, fs, n, bin), hi, target, kv);
        if (pos < hi && key_of(kv) == key) {
          if (kv & 1u) {
            found = 1;
            val = __ldg(ar.vals + d.lvl_off[l] + pos);
          }
          break;
        }
      }
    }
    out_v[g] = val;
    out_f[g] = found;
  }
}

}  // namespace

cudaError_t lookup_launch(const LevelSet& ls, const uint32_t* q, uint64_t nq, uint32_t* val, uint8_t* found,
                          cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  count_launches(1);
  lookup_direct<<<persistent_grid(nq, kThreads, 152 * 8), kThreads, 0, st>>>(ls, q, nq, val, found);
  return cudaGetLastError();
}

cudaError_t lookup_sorted_launch(const LevelSet& ls, const uint32_t* sq, const uint32_t* idx, uint64_t nq,
                                 uint32_t* val, uint8_t* found, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  count_launches(1);
  lookup_sorted<<<persistent_grid(nq, kThreads, 152 * 8), kThreads, 0, st>>>(ls, sq, idx, nq, val, found);
  return cudaGetLastError();
}

cudaError_t count_launch(const LevelSet& ls, const uint32_t* k1, const uint32_t* k2, uint64_t nq,
                         uint32_t* count, uint32_t* bounds, cudaStream_t st, const uint32_t* perm,
                         uint32_t* wide) {
  if (nq == 0) return cudaSuccess;
  cudaError_t e;
  if (wide && (e = cudaMemsetAsync(wide, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
  const unsigned grid = persistent_grid(nq, kThreads, 152 * 8);
  count_launches(1);
  if (ls.count <= 1) count_kernel<1><<<grid, kThreads, 0, st>>>(ls, k1, k2, nq, count, bounds, perm, wide);
  else if (ls.count <= 2) count_kernel<2><<<grid, kThreads, 0, st>>>(ls, k1, k2, nq, count, bounds, perm, wide);
  else if (ls.count <= 4) count_kernel<4><<<grid, kThreads, 0, st>>>(ls, k1, k2, nq, count, bounds, perm, wide);
  else if (ls.count <= 8) count_kernel<8><<<grid, kThreads, 0, st>>>(ls, k1, k2, nq, count, bounds, perm, wide);
  else if (ls.count <= 16) count_kernel<16><<<grid, kThreads, 0, st>>>(ls, k1, k2, nq, count, bounds, perm, wide);
  else count_kernel<kMaxLevels><<<grid, kThreads, 0, st>>>(ls, k1, k2, nq, count, bounds, perm, wide);
  if ((e = cudaGetLastError()) != cudaSuccess || !wide) return e;
  // the wide queries, one warp each (the grid covers every query's warp when
  // all are wide; an empty list ends at once)
  const unsigned wgrid = persistent_grid(nq * 32, kThreads, 152 * 8);
  count_launches(1);
  if (ls.count <= 1) count_wide<1><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, count, perm, wide);
  else if (ls.count <= 2) count_wide<2><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, count, perm, wide);
  else if (ls.count <= 4) count_wide<4><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, count, perm, wide);
  else if (ls.count <= 8) count_wide<8><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, count, perm, wide);
  else if (ls.count <= 16) count_wide<16><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, count, perm, wide);
  else count_wide<kMaxLevels><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, count, perm, wide);
  return cudaGetLastError();
}

cudaError_t scan_launch(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* lookback, uint32_t* tile_ctr,
                        uint32_t* status, cudaStream_t st) {
  cudaError_t e;
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
  const uint64_t ntiles = scan_tiles(n);
  if ((e = cudaMemsetAsync(lookback, 0, sizeof(uint64_t) * ntiles, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
  count_launches(1);
  scan_kernel<<<unsigned(ntiles), kThreads, 0, st>>>(in, n, out, lookback, tile_ctr, status, ntiles);
  return cudaGetLastError();
}

cudaError_t range_emit_launch(const LevelSet& ls, uint64_t nq, const uint32_t* bounds, const uint64_t* offsets,
                              uint32_t* keys, uint32_t* vals, cudaStream_t st, const uint32_t* perm,
                              const uint32_t* k1, const uint32_t* k2, const uint32_t* wide) {
  if (nq == 0) return cudaSuccess;
  cudaError_t e;
  const bool w = wide != nullptr;
  const unsigned grid = persistent_grid(nq, kThreads, 152 * 8);
  count_launches(1);
  if (ls.count <= 1) range_emit<1><<<grid, kThreads, 0, st>>>(ls, nq, bounds, offsets, keys, vals, perm, w);
  else if (ls.count <= 2) range_emit<2><<<grid, kThreads, 0, st>>>(ls, nq, bounds, offsets, keys, vals, perm, w);
  else if (ls.count <= 4) range_emit<4><<<grid, kThreads, 0, st>>>(ls, nq, bounds, offsets, keys, vals, perm, w);
  else if (ls.count <= 8) range_emit<8><<<grid, kThreads, 0, st>>>(ls, nq, bounds, offsets, keys, vals, perm, w);
  else if (ls.count <= 16) range_emit<16><<<grid, kThreads, 0, st>>>(ls, nq, bounds, offsets, keys, vals, perm, w);
  else range_emit<kMaxLevels><<<grid, kThreads, 0, st>>>(ls, nq, bounds, offsets, keys, vals, perm, w);
  if ((e = cudaGetLastError()) != cudaSuccess || !w) return e;
  const unsigned wgrid = persistent_grid(nq * 32, kThreads, 152 * 8);
  count_launches(1);
  if (ls.count <= 1) range_wide<1><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, offsets, keys, vals, perm, wide);
  else if (ls.count <= 2) range_wide<2><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, offsets, keys, vals, perm, wide);
  else if (ls.count <= 4) range_wide<4><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, offsets, keys, vals, perm, wide);
  else if (ls.count <= 8) range_wide<8><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, offsets, keys, vals, perm, wide);
  else if (ls.count <= 16) range_wide<16><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, offsets, keys, vals, perm, wide);
  else range_wide<kMaxLevels><<<wgrid, kThreads, 0, st>>>(ls, k1, k2, nq, offsets, keys, vals, perm, wide);
  return cudaGetLastError();
}


cudaError_t multi_lookup_launch(const MultiArena& ar, const uint32_t* q, const uint64_t* qoff, uint64_t nq,
                                uint32_t* val, uint8_t* found, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  count_launches(1);
  multi_lookup<<<persistent_grid(nq, kThreads, 152 * 8), kThreads, 0, st>>>(ar, q, qoff, nq, val, found);
  return cudaGetLastError();
}


cudaError_t neighbor_launch(const LevelSet& ls, const uint32_t* q, uint64_t nq, bool successor, uint32_t* key,
                            uint32_t* val, uint8_t* found, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  const unsigned grid = persistent_grid(nq, kThreads, 152 * 8);
  count_launches(1);
#define LSM_NB(LL)                                                                                   \
  (successor ? (neighbor_kernel<LL, true><<<grid, kThreads, 0, st>>>(ls, q, nq, key, val, found), 0) \
             : (neighbor_kernel<LL, false><<<grid, kThreads, 0, st>>>(ls, q, nq, key, val, found), 0))
  if (ls.count <= 1) LSM_NB(1);
  else if (ls.count <= 2) LSM_NB(2);
  else if (ls.count <= 4) LSM_NB(4);
  else if (ls.count <= 8) LSM_NB(8);
  else if (ls.count <= 16) LSM_NB(16);
  else LSM_NB(kMaxLevels);
#undef LSM_NB
  return cudaGetLastError();
}

}  // namespace gpulsm
