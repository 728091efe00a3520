// Cascade fold of the GPU LSM (§III-B, §IV-A, Fig. 2(a), Fig. 3) and the
// merge/compaction of cleanup (§III-F, §IV-E).
//
// The paper inserts a batch by merging it with level 0, the result with
// level 1, and so on up to the first empty level k = ffz(r), each merge
// stable on the original key with the newer run first.  The result of that
// chain is the merge of all k + 1 sorted sources at once in the total order
//     (key, source rank, index in source),
// source rank 0 being the sorted batch, rank 1 level 0, ..., rank k level
// k - 1 (newest to oldest).  Here that merge is done in one pass straight into
// level k: every element is read once and written once.
//
//   fold_partition  one warp per output tile boundary p = t * 4096 finds the
//                   co-rank vector (how many elements of each source precede
//                   position p).  The sources' prefix indexes (fences) give
//                   the 2^15-key bin holding the p-th element in a few probes;
//                   a bisection over the low 15 key bits inside that bin,
//                   each lane keeping a bracket in its own source, finds the
//                   key; the elements of that key are then split among the
//                   sources in rank order.
//   fold_merge      one CTA per tile: the TMA engine copies the k + 1 source
//                   segments into shared memory (16-byte aligned supersets);
//                   a left-deep chain of merge-path merges in shared memory
//                   (ranks 0 and 1, then the result with rank 2, ...; ties to
//                   the lower rank) builds the tile as (key, value) pairs in
//                   an XOR-swizzled layout, and the tile is written out
//                   coalesced.  The plain fold also writes the new level's
//                   prefix index.
// Cleanup uses the same two kernels over all full levels; the merge then keeps
// only the first element of every key when it is regular and compacts the
// survivors with a decoupled look-back scan across tiles.
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kMinPer = 8;
constexpr uint32_t kSlotCap = (kFoldTile + 8 * kMaxSources + 15) / 16 * 16;  // TMA slots + alignment slack
static_assert(kSlotCap % 16 == 0, "16-byte aligned buffers");
static_assert(kFoldTile % kThreads == 0 && kFoldTile / kThreads <= 32, "keep bits per thread");
constexpr size_t kMergeSmem = 2 * size_t(kSlotCap) * sizeof(uint32_t) + 2 * size_t(kFoldTile) * sizeof(uint2);

constexpr uint64_t kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbMask = (1ull << 62) - 1;

// Slot of pair q of a merge step in shared memory: q with its low 4 bits
// XORed by bits 4..7.  A thread writing 8 consecutive pairs (q = 8 t + e)
// then hits pair slot 8 (t & 1) + (e ^ (t >> 1)) modulo 16: the 16 lanes of
// each half-warp phase of a 64-bit access use 16 different bank pairs, and 16
// consecutive pairs stay a permutation of one 128-byte row.
__device__ __forceinline__ uint32_t psw(uint32_t q) { return q ^ ((q >> 4) & 15u); }

// Sum over the sources of fence_j[P] (lanes >= S contribute 0).
__device__ __forceinline__ uint64_t fence_sum(const uint32_t* f, bool act, uint32_t P) {
  return warp_sum<uint64_t>(act ? __ldg(f + P) : 0u);
}

__global__ void __launch_bounds__(256) fold_partition(FoldSources src, uint64_t total, uint32_t ntiles,
                                                      uint32_t* __restrict__ part) {
  const uint32_t t = (blockIdx.x * 256u + threadIdx.x) >> 5;
  if (t > ntiles) return;  // whole warp leaves together
  const uint32_t lane = lane_id();
  const int S = src.count;
  const bool act = lane < uint32_t(S);
  const uint32_t n = act ? src.n[lane] : 0u;
  const uint32_t* a = act ? src.keys[lane] : nullptr;
  const uint32_t* f = act ? src.fence[lane] : nullptr;
  const uint64_t p = uint64_t(t) * kFoldTile < total ? uint64_t(t) * kFoldTile : total;
  uint32_t* out = part + uint64_t(t) * S;
  if (p >= total) {
    if (act) out[lane] = n;
    return;
  }
  // 1. The bin: largest P with C(P) <= p, C(P) = sum of fence_j[P]
  //    (C(0) = 0 <= p < C(65536) = total).  Start from the proportional
  //    guess, gallop to a bracket, then bisect.
  uint32_t lo, hi;
  {
    uint32_t g = uint32_t((p * kFenceBins) / total);
    if (g >= kFenceBins) g = kFenceBins - 1;
    if (fence_sum(f, act, g) <= p) {
      lo = g;
      uint32_t step = 1;
      while (true) {
        hi = lo + step < kFenceBins ? lo + step : kFenceBins;
        if (hi == kFenceBins || fence_sum(f, act, hi) > p) break;
        lo = hi;
        step <<= 1;
      }
    } else {
      hi = g;
      uint32_t step = 1;
      while (true) {
        lo = hi > step ? hi - step : 0u;
        if (lo == 0 || fence_sum(f, act, lo) <= p) break;
        hi = lo;
        step <<= 1;
      }
    }
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (fence_sum(f, act, mid) <= p) lo = mid; else hi = mid;
    }
  }
  // 2. Smallest key x in the bin with #{key <= x} > p.  Invariant per lane:
  //    blo = #{key <= xlo - 1}, bhi = #{key <= xhi} in this lane's source.
  uint32_t blo = act ? __ldg(f + lo) : 0u, bhi = act ? __ldg(f + lo + 1) : 0u;
  uint32_t xlo = lo << 15, xhi = ((lo + 1) << 15) - 1;
  while (xlo < xhi) {
    const uint32_t mid = xlo + ((xhi - xlo) >> 1);
    const uint32_t u = act ? upper_bound_key(a, blo, bhi, mid) : 0u;
    const uint64_t s = warp_sum<uint64_t>(u);
    if (s > p) {
      xhi = mid;
      bhi = u;
    } else {
      xlo = mid + 1;
      blo = u;
    }
  }
  // 3. blo / bhi are now the lower / upper bound of key x in this source; the
  //    p - sum(blo) elements of key x that precede p come from the lowest ranks.
  const uint32_t cnt = bhi - blo;
  const uint64_t need = p - warp_sum<uint64_t>(blo);
  const uint64_t excl = warp_incl_scan<uint64_t>(cnt) - cnt;
  uint64_t take = 0;
  if (need > excl) take = (need - excl) < cnt ? (need - excl) : cnt;
  if (act) out[lane] = blo + uint32_t(take);
}

// One merge step of the tile: output[0, nA + nB) = merge of run A (the
// newer ranks) and run B (the next rank), ties to A.  B always sits in the
// TMA slot area (separate key and value arrays); A is either there too (the
// first step) or the (key, value) pair buffer X written by the step before.
// Each thread produces ceil(m / 256) consecutive outputs after a merge-path
// search for its first one; outputs go to the pair buffer Y, swizzled.
template <bool kAFromSlot>
__device__ __forceinline__ void merge_step(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                                           const uint2* __restrict__ X, uint2* __restrict__ Y, uint32_t aS,
                                           uint32_t nA, uint32_t bS, uint32_t nB) {
  const uint32_t m = nA + nB;
  // at least kMinPer outputs per working thread: each thread pays one
  // merge-path search, so small steps use few threads
  uint32_t per = (m + kThreads - 1) / kThreads;
  per = per < kMinPer ? kMinPer : per;
  const uint32_t q0 = threadIdx.x * per;
  if (q0 >= m) return;
  const uint32_t q1 = q0 + per < m ? q0 + per : m;
  const uint32_t* xk = reinterpret_cast<const uint32_t*>(X);
  auto keyA = [&](uint32_t i) { return kAFromSlot ? sk[aS + i] : xk[2 * psw(i)]; };
  auto pairA = [&](uint32_t i) { return kAFromSlot ? make_uint2(sk[aS + i], sv[aS + i]) : X[psw(i)]; };
  // merge path: how many of the first q0 outputs come from A
  uint32_t lo = q0 > nB ? q0 - nB : 0u, hi = q0 < nA ? q0 : nA;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (key_of(keyA(mid)) <= key_of(sk[bS + q0 - 1 - mid])) lo = mid + 1; else hi = mid;
  }
  uint32_t ia = lo, ib = q0 - lo;
  uint2 a = ia < nA ? pairA(ia) : make_uint2(0u, 0u);
  uint2 b = ib < nB ? make_uint2(sk[bS + ib], sv[bS + ib]) : make_uint2(0u, 0u);
  for (uint32_t q = q0; q < q1; ++q) {
    const bool take_a = ia < nA && (ib >= nB || key_of(a.x) <= key_of(b.x));
    if (take_a) {
      Y[psw(q)] = a;
      if (++ia < nA) a = pairA(ia);
    } else {
      Y[psw(q)] = b;
      if (++ib < nB) b = make_uint2(sk[bS + ib], sv[bS + ib]);
    }
  }
}

template <bool kCleanup>
__global__ void __launch_bounds__(kThreads) fold_merge(FoldSources src, uint64_t total,
                                                       const uint32_t* __restrict__ part,
                                                       uint32_t* __restrict__ out_k,
                                                       uint32_t* __restrict__ out_v,
                                                       uint32_t* __restrict__ out_fence, uint32_t* status,
                                                       uint64_t* lookback, uint32_t* tile_ctr,
                                                       uint64_t* out_count, uint32_t ntiles) {
  extern __shared__ __align__(128) uint32_t sm[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_rstart[kMaxSources], s_rlen[kMaxSources];
  __shared__ uint32_t s_a0[kMaxSources], s_span[kMaxSources], s_slot[kMaxSources];
  __shared__ uint32_t s_scan[kThreads / 32];
  __shared__ uint32_t s_tile, s_prev_key, s_ok;
  __shared__ uint64_t s_prefix;

  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const int S = src.count;
  if (kCleanup) {
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
  } else if (tid == 0) {
    s_tile = blockIdx.x;
  }
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t obase = uint64_t(tile) * kFoldTile;
  const uint32_t tile_n = uint32_t((total - obase) < kFoldTile ? (total - obase) : kFoldTile);
  uint32_t* sk = sm;                                          // slot keys
  uint32_t* sv = sm + kSlotCap;                               // slot values
  uint2* X = reinterpret_cast<uint2*>(sm + 2 * kSlotCap);     // pair buffers
  uint2* Y = X + kFoldTile;

  // Segment of each source in this tile, and its 16-byte aligned superset.
  if (warp == 0) {
    uint32_t c0 = 0, c1 = 0, a0 = 0, span = 0, prev = 0;
    bool has_prev = false;
    if (lane < uint32_t(S)) {
      c0 = part[uint64_t(tile) * S + lane];
      c1 = part[uint64_t(tile + 1) * S + lane];
      if (c1 > c0) {
        a0 = c0 & ~3u;
        span = ((c1 + 3u) & ~3u) - a0;
      }
      if (c0 > 0) {
        has_prev = true;
        prev = key_of(__ldg(src.keys[lane] + c0 - 1));
      }
    }
    const uint32_t slot = warp_incl_scan(span) - span;
    if (lane < uint32_t(S)) {
      s_rstart[lane] = slot + (c0 - a0);
      s_rlen[lane] = c1 - c0;
      s_a0[lane] = a0;
      s_span[lane] = span;
      s_slot[lane] = slot;
    }
    // Key of the element just before this tile in merged order: the largest
    // key among the sources' last elements before their co-ranks.
    uint32_t mx = has_prev ? prev : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const bool any_prev = __any_sync(0xffffffffu, has_prev);
    if (lane == 0) s_prev_key = any_prev ? mx : 0xFFFFFFFFu;  // no key equals 2^32 - 1
  }
  __syncthreads();

  // Stage the segments with the TMA engine (one thread issues, all wait).
  if (tid == 0) {
    uint32_t bytes = 0, ok = 1;
    for (int r = 0; r < S; ++r) {
      if (!s_span[r]) continue;
      const uintptr_t gk = reinterpret_cast<uintptr_t>(src.keys[r] + s_a0[r]);
      const uintptr_t gv = reinterpret_cast<uintptr_t>(src.vals[r] + s_a0[r]);
      if ((gk | gv) & 15u) ok = 0;
      bytes += 2u * s_span[r] * 4u;
    }
    s_ok = ok;
    if (!ok) {
      atomicOr(status, kErrAlign);
      bytes = 0;
    }
    mbar_arrive_expect_tx(&s_bar, bytes);
    if (ok) {
      for (int r = 0; r < S; ++r) {
        if (!s_span[r]) continue;
        bulk_g2s(sk + s_slot[r], src.keys[r] + s_a0[r], s_span[r] * 4u, &s_bar);
        bulk_g2s(sv + s_slot[r], src.vals[r] + s_a0[r], s_span[r] * 4u, &s_bar);
      }
    }
  }
  const bool landed = mbar_wait_bounded(&s_bar, 0, status);
  __syncthreads();
  if (!s_ok) {  // never expected: plain loads instead of the bulk copies
    for (int r = 0; r < S; ++r)
      for (uint32_t i = tid; i < s_span[r]; i += kThreads) {
        sk[s_slot[r] + i] = __ldg(src.keys[r] + s_a0[r] + i);
        sv[s_slot[r] + i] = __ldg(src.vals[r] + s_a0[r] + i);
      }
    __syncthreads();
  }
  if (!__syncthreads_and(landed)) {
    // A copy never completed; give it one more bounded wait before leaving
    // so that no transfer lands in shared memory after this CTA is gone.
    if (tid == 0) mbar_wait_bounded(&s_bar, 0, status);
    return;
  }

  // Left-deep merge order: X = run 0 + run 1, then X = X + run r for each
  // further rank.  Runs grow with their rank (the batch and level 0 are the
  // smallest), so every element moves about twice in all.
  if (S == 1) {
    merge_step<true>(sk, sv, nullptr, X, s_rstart[0], s_rlen[0], 0u, 0u);
  } else {
    merge_step<true>(sk, sv, nullptr, X, s_rstart[0], s_rlen[0], s_rstart[1], s_rlen[1]);
  }
  uint32_t m = s_rlen[0] + (S > 1 ? s_rlen[1] : 0u);
  for (int r = 2; r < S; ++r) {
    __syncthreads();
    merge_step<false>(sk, sv, X, Y, 0u, m, s_rstart[r], s_rlen[r]);
    m += s_rlen[r];
    uint2* t = X;
    X = Y;
    Y = t;
  }
  __syncthreads();
  const uint32_t* xk = reinterpret_cast<const uint32_t*>(X);

  if (!kCleanup) {
    // Write the tile (coalesced) and, when asked, the new level's prefix
    // index: for every bin P after the previous element's bin up to this
    // element's bin, fence[P] = this element's position; the last element of
    // the fold closes the table up to bin 65536.
    const int first_prev_bin = s_prev_key == 0xFFFFFFFFu ? -1 : int(s_prev_key >> 15);
    for (uint32_t base = warp * 32; base < tile_n; base += kThreads) {
      const uint32_t q = base + lane;
      const bool valid = q < tile_n;
      const uint2 p = valid ? X[psw(q)] : make_uint2(0u, 0u);
      if (valid) {
        out_k[obase + q] = p.x;
        out_v[obase + q] = p.y;
      }
      if (out_fence) {
        uint32_t kprev = __shfl_up_sync(0xffffffffu, p.x, 1);
        if (lane == 0 && base > 0) kprev = xk[2 * psw(base - 1)];
        if (valid) {
          const int bin = int(fence_bin(p.x));
          const int pb = q ? int(fence_bin(kprev)) : first_prev_bin;
          for (int P = pb + 1; P <= bin; ++P) out_fence[P] = uint32_t(obase + q);
          if (obase + q + 1 == total)
            for (uint32_t P = uint32_t(bin) + 1; P <= kFenceBins; ++P) out_fence[P] = uint32_t(total);
        }
      }
    }
    return;
  }

  // Cleanup: keep the first element of each key (the newest one, §IV-E) when
  // it is regular; compact across tiles.
  constexpr int kE = kFoldTile / kThreads;
  const uint32_t q0 = tid * kE;
  uint32_t keep = 0, nkeep = 0;
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const uint32_t q = q0 + e;
    if (q < tile_n) {
      const uint32_t kv = xk[2 * psw(q)];
      const uint32_t prev = q ? key_of(xk[2 * psw(q - 1)]) : s_prev_key;
      if (key_of(kv) != prev && (kv & 1u)) {
        keep |= 1u << e;
        ++nkeep;
      }
    }
  }
  uint32_t tile_keep;
  const uint32_t before = block_excl_scan<kThreads>(nkeep, s_scan, tile_keep);
  if (tid == 0) {
    uint64_t prefix = 0;
    if (tile == 0) {
      st_relaxed_u64(lookback, kLbIncl | tile_keep);
    } else {
      st_relaxed_u64(lookback + tile, kLbAgg | tile_keep);
      int64_t t = int64_t(tile) - 1;
      uint64_t t0 = 0;
      while (t >= 0) {
        const uint64_t w = ld_relaxed_u64(lookback + t);
        if (!(w & (kLbAgg | kLbIncl))) {
          if (t0 == 0) t0 = globaltimer_ns();
          else if (globaltimer_ns() - t0 > kWaitLimitNs) {
            atomicOr(status, kErrTimeout);
            break;
          }
          continue;
        }
        prefix += w & kLbMask;
        if (w & kLbIncl) break;
        --t;
      }
      st_relaxed_u64(lookback + tile, kLbIncl | (prefix + tile_keep));
    }
    s_prefix = prefix;
    if (tile == ntiles - 1) *out_count = prefix + tile_keep;
  }
  __syncthreads();
  uint64_t dst = s_prefix + before;
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    if (keep & (1u << e)) {
      const uint2 p = X[psw(q0 + e)];
      out_k[dst] = p.x;
      out_v[dst] = p.y;
      ++dst;
    }
  }
}

__global__ void __launch_bounds__(256) distribute(DistributeArgs a) {
  for (uint64_t g = blockIdx.x * 256ull + threadIdx.x; g < a.total; g += uint64_t(gridDim.x) * 256ull) {
    int l = 0;
    while (l + 1 < a.nlevels && g >= a.level_start[l + 1]) ++l;
    const uint64_t dst = a.level_off[l] + (g - a.level_start[l]);
    uint32_t k = kPlaceboKv, v = 0u;
    if (g < a.n_live) {
      k = __ldg(a.src_keys + g);
      v = __ldg(a.src_vals + g);
    }
    a.keys[dst] = k;
    a.vals[dst] = v;
  }
}

// Prefix index of a sorted run: position i opens every bin after the bin of
// element i - 1 up to its own; position n closes the table.
__global__ void __launch_bounds__(256) build_fence(const uint32_t* __restrict__ keys, uint32_t n,
                                                   uint32_t* __restrict__ fence) {
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i <= n; i += uint64_t(gridDim.x) * 256ull) {
    const uint32_t bin = i < n ? fence_bin(__ldg(keys + i)) : kFenceBins;
    const int pb = i ? int(fence_bin(__ldg(keys + i - 1))) : -1;
    for (int P = pb + 1; P <= int(bin); ++P) fence[P] = uint32_t(i);
  }
}

}  // namespace

cudaError_t fold_partition_launch(const FoldArgs& a, cudaStream_t st) {
  const uint64_t ntiles = fold_tiles(a.total);
  if (ntiles == 0) return cudaSuccess;
  const uint64_t pblocks = ((ntiles + 1) * 32 + 255) / 256;
  count_launches(1);
  fold_partition<<<unsigned(pblocks), 256, 0, st>>>(a.src, a.total, uint32_t(ntiles), a.part);
  return cudaGetLastError();
}

cudaError_t fold_merge_launch(const FoldArgs& a, cudaStream_t st) {
  static bool attr_set = false;
  cudaError_t e;
  if (!attr_set) {
    if ((e = cudaFuncSetAttribute(fold_merge<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(kMergeSmem))) != cudaSuccess)
      return e;
    if ((e = cudaFuncSetAttribute(fold_merge<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(kMergeSmem))) != cudaSuccess)
      return e;
    attr_set = true;
  }
  const uint64_t ntiles = fold_tiles(a.total);
  if (a.cleanup) {
    if ((e = cudaMemsetAsync(a.out_count, 0, sizeof(uint64_t), st)) != cudaSuccess) return e;
  }
  if (ntiles == 0) return cudaSuccess;
  if (a.cleanup) {
    if ((e = cudaMemsetAsync(a.lookback, 0, sizeof(uint64_t) * ntiles, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.tile_ctr, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    count_launches(1);
    fold_merge<true><<<unsigned(ntiles), kThreads, kMergeSmem, st>>>(
        a.src, a.total, a.part, a.out_keys, a.out_vals, nullptr, a.status, a.lookback, a.tile_ctr,
        a.out_count, uint32_t(ntiles));
  } else {
    count_launches(1);
    fold_merge<false><<<unsigned(ntiles), kThreads, kMergeSmem, st>>>(
        a.src, a.total, a.part, a.out_keys, a.out_vals, a.out_fence, a.status, nullptr, nullptr, nullptr,
        uint32_t(ntiles));
  }
  return cudaGetLastError();
}

cudaError_t fold_launch(const FoldArgs& a, cudaStream_t st) {
  cudaError_t e = fold_partition_launch(a, st);
  if (e != cudaSuccess) return e;
  return fold_merge_launch(a, st);
}

cudaError_t distribute_launch(const DistributeArgs& a, cudaStream_t st) {
  if (a.total == 0) return cudaSuccess;
  uint64_t blocks = (a.total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  distribute<<<unsigned(blocks), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t build_fence_launch(const uint32_t* keys, uint32_t n, uint32_t* fence, cudaStream_t st) {
  uint64_t blocks = (uint64_t(n) + 1 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_launches(1);
  build_fence<<<unsigned(blocks), 256, 0, st>>>(keys, n, fence);
  return cudaGetLastError();
}

}  // namespace gpulsm
