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
//                   position p) by bisection over the 31-bit key space, each
//                   lane keeping a shrinking bracket in its own source, then
//                   splits the tied key among the sources in rank order.
//   fold_merge      one CTA per tile: the TMA engine copies the k + 1 source
//                   segments into shared memory (16-byte aligned supersets),
//                   a tree of pairwise merge-path merges in shared memory
//                   combines adjacent ranks (ties to the lower rank), and the
//                   tile is written out with 16-byte stores.
// Cleanup uses the same two kernels over all full levels; the merge then keeps
// only the first element of every key when it is regular and compacts the
// survivors with a decoupled look-back scan across tiles.
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

constexpr int kThreads = 256;
constexpr int kE = kFoldTile / kThreads;                       // outputs per thread per round
constexpr uint32_t kCap = kFoldTile + 8 * kMaxSources;          // per buffer, with alignment slack
static_assert(kCap % 4 == 0, "16-byte aligned buffers");
constexpr size_t kMergeSmem = 4 * size_t(kCap) * sizeof(uint32_t);

constexpr uint64_t kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbMask = (1ull << 62) - 1;

__global__ void __launch_bounds__(256) fold_partition(FoldSources src, uint64_t total, uint32_t ntiles,
                                                      uint32_t* __restrict__ part) {
  const uint32_t t = (blockIdx.x * 256u + threadIdx.x) >> 5;
  if (t > ntiles) return;  // whole warp leaves together
  const uint32_t lane = lane_id();
  const int S = src.count;
  const bool act = lane < uint32_t(S);
  const uint32_t n = act ? src.n[lane] : 0u;
  const uint32_t* a = act ? src.keys[lane] : nullptr;
  const uint64_t p = uint64_t(t) * kFoldTile < total ? uint64_t(t) * kFoldTile : total;
  uint32_t* out = part + uint64_t(t) * S;
  if (p >= total) {
    if (act) out[lane] = n;
    return;
  }
  // Smallest key x with #{elements with key <= x} > p.  Invariant per lane:
  // blo = #{key <= xlo - 1}, bhi = #{key <= xhi} in this lane's source.
  uint32_t blo = 0, bhi = n, xlo = 0, xhi = 0x7FFFFFFFu;
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
  // blo / bhi are now the lower / upper bound of key x in this source; the
  // p - sum(blo) elements of key x that precede p come from the lowest ranks.
  const uint32_t cnt = bhi - blo;
  const uint64_t need = p - warp_sum<uint64_t>(blo);
  const uint64_t excl = warp_incl_scan<uint64_t>(cnt) - cnt;
  uint64_t take = 0;
  if (need > excl) take = (need - excl) < cnt ? (need - excl) : cnt;
  if (act) out[lane] = blo + uint32_t(take);
}

template <bool kCleanup>
__global__ void __launch_bounds__(kThreads) fold_merge(FoldSources src, uint64_t total,
                                                       const uint32_t* __restrict__ part,
                                                       uint32_t* __restrict__ out_k,
                                                       uint32_t* __restrict__ out_v, uint32_t* status,
                                                       uint64_t* lookback, uint32_t* tile_ctr,
                                                       uint64_t* out_count, uint32_t ntiles) {
  extern __shared__ __align__(128) uint32_t sm[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_rstart[kMaxSources], s_rlen[kMaxSources], s_ostart[kMaxSources + 1];
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
  uint32_t* ak = sm;
  uint32_t* av = sm + kCap;
  uint32_t* bk = sm + 2 * kCap;
  uint32_t* bv = sm + 3 * kCap;

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
      if (kCleanup && c0 > 0) {
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
    if (kCleanup) {
      // Key of the element just before this tile in merged order: the largest
      // key among the sources' last elements before their co-ranks.
      uint32_t m = has_prev ? prev : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      const bool any_prev = __any_sync(0xffffffffu, has_prev);
      if (lane == 0) s_prev_key = any_prev ? m : 0xFFFFFFFFu;  // no key is 2^32 - 1 >> 0
    }
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
        bulk_g2s(ak + s_slot[r], src.keys[r] + s_a0[r], s_span[r] * 4u, &s_bar);
        bulk_g2s(av + s_slot[r], src.vals[r] + s_a0[r], s_span[r] * 4u, &s_bar);
      }
    }
  }
  const bool landed = mbar_wait_bounded(&s_bar, 0, status);
  __syncthreads();
  if (!s_ok) {  // never expected: plain loads instead of the bulk copies
    for (int r = 0; r < S; ++r)
      for (uint32_t i = tid; i < s_span[r]; i += kThreads) {
        ak[s_slot[r] + i] = __ldg(src.keys[r] + s_a0[r] + i);
        av[s_slot[r] + i] = __ldg(src.vals[r] + s_a0[r] + i);
      }
    __syncthreads();
  }
  if (!__syncthreads_and(landed)) {
    // A copy never completed; give it one more bounded wait before leaving
    // so that no transfer lands in shared memory after this CTA is gone.
    if (tid == 0) mbar_wait_bounded(&s_bar, 0, status);
    return;
  }

  // Tree of pairwise merges: runs 2j and 2j+1 (adjacent ranks) -> run j.
  uint32_t runs = uint32_t(S);
  uint32_t *ck = ak, *cv = av, *nk = bk, *nv = bv;
  do {
    const uint32_t pairs = (runs + 1) >> 1;
    if (tid == 0) {
      uint32_t o = 0;
      for (uint32_t j = 0; j < pairs; ++j) {
        s_ostart[j] = o;
        o += s_rlen[2 * j] + ((2 * j + 1 < runs) ? s_rlen[2 * j + 1] : 0u);
      }
      s_ostart[pairs] = o;
    }
    __syncthreads();
    uint32_t q = tid * kE;
    const uint32_t q_end = (q + kE < tile_n) ? q + kE : tile_n;
    uint32_t j = 0;
    while (q < q_end) {
      while (s_ostart[j + 1] <= q) ++j;
      const uint32_t aS = s_rstart[2 * j], nA = s_rlen[2 * j];
      const bool hasB = 2 * j + 1 < runs;
      const uint32_t bS = hasB ? s_rstart[2 * j + 1] : 0u, nB = hasB ? s_rlen[2 * j + 1] : 0u;
      const uint32_t d = q - s_ostart[j];
      const uint32_t seg_end = (q_end < s_ostart[j + 1]) ? q_end : s_ostart[j + 1];
      uint32_t lo = d > nB ? d - nB : 0u, hi = d < nA ? d : nA;
      while (lo < hi) {  // merge path: how many of the first d come from A
        const uint32_t mid = (lo + hi) >> 1;
        if (key_of(ck[aS + mid]) <= key_of(ck[bS + d - 1 - mid])) lo = mid + 1; else hi = mid;
      }
      uint32_t ia = lo, ib = d - lo;
      for (; q < seg_end; ++q) {
        bool take_a;
        if (ia >= nA) take_a = false;
        else if (ib >= nB) take_a = true;
        else take_a = key_of(ck[aS + ia]) <= key_of(ck[bS + ib]);
        if (take_a) {
          nk[q] = ck[aS + ia];
          nv[q] = cv[aS + ia];
          ++ia;
        } else {
          nk[q] = ck[bS + ib];
          nv[q] = cv[bS + ib];
          ++ib;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      for (uint32_t jj = 0; jj < pairs; ++jj) {
        s_rstart[jj] = s_ostart[jj];
        s_rlen[jj] = s_ostart[jj + 1] - s_ostart[jj];
      }
    }
    runs = pairs;
    uint32_t* t;
    t = ck; ck = nk; nk = t;
    t = cv; cv = nv; nv = t;
    __syncthreads();
  } while (runs > 1);

  if (!kCleanup) {
    uint32_t* ok = out_k + obase;
    uint32_t* ov = out_v + obase;
    const uint32_t n4 = ((reinterpret_cast<uintptr_t>(ok) | reinterpret_cast<uintptr_t>(ov)) & 15u) ? 0u
                                                                                                     : (tile_n & ~3u);
    for (uint32_t i = tid * 4; i < n4; i += kThreads * 4) {
      *reinterpret_cast<uint4*>(ok + i) = *reinterpret_cast<const uint4*>(ck + i);
      *reinterpret_cast<uint4*>(ov + i) = *reinterpret_cast<const uint4*>(cv + i);
    }
    for (uint32_t i = n4 + tid; i < tile_n; i += kThreads) {
      ok[i] = ck[i];
      ov[i] = cv[i];
    }
    return;
  }

  // Cleanup: keep the first element of each key (the newest one, §IV-E) when
  // it is regular; compact across tiles.
  const uint32_t q0 = tid * kE;
  uint32_t keep = 0, nkeep = 0;
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const uint32_t q = q0 + e;
    if (q < tile_n) {
      const uint32_t kv = ck[q];
      const uint32_t prev = q ? key_of(ck[q - 1]) : s_prev_key;
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
      out_k[dst] = ck[q0 + e];
      out_v[dst] = cv[q0 + e];
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
        a.src, a.total, a.part, a.out_keys, a.out_vals, a.status, a.lookback, a.tile_ctr, a.out_count,
        uint32_t(ntiles));
  } else {
    count_launches(1);
    fold_merge<false><<<unsigned(ntiles), kThreads, kMergeSmem, st>>>(
        a.src, a.total, a.part, a.out_keys, a.out_vals, a.status, nullptr, nullptr, nullptr,
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

}  // namespace gpulsm
