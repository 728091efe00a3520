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
//   partition   one warp per output tile boundary p finds the co-rank vector
//               (how many elements of each source precede position p).  The
//               sources' prefix indexes (fences) give the bin holding the
//               p-th element: the lanes, in groups of one lane per source,
//               probe several bins of the bracket each round.  A bin of at
//               most 32 elements (the usual
//               case: about 8 per source) is loaded one element per lane and
//               ranked by (key, source rank, index); a crowded bin is
//               bisected over its key range instead, each lane keeping a
//               bracket in its own source, and the elements of the key found
//               are split among the sources in rank order.
//   merge       one tile per CTA: the k + 1 source segments are staged in
//               shared memory (16-byte aligned supersets starting one
//               element early), by TMA bulk copies for up to three sources
//               and by 16-byte cp.async copies from every thread for more; a
//               left-deep chain of merge-path merges in shared memory (ranks
//               0 and 1, then the result with rank 2, ...; ties to the lower
//               rank) builds the tile as key variables with the 16-bit
//               index of each element's window slot (6 bytes per element
//               instead of a key-value pair's 8), rewritten in place by
//               each step (one such buffer: six tiles fit per SM), the last
//               step keeping its outputs in registers and gathering their
//               values through the indices;
//               they are written out with 16-byte stores.  The plain fold
//               also writes the new level's prefix index.
// Cleanup uses the same two kernels over all full levels; the merge then keeps
// only the first element of every key when it is regular and compacts the
// survivors with a decoupled look-back scan across tiles.
//
// The batched form (many dictionaries, one batch each per round) runs the
// same partition and tile merge for every (instance, tile): a partition
// kernel over all boundaries of all instances and a persistent merge kernel
// whose CTAs take (instance, tile) work items from an atomic counter.
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

constexpr int kThreads = 256;
constexpr uint64_t kLbAgg = 1ull << 62, kLbIncl = 2ull << 62, kLbMask = (1ull << 62) - 1;

// Tile geometry for E outputs per thread per merge step.
template <int E>
struct TileGeom {
  static constexpr uint32_t kTile = kThreads * E;
  static constexpr uint32_t kSlotCap = (kTile + 8 * kMaxSources + 15) / 16 * 16;  // TMA slots + slack
  // a chain buffer: kTile keys (u32) + kTile slot indices (u16)
  static constexpr size_t kChainBytes = size_t(kTile) * (sizeof(uint32_t) + sizeof(uint16_t));
  static constexpr size_t kSmem = 2 * size_t(kSlotCap) * sizeof(uint32_t) + 2 * kChainBytes + 16;  // + kChainPad
};
// Bytes after the last chain buffer: a merge cursor one past a full tile's
// chain reads its 16-bit index there.
constexpr size_t kChainPad = 16;
constexpr int kFoldE = kFoldTile / kThreads;  // outputs per thread of the plain fold
static_assert(TileGeom<kFoldE>::kTile == kFoldTile, "the plain fold's tile");
// Slots of a plain-fold tile of S sources: the tile plus up to 8 elements a
// window (one before its co-rank, and alignment to 4 elements at both
// ends), a multiple of 16 elements.  Sized by S, a fold of up to eight
// sources fits seven CTAs per SM.
__host__ __device__ constexpr uint32_t plain_slot_cap(uint32_t S) { return (uint32_t(kFoldTile) + 8u * S + 15u) / 16u * 16u; }

// Element q of a chain buffer (32-bit keys, 16-bit indices) sits at index q.
// An XOR swizzle of the low bits (q ^ ((q >> 5) & 7), which gives the 32
// lanes of a warp writing 8 consecutive elements each 32 banks) cost more in
// index arithmetic than its bank conflicts: without it the k = 7 fold at
// b = 2^18 executes 233.8 instead of 250.9 M warp instructions, 269 instead
// of 278 us (the kernel is close to issue-bound).

// Number of elements of the sorted run a[0, n) whose key variable is below
// x, from its prefix index f at shift fs: one table entry when x starts one
// of its bins, else that bin's start plus a lower bound inside the bin
// (about 2^3 elements).
__device__ __forceinline__ uint32_t count_below(const uint32_t* a, const uint32_t* f, int fs, uint32_t n,
                                                uint32_t x) {
  const uint32_t P = x >> fs;
  const uint32_t lo = fence_at(f, fs, n, P);
  if ((x & ((1u << fs) - 1u)) == 0u) return lo;
  return lower_bound_kv(a, lo, fence_at(f, fs, n, P + 1), x);
}

// Largest bin P in [lo, hi) (at shift `shift`) with C(P) <= p, where C(P) =
// sum over the sources of count(P): the warp splits into G = 32 / S' groups
// of S' >= S lanes (lane j of a group reads source j, count(j, P) its count);
// each round the groups evaluate C at the points that split the bracket
// into G parts (2 for a single group) and the bracket shrinks to the part
// where C crosses p.  Requires C(lo) <= p < C(hi).
template <class Count>
__device__ __forceinline__ uint32_t group_search(uint32_t lo, uint32_t hi, uint64_t p, int lg, const Count& count) {
  const uint32_t lane = lane_id();
  const uint32_t G = 32u >> lg, q = lane >> lg;
  // at most log2(2^32) rounds; the bound only guards the loop
  for (int round = 0; hi - lo > 1 && round < 64; ++round) {
    const uint32_t span = hi - lo;
    uint32_t P;
    bool valid;
    if (span <= G) {
      P = lo + 1 + q;
      valid = P < hi;
    } else {  // probes split the bracket into max(G, 2) equal parts
      const int parts = lg < 5 ? 5 - lg : 1;
      P = lo + uint32_t((uint64_t(q + 1) * span) >> parts);
      valid = q + 1 < (1u << parts);
    }
    uint32_t c = valid ? count(P) : 0u;  // C(P) <= total < 2^32
    for (uint32_t o = (1u << lg) >> 1; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, int(o));
    // C is non-decreasing and the probes ascend with the group: a prefix
    const uint32_t j = lane & ((1u << lg) - 1u);
    const int cnt = __popc(__ballot_sync(0xffffffffu, j == 0 && valid && c <= p));
    const uint32_t p_lo = __shfl_sync(0xffffffffu, P, ((cnt + 31) & 31) << lg & 31);
    const uint32_t p_hi = __shfl_sync(0xffffffffu, P, (cnt << lg) & 31);
    const bool v_hi = __shfl_sync(0xffffffffu, valid, (cnt << lg) & 31);
    if (cnt > 0) lo = p_lo;
    if (uint32_t(cnt) < G && v_hi) hi = p_hi;
  }
  return lo;
}

// This lane's co-rank at output position p < total (warp-collective; lane j
// holds source j when act, the active lanes being 0 .. S-1).
__device__ __forceinline__ uint32_t corank_lane(bool act, const uint32_t* a, const uint32_t* f, int fs,
                                                uint32_t n, uint64_t p, uint64_t total) {
  const uint32_t lane = lane_id();
  const int S = __popc(__ballot_sync(0xffffffffu, act));
  // The first search runs at the coarsest of the sources' prefix-index
  // resolutions (shift fc), which every source's table answers with one
  // load; a crowded bin there is searched again at the finest (fm).
  int fc = act ? fs : 0, fm = act ? fs : 32;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fc = max(fc, __shfl_xor_sync(0xffffffffu, fc, o));
    fm = min(fm, __shfl_xor_sync(0xffffffffu, fm, o));
  }
  const int cs = act ? fc - fs : 0;
  uint32_t bmin = 0, bmax = 0;
  if (act) {
    bmin = __ldg(f + fence_bins(fs) + 2);
    bmax = __ldg(f + fence_bins(fs) + 3);
  }
  int lg = 0;
  while ((1 << lg) < S) ++lg;
  const uint32_t j = lane & ((1u << lg) - 1u);
  const bool jact = j < uint32_t(S);
  const uint32_t* fj = reinterpret_cast<const uint32_t*>(
      __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(f), int(j)));
  const uint32_t* aj = reinterpret_cast<const uint32_t*>(
      __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(a), int(j)));
  const int csj = __shfl_sync(0xffffffffu, cs, int(j));
  const uint32_t bminj = __shfl_sync(0xffffffffu, bmin, int(j)), bmaxj = __shfl_sync(0xffffffffu, bmax, int(j));
  const uint32_t nj = __shfl_sync(0xffffffffu, n, int(j));
  // 1. The bin at shift fc: largest P with C(P) <= p (C(0) = 0 <= p <
  //    C(nbins) = total).  First a bracket of 2 delta bins around the
  //    proportional guess over the sources' populated bin range (exact for
  //    evenly spread keys), checked with one probe at each end; the search
  //    runs inside it when it holds the answer, else over all bins.
  auto coarse = [&](uint32_t P) -> uint32_t {
    if (!jact) return 0u;
    const uint32_t Pj = P << csj;
    // an entry inside the populated range is always loaded, then selected
    const uint32_t v = __ldg(fj + (Pj <= bminj ? bminj : (Pj > bmaxj ? bmaxj : Pj)));
    return Pj <= bminj ? 0u : (Pj > bmaxj ? nj : min(v, nj));
  };
  const uint32_t nbins = 1u << (32 - fc);
  uint32_t rlo = act ? (bmin >> cs) : 0xFFFFFFFFu, rhi = act ? (bmax >> cs) : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rlo = min(rlo, __shfl_xor_sync(0xffffffffu, rlo, o));
    rhi = max(rhi, __shfl_xor_sync(0xffffffffu, rhi, o));
  }
  const uint32_t guess = rlo + uint32_t((p * uint64_t(rhi - rlo + 1u)) / total);
  // half-width 1/2048 of the bins: for evenly spread keys the guess is off by
  // a few bins (the spread of a count is about its square root); a bracket
  // that misses costs one round more than a full search
  const uint32_t delta = max(8u, nbins >> 11);
  const uint32_t lo0 = guess > delta ? guess - delta : 0u;
  const uint32_t hi0 = (nbins - guess) > delta ? guess + delta : nbins;
  // C(lo0) by group 0 and C(hi0) by group 1 in one round (a warp of a
  // single group, S > 16, takes two)
  uint32_t c_lo = 0, c_hi = 0;
  for (int e = 0; e < (lg < 5 ? 1 : 2); ++e) {
    const uint32_t q = lg < 5 ? (lane >> lg) : uint32_t(e);
    uint32_t c = q < 2 && (lg < 5 || e == int(q)) ? coarse(q ? hi0 : lo0) : 0u;
    for (uint32_t o = (1u << lg) >> 1; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, int(o));
    if (lg < 5) {
      c_lo = __shfl_sync(0xffffffffu, c, 0);
      c_hi = __shfl_sync(0xffffffffu, c, int(1u << lg));
    } else if (e == 0) {
      c_lo = __shfl_sync(0xffffffffu, c, 0);
    } else {
      c_hi = __shfl_sync(0xffffffffu, c, 0);
    }
  }
  const bool inside = c_lo <= p && p < c_hi;
  uint32_t bin = group_search(inside ? lo0 : 0u, inside ? hi0 : nbins, p, lg, coarse);
  int bs = fc;  // shift of the bin found
  // 2. The bin's elements: [blo, bhi) of each source, need = p - C(bin) of
  //    them precede p.
  uint32_t blo = act ? fence_at(f, fs, n, bin << cs) : 0u, bhi = act ? fence_at(f, fs, n, (bin + 1) << cs) : 0u;
  if (warp_sum(bhi - blo) > 32u && fm < fc) {
    // A crowded bin at fc: its 2^(fc - fm) bins at the finest shift fm,
    // counted with count_below (a table entry, or a short search inside a
    // coarser source's bin).
    const int d = fc - fm;
    const int fsj = fc - csj;
    bin = group_search(bin << d, (bin + 1) << d, p, lg, [&](uint32_t P) -> uint32_t {
      return jact ? count_below(aj, fj, fsj, nj, P << fm) : 0u;
    });
    bs = fm;
    blo = act ? count_below(a, f, fs, n, bin << fm) : 0u;
    const uint32_t nb_fm = 1u << (32 - fm);
    bhi = act ? (bin + 1 < nb_fm ? count_below(a, f, fs, n, (bin + 1) << fm) : n) : 0u;
  }
  const uint32_t cnt = bhi - blo;
  const uint32_t tot = warp_sum(cnt);
  const uint64_t need = p - warp_sum<uint64_t>(blo);
  if (tot <= 32) {
    // One element per lane in source order (which is the tie order); its
    // rank in the bin by (key, lane) says whether it precedes p.
    const uint32_t off = warp_incl_scan(cnt) - cnt;
    int jj = 0;
    for (int q = 0; q < S; ++q)
      if (lane >= __shfl_sync(0xffffffffu, off + cnt, q)) jj = q + 1;
    const bool has = lane < tot;
    const uint32_t* ajj = reinterpret_cast<const uint32_t*>(
        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(a), jj & 31));
    const uint32_t offj = __shfl_sync(0xffffffffu, off, jj & 31), bloj = __shfl_sync(0xffffffffu, blo, jj & 31);
    const uint32_t key = has ? key_of(__ldg(ajj + bloj + (lane - offj))) : 0xFFFFFFFFu;
    uint32_t rank = 0;
    for (uint32_t q = 0; q < tot; ++q) {
      const uint32_t kq = __shfl_sync(0xffffffffu, key, q);
      rank += (kq < key || (kq == key && q < lane)) ? 1u : 0u;
    }
    const uint32_t before = __ballot_sync(0xffffffffu, has && rank < need);
    const uint32_t mask = cnt ? ((cnt >= 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u)) << off) : 0u;
    return blo + uint32_t(__popc(before & mask));
  }
  // A crowded bin (many equal or close keys): smallest key x in the bin
  // with #{key <= x} > p by bisection over the bin's key range.
  // Invariant per lane: blo = #{key <= xlo - 1}, bhi = #{key <= xhi} in
  // this lane's source.  A bin at shift bs holds the keys
  // [P << (bs - 1), (P + 1) << (bs - 1)).
  uint32_t xlo = bin << (bs - 1), xhi = ((bin + 1) << (bs - 1)) - 1;
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
  const uint32_t kc = bhi - blo;
  const uint64_t kneed = p - warp_sum<uint64_t>(blo);
  const uint64_t excl = warp_incl_scan<uint64_t>(kc) - kc;
  uint64_t take = 0;
  if (kneed > excl) take = (kneed - excl) < kc ? (kneed - excl) : kc;
  return blo + uint32_t(take);
}

__global__ void __launch_bounds__(256) fold_partition(FoldSources src, uint64_t total, uint32_t ntiles,
                                                      uint32_t tile, uint32_t* __restrict__ part) {
  // No early trigger: the merge's CTAs are launched at this kernel's exit,
  // instead of waiting on SMs (and holding their shared memory) through the
  // whole search (insert phase at b = 2^20: 8.03 -> 7.96 ms).
  pdl_wait();
  const uint32_t t = (blockIdx.x * 256u + threadIdx.x) >> 5;
  if (t > ntiles) return;  // whole warp leaves together
  const uint32_t lane = lane_id();
  const int S = src.count;
  const bool act = lane < uint32_t(S);
  const uint32_t n = act ? src.n[lane] : 0u;
  const uint64_t p = uint64_t(t) * tile < total ? uint64_t(t) * tile : total;
  uint32_t* out = part + uint64_t(t) * S;
  if (p >= total) {
    if (act) out[lane] = n;
    return;
  }
  const uint32_t c = corank_lane(act, act ? src.keys[lane] : nullptr, act ? src.fence[lane] : nullptr,
                                 act ? src.fshift[lane] : 16, n, p, total);
  if (act) out[lane] = c;
}

// Source j of instance `in`'s fold into level k: the sorted batch (j = 0),
// then levels 0 .. k - 1.
__device__ __forceinline__ void multi_source(const MultiArena& ar, const MultiInst& in, int j,
                                             const uint32_t*& keys, const uint32_t*& vals, const uint32_t*& fence,
                                             uint32_t& n, int& fshift) {
  if (j == 0) {
    keys = ar.bkeys + in.boff;
    vals = ar.bvals + in.boff;
    fence = ar.fence + in.batch_fence;
    n = in.b;
    fshift = in.fshift0;
  } else {
    keys = ar.keys + in.lvl_off[j - 1];
    vals = ar.vals + in.lvl_off[j - 1];
    fence = ar.fence + in.lvl_fence[j - 1];
    n = in.b << (j - 1);
    fshift = in.lvl_fshift[j - 1];
  }
}

// Co-ranks of every tile boundary of every instance that folds this round
// (one warp per boundary, grid-stride over part_prefix[n] boundaries).
__global__ void __launch_bounds__(256) multi_partition(MultiArena ar) {
  const uint32_t lane = lane_id();
  const uint64_t total_items = *reinterpret_cast<volatile const uint64_t*>(ar.part_prefix + ar.n);
  const uint64_t nwarps = uint64_t(gridDim.x) * 8u;
  for (uint64_t w = (uint64_t(blockIdx.x) * 256u + threadIdx.x) >> 5; w < total_items; w += nwarps) {
    const uint32_t i = find_instance(ar.part_prefix, ar.n, w);
    const MultiInst& in = ar.inst[i];
    const int k = ar.k[i];
    const uint32_t t = uint32_t(w - ar.part_prefix[i]);
    const int S = k + 1;
    const bool act = lane < uint32_t(S);
    const uint32_t *keys = nullptr, *vals = nullptr, *fence = nullptr;
    uint32_t n = 0;
    int fs = 16;
    if (act) multi_source(ar, in, int(lane), keys, vals, fence, n, fs);
    const uint64_t total = uint64_t(in.b) << k;
    const uint64_t p = uint64_t(t) * in.tile < total ? uint64_t(t) * in.tile : total;
    uint32_t* out = ar.part + w * kMultiPartStride;
    if (p >= total) {
      if (act) out[lane] = n;
      continue;
    }
    const uint32_t c = corank_lane(act, keys, fence, fs, n, p, total);
    if (act) out[lane] = c;
  }
}

// One merge step of the tile: output[0, nA + nB) = merge of run A (the
// newer ranks) and run B (the next rank), ties to A.  B always sits in the
// staged windows (separate key and value arrays, the slots); A is either
// there too (the first step) or the chain buffer X written by the step
// before: key variables Xk and the 16-bit slot index Xi of each element.
// Thread t produces `per` consecutive outputs from per * t after a
// merge-path search for its first one (threads past the end idle); the
// outputs go to the chain buffer Y (key and slot index), or stay in
// registers (kToRegs, per = E) when this is the last step, which then reads
// each output's value from its slot.  An intermediate step spreads its
// m outputs over all threads (per = ceil(m / threads)), so the short early
// steps of the chain cost one or two outputs per thread instead of E.
// Keys are compared as key variables: key(a) <= key(b) exactly when
// a <= (b | 1), the status bit being the lowest.
template <int E, bool kAFromSlot, bool kToRegs>
__device__ __forceinline__ void merge_step(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                                           const uint32_t* __restrict__ Xk, const uint16_t* __restrict__ Xi,
                                           uint32_t* __restrict__ Yk, uint16_t* __restrict__ Yi, uint32_t aS,
                                           uint32_t nA, uint32_t bS, uint32_t nB, uint2 (&out)[E]) {
  const uint32_t m = nA + nB;
  const uint32_t per = kToRegs ? uint32_t(E) : (m + kThreads - 1) / kThreads;
  const uint32_t q0 = threadIdx.x * per;
  if (q0 >= m) return;
  auto keyA = [&](uint32_t i) { return kAFromSlot ? sk[aS + i] : Xk[i]; };
  auto idxA = [&](uint32_t i) { return kAFromSlot ? aS + i : uint32_t(Xi[i]); };
  // merge path: how many of the first q0 outputs come from A
  uint32_t lo = q0 > nB ? q0 - nB : 0u, hi = q0 < nA ? q0 : nA;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (keyA(mid) <= (sk[bS + q0 - 1 - mid] | 1u)) lo = mid + 1; else hi = mid;
  }
  // Branch-free walk: after every output both heads are reloaded from their
  // cursors, and a run past its end is never taken.  A cursor at most one past
  // its run's end reads a word that is garbage but in bounds: the slots hold
  // the windows' slack, the values follow the keys, and the launch adds
  // kChainPad bytes after the last chain buffer.  A data-dependent branch on
  // which run advanced would make every warp execute both sides.
  uint32_t ia = lo, ib = q0 - lo;
  uint32_t va = keyA(ia), xa = idxA(ia), vb = sk[bS + ib], xb = bS + ib;   // key variable, slot index
  // one output: the smaller head (the newer run's on equal keys), then both
  // heads reloaded
  auto emit = [&](uint32_t e, uint2& o) {
    const bool take_a = ia < nA && (ib >= nB || va <= (vb | 1u));
    const uint32_t v = take_a ? va : vb, x = take_a ? xa : xb;
    if (kToRegs) {
      o = make_uint2(v, x);   // the value is gathered by slot index after the step
    } else {
      Yk[q0 + e] = v;
      Yi[q0 + e] = uint16_t(x);
    }
    ia += take_a ? 1u : 0u;
    ib += take_a ? 0u : 1u;
    va = keyA(ia);
    xa = idxA(ia);
    vb = sk[bS + ib];
    xb = bS + ib;
  };
  if (kToRegs) {
    if (q0 + E <= m) {  // a full thread (all but the ragged end of the last tile): no guards
#pragma unroll
      for (int e = 0; e < E; ++e) emit(uint32_t(e), out[e]);
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (q0 + e < m) emit(uint32_t(e), out[e]);
    }
  } else {
    // an intermediate step has per <= E outputs per thread, most often one
    // or two: a loop over exactly those (an unrolled loop over E guarded
    // per output issued more instructions: at b = 2^20 the k = 7 fold took
    // 1.52 instead of 1.42 ms)
    const uint32_t cnt = (m - q0) < per ? (m - q0) : per;
    uint2 unused;
#pragma unroll 2
    for (uint32_t e = 0; e < cnt; ++e) emit(e, unused);
  }
  if (kToRegs) {
    if (q0 + E <= m) {
#pragma unroll
      for (int e = 0; e < E; ++e) out[e].y = sv[out[e].y];
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (q0 + e < m) out[e].y = sv[out[e].y];
    }
  }
}

// An intermediate merge step in place: X[0, nA + nB) = merge of X[0, nA)
// (the newer ranks) and run B of the slots, ties to X.  Each thread's
// outputs (at most E) go to registers first and are written back after a
// CTA barrier, once every thread has read X; so the tile needs one chain
// buffer instead of two, and six CTAs of the plain fold fit on an SM instead
// of five (k = 7 fold at b = 2^20: 1.39 -> 1.31 ms).  The outputs are
// emitted by a loop of exactly the thread's count (a switch over the eight
// counts), not by a loop over E guarded per output.  Every thread of the
// CTA must call it.
template <int N, int E, class Emit>
__device__ __forceinline__ void emit_n(const Emit& emit, uint2 (&o)[E]) {
#pragma unroll
  for (int e = 0; e < N; ++e) emit(uint32_t(e), o[e]);
}
template <int N, int E>
__device__ __forceinline__ void store_n(uint32_t* Xk, uint16_t* Xi, uint32_t q0, const uint2 (&o)[E]) {
#pragma unroll
  for (int e = 0; e < N; ++e) {
    Xk[q0 + e] = o[e].x;
    Xi[q0 + e] = uint16_t(o[e].y);
  }
}
template <int E>
__device__ __forceinline__ void merge_step_inplace(const uint32_t* __restrict__ sk, uint32_t* __restrict__ Xk,
                                                   uint16_t* __restrict__ Xi, uint32_t nA, uint32_t bS,
                                                   uint32_t nB) {
  static_assert(E == 8, "the switches below cover one to eight outputs");
  const uint32_t m = nA + nB;
  // at least two outputs a thread: half the searches of the shortest steps
  // for one output more of latency (k = 7 fold at b = 2^18: 268.6 -> 266.2
  // us; four outputs: 272.2 us)
  uint32_t per = (m + kThreads - 1) / kThreads;  // <= E: m is at most a tile
  if (per < 2u) per = 2u;
  const uint32_t q0 = threadIdx.x * per;
  const uint32_t cnt = q0 < m ? ((m - q0) < per ? (m - q0) : per) : 0u;
  uint2 o[E];
  if (cnt) {
    uint32_t lo = q0 > nB ? q0 - nB : 0u, hi = q0 < nA ? q0 : nA;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (Xk[mid] <= (sk[bS + q0 - 1 - mid] | 1u)) lo = mid + 1; else hi = mid;
    }
    uint32_t ia = lo, ib = q0 - lo;
    uint32_t va = Xk[ia], xa = Xi[ia], vb = sk[bS + ib], xb = bS + ib;
    auto emit = [&](uint32_t, uint2& r) {
      const bool take_a = ia < nA && (ib >= nB || va <= (vb | 1u));
      r = make_uint2(take_a ? va : vb, take_a ? xa : xb);
      ia += take_a ? 1u : 0u;
      ib += take_a ? 0u : 1u;
      va = Xk[ia];
      xa = Xi[ia];
      vb = sk[bS + ib];
      xb = bS + ib;
    };
    switch (cnt) {
      case 1: emit_n<1, E>(emit, o); break;
      case 2: emit_n<2, E>(emit, o); break;
      case 3: emit_n<3, E>(emit, o); break;
      case 4: emit_n<4, E>(emit, o); break;
      case 5: emit_n<5, E>(emit, o); break;
      case 6: emit_n<6, E>(emit, o); break;
      case 7: emit_n<7, E>(emit, o); break;
      default: emit_n<E, E>(emit, o); break;
    }
  }
  __syncthreads();
  switch (cnt) {
    case 0: break;
    case 1: store_n<1, E>(Xk, Xi, q0, o); break;
    case 2: store_n<2, E>(Xk, Xi, q0, o); break;
    case 3: store_n<3, E>(Xk, Xi, q0, o); break;
    case 4: store_n<4, E>(Xk, Xi, q0, o); break;
    case 5: store_n<5, E>(Xk, Xi, q0, o); break;
    case 6: store_n<6, E>(Xk, Xi, q0, o); break;
    case 7: store_n<7, E>(Xk, Xi, q0, o); break;
    default: store_n<E, E>(Xk, Xi, q0, o); break;
  }
}

// Shared state of the tile merge (static shared memory of the kernels).
struct MergeShared {
  uint32_t rstart[kMaxSources], rlen[kMaxSources];
  uint32_t a0[kMaxSources], span[kMaxSources], slot[kMaxSources];
  uint32_t scan[kThreads / 32], last[kThreads / 32];
  uint32_t prev_mask, ok, ngap, landed, prev0;
  FenceGap gaps[kFenceGapSlots];
  uint64_t prefix;
};

// From this many sources a tile stages its windows with 16-byte cp.async
// copies from every thread rather than bulk copies (at b = 2^20 the k = 7
// fold took 1.49 instead of 1.69 ms; folds of two or three sources, a few
// bulk copies each, gained nothing).
constexpr int kVecStageSources = 4;

// Merge tile `tile` of a fold whose sources are `src` (rank order), whose
// co-ranks are part[tile * pstride + j] .. part[(tile + 1) * pstride + j],
// into out_k/out_v.  `bar` is an initialised mbarrier and `phase` the number
// of its phases completed so far (a tile staged with bulk copies completes
// one and advances it).  Returns false if a copy never arrived (the CTA must
// then stop).  Called by all threads of the CTA.
template <int E, bool kCleanup, bool kInPlace>
__device__ __forceinline__ bool merge_tile(const FoldSources& src, uint64_t total, const uint32_t* __restrict__ part,
                                           uint32_t pstride, uint32_t tile, uint32_t ntiles, uint32_t* __restrict__ out_k,
                                           uint32_t* __restrict__ out_v, uint32_t* __restrict__ out_fence,
                                           int fshift, uint32_t* status, uint64_t* lookback, uint64_t* out_count,
                                           uint32_t* sm, MergeShared& sh, uint64_t* bar, uint32_t& phase) {
  using G = TileGeom<E>;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const int S = src.count;
  const uint64_t obase = uint64_t(tile) * G::kTile;
  const uint32_t tile_n = uint32_t((total - obase) < G::kTile ? (total - obase) : G::kTile);
  uint32_t* sk = sm;                                           // slot keys
  // the plain fold sizes its slots by its source count (the launch's shared
  // memory does the same: plain_slot_cap), the batched form for any count
  const uint32_t cap = kInPlace ? plain_slot_cap(uint32_t(S)) : G::kSlotCap;
  uint32_t* sv = sm + cap;                                     // slot values
  // chain buffers X and Y: kTile keys, then kTile 16-bit slot indices each
  uint32_t* Xk = sm + 2 * cap;
  uint16_t* Xi = reinterpret_cast<uint16_t*>(Xk + G::kTile);
  uint32_t* Yk = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(Xk) + G::kChainBytes);
  uint16_t* Yi = reinterpret_cast<uint16_t*>(Yk + G::kTile);

  // Segment of each source in this tile, and its 16-byte aligned superset.
  // The copy window starts one element early when there is one: the key
  // just before the tile in merged order (the largest key among the
  // sources' elements before their co-ranks) is then read from shared
  // memory instead of by a dependent global load before the copies.
  if (warp == 0) {
    uint32_t c0 = 0, c1 = 0, a0 = 0, span = 0;
    if (lane < uint32_t(S)) {
      c0 = part[uint64_t(tile) * pstride + lane];
      c1 = part[uint64_t(tile + 1) * pstride + lane];
      const uint32_t lo = c0 > 0 ? c0 - 1 : 0u;
      if (c1 > lo) {
        a0 = lo & ~3u;
        span = ((c1 + 3u) & ~3u) - a0;
      }
    }
    const uint32_t slot = warp_incl_scan(span) - span;
    if (lane < uint32_t(S)) {
      sh.rstart[lane] = slot + (c0 - a0);
      sh.rlen[lane] = c1 - c0;
      sh.a0[lane] = a0;
      sh.span[lane] = span;
      sh.slot[lane] = slot;
    }
    const uint32_t pm = __ballot_sync(0xffffffffu, lane < uint32_t(S) && c0 > 0);
    // every window 16-byte aligned (so by construction: level and buffer
    // starts are multiples of 32 elements); otherwise plain loads
    bool al = true;
    if (span)
      al = ((reinterpret_cast<uintptr_t>(src.keys[lane] + a0) | reinterpret_cast<uintptr_t>(src.vals[lane] + a0)) &
            15u) == 0;
    const bool ok = __all_sync(0xffffffffu, al);
    if (lane == 0) {
      sh.prev_mask = pm;
      sh.ngap = 0;
      sh.ok = ok ? 1u : 0u;
      if (!ok) atomicOr(status, kErrAlign);
    }
  }
  __syncthreads();

  if (S >= kVecStageSources && sh.ok) {
    // Many sources: 16-byte asynchronous copies issued by every thread (two
    // to three per thread and array, all in flight at once) stage the
    // windows faster than one bulk copy per source and array, which the
    // copy engine serves one after another.
    const uint32_t chunks = (sh.slot[S - 1] + sh.span[S - 1]) >> 2;
    int r = 0;
    for (uint32_t u = tid; u < chunks; u += kThreads) {
      const uint32_t w = u * 4u;
      while (w >= sh.slot[r] + sh.span[r]) ++r;
      const uint32_t off = sh.a0[r] + (w - sh.slot[r]);
      cp_async16(sk + w, src.keys[r] + off);
      cp_async16(sv + w, src.vals[r] + off);
    }
    cp_async_wait_all();
    __syncthreads();
  } else {
    // Stage the segments with the TMA engine (one thread issues and waits);
    // this completes one phase of the CTA's mbarrier.
    const uint32_t parity = phase & 1u;
    ++phase;
    if (tid == 0) {
      uint32_t bytes = 0;
      const bool ok = sh.ok != 0;
      for (int r = 0; r < S; ++r) bytes += 2u * sh.span[r] * 4u;
      if (!ok) bytes = 0;
      mbar_arrive_expect_tx(bar, bytes);
      if (ok) {
        for (int r = 0; r < S; ++r) {
          if (!sh.span[r]) continue;
          bulk_g2s(sk + sh.slot[r], src.keys[r] + sh.a0[r], sh.span[r] * 4u, bar);
          bulk_g2s(sv + sh.slot[r], src.vals[r] + sh.a0[r], sh.span[r] * 4u, bar);
        }
      }
      // One thread waits for the copies (bounded); the barrier below then
      // releases the CTA, so the other threads do not spin on the mbarrier.
      sh.landed = mbar_wait_bounded(bar, parity, status) ? 1u : 0u;
    }
    __syncthreads();
    const bool landed = sh.landed != 0;
    // each thread acquires the completed phase itself (returns at once)
    if (landed) mbar_try_wait(bar, parity);
    if (!sh.ok) {  // never expected: plain loads instead of the bulk copies
      for (int r = 0; r < S; ++r)
        for (uint32_t i = tid; i < sh.span[r]; i += kThreads) {
          sk[sh.slot[r] + i] = __ldg(src.keys[r] + sh.a0[r] + i);
          sv[sh.slot[r] + i] = __ldg(src.vals[r] + sh.a0[r] + i);
        }
      __syncthreads();
    }
    if (!__syncthreads_and(landed)) {
      // A copy never completed; give it one more bounded wait before leaving
      // so that no transfer lands in shared memory after this CTA is gone.
      if (tid == 0) mbar_wait_bounded(bar, parity, status);
      return false;
    }
  }

  // The element before the tile (for thread 0): only its key (and so its
  // bin) matters; a key variable with the largest key before the co-ranks
  // (lane j of warp 0 reads source j's element before its co-rank).
  if (warp == 0) {
    const bool has = lane < uint32_t(S) && ((sh.prev_mask >> lane) & 1u);
    uint32_t mx = has ? key_of(sk[sh.rstart[lane] - 1]) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) sh.prev0 = mx << 1;
  }
  __syncthreads();
  const uint32_t prev0 = sh.prev0;

  // Left-deep merge order: X = run 0 + run 1, then X = X + run r for each
  // further rank; the last step keeps its E outputs per thread in registers.
  // Runs grow with their rank (the batch and level 0 are the smallest), so
  // every element moves about twice in all.  The plain fold (kInPlace)
  // rewrites X in place; the batched form alternates between X and Y.
  uint2 out[E];
  if (S <= 2) {
    merge_step<E, true, true>(sk, sv, nullptr, nullptr, nullptr, nullptr, sh.rstart[0], sh.rlen[0],
                              S == 2 ? sh.rstart[1] : 0u, S == 2 ? sh.rlen[1] : 0u, out);
  } else {
    merge_step<E, true, false>(sk, sv, nullptr, nullptr, Xk, Xi, sh.rstart[0], sh.rlen[0], sh.rstart[1],
                               sh.rlen[1], out);
    uint32_t m = sh.rlen[0] + sh.rlen[1];
    for (int r = 2; r < S - 1; ++r) {
      __syncthreads();
      if constexpr (kInPlace) {
        merge_step_inplace<E>(sk, Xk, Xi, m, sh.rstart[r], sh.rlen[r]);
        m += sh.rlen[r];
        continue;
      }
      merge_step<E, false, false>(sk, sv, Xk, Xi, Yk, Yi, 0u, m, sh.rstart[r], sh.rlen[r], out);
      m += sh.rlen[r];
      uint32_t* tk = Xk;
      Xk = Yk;
      Yk = tk;
      uint16_t* ti = Xi;
      Xi = Yi;
      Yi = ti;
    }
    __syncthreads();
    merge_step<E, false, true>(sk, sv, Xk, Xi, nullptr, nullptr, 0u, m, sh.rstart[S - 1], sh.rlen[S - 1], out);
  }
  // Outputs q0 .. q0 + cnt - 1 are in out[]; the key before q0 in merged
  // order comes from the thread before (a shuffle, or across warps through
  // shared memory), or from before the tile.
  const uint32_t q0 = tid * E;
  const uint32_t cnt = q0 < tile_n ? ((tile_n - q0) < uint32_t(E) ? (tile_n - q0) : uint32_t(E)) : 0u;
  uint32_t last = 0;
#pragma unroll
  for (int e = 0; e < E; ++e)
    if (uint32_t(e) < cnt) last = out[e].x;
  uint32_t prev_kv = __shfl_up_sync(0xffffffffu, last, 1);
  if (lane == 31) sh.last[warp] = last;
  __syncthreads();
  if (lane == 0 && warp > 0) prev_kv = sh.last[warp - 1];
  const bool has_prev = tid > 0 || sh.prev_mask != 0;
  if (tid == 0) prev_kv = prev0;

  if (!kCleanup) {
    if (cnt == uint32_t(E) && (E % 4) == 0 &&
        ((reinterpret_cast<uintptr_t>(out_k + obase + q0) | reinterpret_cast<uintptr_t>(out_v + obase + q0)) &
         15u) == 0) {
      uint4* ok4 = reinterpret_cast<uint4*>(out_k + obase + q0);
      uint4* ov4 = reinterpret_cast<uint4*>(out_v + obase + q0);
#pragma unroll
      for (int c = 0; c < E / 4; ++c) {
        ok4[c] = make_uint4(out[4 * c].x, out[4 * c + 1].x, out[4 * c + 2].x, out[4 * c + 3].x);
        ov4[c] = make_uint4(out[4 * c].y, out[4 * c + 1].y, out[4 * c + 2].y, out[4 * c + 3].y);
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e)
        if (uint32_t(e) < cnt) {
          out_k[obase + q0 + e] = out[e].x;
          out_v[obase + q0 + e] = out[e].y;
        }
    }
    if (out_fence) {
      // Prefix index of the new level: the element at position pos owns the
      // entries between the previous element's bin and its own; the first and
      // last elements record the populated bin range instead of the edges.
      // At about 8 elements per bin an output crosses one bin boundary or
      // none, so every output writes at most the entry after the previous
      // bin (one predicated store, no branch a warp would diverge on); a
      // thread that met a wider gap (empty bins) writes the rest of its
      // gaps afterwards.
      const uint32_t nb = fence_bins(fshift);
      const uint32_t pb0 = has_prev ? fence_bin(prev_kv, fshift) : 0u;
      const bool level_start = obase + q0 == 0;  // this thread holds the level's first element
      uint32_t pb = pb0;
      bool wide = false;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if (uint32_t(e) < cnt) {
          const uint32_t bin = fence_bin(out[e].x, fshift);
          const uint32_t pos = uint32_t(obase) + q0 + uint32_t(e);
          const bool first = e == 0 && level_start;
          if (first) out_fence[nb + 2] = bin;
          if (!first && bin > pb) {
            out_fence[pb + 1] = pos;
            wide |= bin > pb + 1;
          }
          pb = bin;
        }
      }
      if (wide) {
        uint32_t qb = pb0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (uint32_t(e) < cnt) {
            const uint32_t bin = fence_bin(out[e].x, fshift);
            const uint64_t pos = obase + q0 + e;
            if (pos != 0 && bin > qb + 1) fence_write_gap(out_fence, qb + 1, bin, uint32_t(pos), sh.gaps, &sh.ngap);
            qb = bin;
          }
        }
      }
      if (cnt && obase + q0 + cnt == total) out_fence[nb + 3] = pb;
      __syncthreads();
      fence_fill_gaps(out_fence, sh.gaps, sh.ngap);
    }
    return true;
  }

  // Cleanup: keep the first element of each key (the newest one, §IV-E) when
  // it is regular; compact across tiles.
  uint32_t keep = 0, nkeep = 0;
  uint32_t pk = has_prev ? key_of(prev_kv) : 0xFFFFFFFFu;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (uint32_t(e) < cnt) {
      const uint32_t kv = out[e].x;
      if (key_of(kv) != pk && (kv & 1u)) {
        keep |= 1u << e;
        ++nkeep;
      }
      pk = key_of(kv);
    }
  }
  uint32_t tile_keep;
  const uint32_t before = block_excl_scan<kThreads>(nkeep, sh.scan, tile_keep);
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
          if (!spin_continue(t0, kWaitLimitNs, status)) break;
          continue;
        }
        prefix += w & kLbMask;
        if (w & kLbIncl) break;
        --t;
      }
      st_relaxed_u64(lookback + tile, kLbIncl | (prefix + tile_keep));
    }
    sh.prefix = prefix;
    if (tile == ntiles - 1) *out_count = prefix + tile_keep;
  }
  __syncthreads();
  uint64_t dst = sh.prefix + before;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (keep & (1u << e)) {
      out_k[dst] = out[e].x;
      out_v[dst] = out[e].y;
      ++dst;
    }
  }
  return true;
}

// Seven CTAs per SM: 32 registers a thread (a few bytes of spill) and, for
// folds of up to eight sources, 29 KB of shared memory a CTA (k = 7 fold at
// b = 2^20: 1.258 ms, against 1.316 ms at six CTAs and 40 registers).
template <bool kCleanup>
__global__ void __launch_bounds__(kThreads, 7) fold_merge(FoldSources src, uint64_t total,
                                                          const uint32_t* __restrict__ part,
                                                          uint32_t* __restrict__ out_k,
                                                          uint32_t* __restrict__ out_v,
                                                          uint32_t* __restrict__ out_fence, int fshift,
                                                          uint32_t* status, uint64_t* lookback, uint32_t* tile_ctr,
                                                          uint64_t* out_count, uint32_t ntiles) {
  extern __shared__ __align__(128) uint32_t sm[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ MergeShared sh;
  __shared__ uint32_t s_tile;
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x == 0) {
    s_tile = kCleanup ? atomicAdd(tile_ctr, 1u) : blockIdx.x;
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;
  merge_tile<kFoldE, kCleanup, true>(src, total, part, uint32_t(src.count), s_tile, ntiles, out_k, out_v, out_fence,
                               fshift, status, lookback, out_count, sm, sh, &s_bar, phase);
}

// Persistent merge for every (instance, tile) of a round: each CTA takes
// work items from an atomic counter until none is left.  An instance's tile
// size (1024 or 2048 outputs) selects the tile code per item.
__global__ void __launch_bounds__(kThreads, 4) multi_merge(MultiArena ar) {
  extern __shared__ __align__(128) uint32_t sm[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ MergeShared sh;
  __shared__ FoldSources s_src;
  __shared__ uint64_t s_item;
  __shared__ uint32_t s_inst;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  const uint64_t total_items = *reinterpret_cast<volatile const uint64_t*>(ar.tile_prefix + ar.n);
  uint32_t phase = 0;  // completed phases of s_bar (the same in every thread)
  for (;;) {
    __syncthreads();  // the previous item is finished with the shared state
    if (threadIdx.x == 0) {
      const uint64_t w = atomicAdd(ar.work_ctr, 1u);
      s_item = w;
      if (w < total_items) s_inst = find_instance(ar.tile_prefix, ar.n, w);
    }
    __syncthreads();
    const uint64_t w = s_item;
    if (w >= total_items) break;
    const uint32_t i = s_inst;
    const MultiInst& in = ar.inst[i];
    const int k = ar.k[i];
    const int S = k + 1;
    if (threadIdx.x < uint32_t(S)) {
      const uint32_t *kk = nullptr, *v = nullptr, *f = nullptr;
      uint32_t n = 0;
      int fs = 16;
      multi_source(ar, in, int(threadIdx.x), kk, v, f, n, fs);
      s_src.keys[threadIdx.x] = kk;
      s_src.vals[threadIdx.x] = v;
      s_src.fence[threadIdx.x] = f;
      s_src.n[threadIdx.x] = n;
      s_src.fshift[threadIdx.x] = fs;
    }
    if (threadIdx.x == 0) s_src.count = S;
    __syncthreads();
    const uint64_t total = uint64_t(in.b) << k;
    const uint32_t t = uint32_t(w - ar.tile_prefix[i]);
    const uint32_t ntiles = uint32_t(ar.tile_prefix[i + 1] - ar.tile_prefix[i]);
    const uint32_t* part = ar.part + ar.part_prefix[i] * kMultiPartStride;
    uint32_t* ok = ar.keys + in.lvl_off[k];
    uint32_t* ov = ar.vals + in.lvl_off[k];
    uint32_t* of = ar.fence + in.lvl_fence[k];
    const int fs = in.lvl_fshift[k];
    const bool done =
        in.tile == TileGeom<4>::kTile
            ? merge_tile<4, false, false>(s_src, total, part, kMultiPartStride, t, ntiles, ok, ov, of, fs, ar.status,
                                   nullptr, nullptr, sm, sh, &s_bar, phase)
            : merge_tile<8, false, false>(s_src, total, part, kMultiPartStride, t, ntiles, ok, ov, of, fs, ar.status,
                                   nullptr, nullptr, sm, sh, &s_bar, phase);
    if (!done) break;
  }
}

// The round's plan, one CTA: for every instance with a batch this round,
// the fold's target level k = ffz(r) (§III-B) and r += 1, or the reason the
// batch is refused; then the prefix sums of merge tiles and partition
// boundaries over the instances, and the merge queue reset.
__global__ void __launch_bounds__(1024) multi_prep(MultiArena ar, MultiBatch in) {
  __shared__ uint64_t s_w1[32], s_w2[32];
  __shared__ uint64_t s_carry_t, s_carry_p;
  __shared__ uint32_t s_err;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    s_carry_t = 0;
    s_carry_p = 0;
    s_err = 0;
  }
  __syncthreads();
  for (uint32_t base = 0; base < ar.n; base += 1024) {
    const uint32_t i = base + tid;
    uint64_t nt = 0, np = 0;
    if (i < ar.n) {
      const MultiInst& d = ar.inst[i];
      const uint32_t nops = in.counts ? __ldg(in.counts + i) : d.b;
      uint32_t fl = 0;
      int k = -1;
      if (nops > d.b) {
        fl = kErrArg;
      } else if (nops > 0) {
        if (ar.badkey[i]) {
          fl = kErrBadKey;
        } else {
          const uint32_t r = ar.r[i];
          const int kk = (~r) ? __ffs(~r) - 1 : 32;
          if (kk >= int(d.levels)) {
            fl = kErrFull;
          } else {
            k = kk;
            ar.r[i] = r + 1;
            if (k > 0) {
              nt = ((uint64_t(d.b) << k) + d.tile - 1) / d.tile;
              np = nt + 1;
            }
          }
        }
      }
      ar.badkey[i] = 0;
      ar.k[i] = k;
      ar.flags[i] = fl;
      if (fl) atomicOr(&s_err, fl);
    }
    uint64_t tt, tp;
    const uint64_t et = block_excl_scan<1024, uint64_t>(nt, s_w1, tt);
    const uint64_t ep = block_excl_scan<1024, uint64_t>(np, s_w2, tp);
    if (i < ar.n) {
      ar.tile_prefix[i] = s_carry_t + et;
      ar.part_prefix[i] = s_carry_p + ep;
    }
    __syncthreads();
    if (tid == 0) {
      s_carry_t += tt;
      s_carry_p += tp;
    }
    __syncthreads();
  }
  if (tid == 0) {
    ar.tile_prefix[ar.n] = s_carry_t;
    ar.part_prefix[ar.n] = s_carry_p;
    *ar.work_ctr = 0u;
    if (s_err) atomicOr(ar.status, s_err);
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

// Prefix index of a sorted run: the element at position i owns the entries
// between the bin of element i - 1 and its own; the first and last elements
// record the populated bin range.
__global__ void __launch_bounds__(256) build_fence(const uint32_t* __restrict__ keys, uint32_t n,
                                                   uint32_t* __restrict__ fence, int fshift) {
  __shared__ uint32_t s_ngap;
  __shared__ FenceGap s_gaps[kFenceGapSlots];
  if (threadIdx.x == 0) s_ngap = 0;
  __syncthreads();
  const uint32_t nb = fence_bins(fshift);
  for (uint64_t i = blockIdx.x * 256ull + threadIdx.x; i < n; i += uint64_t(gridDim.x) * 256ull) {
    const uint32_t bin = fence_bin(__ldg(keys + i), fshift);
    if (i == 0) {
      fence[nb + 2] = bin;
    } else {
      const uint32_t pb = fence_bin(__ldg(keys + i - 1), fshift);
      if (bin > pb) fence_write_gap(fence, pb, bin, uint32_t(i), s_gaps, &s_ngap);
    }
    if (i + 1 == n) fence[nb + 3] = bin;
  }
  __syncthreads();
  fence_fill_gaps(fence, s_gaps, s_ngap);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
}

}  // namespace

cudaError_t fold_partition_launch(const FoldArgs& a, cudaStream_t st) {
  const uint64_t ntiles = fold_tiles(a.total);
  if (ntiles == 0) return cudaSuccess;
  const uint64_t pblocks = ((ntiles + 1) * 32 + 255) / 256;
  count_launches(1);
  return launch_pdl(fold_partition, dim3(unsigned(pblocks)), dim3(256), 0, st, a.src, a.total, uint32_t(ntiles),
                    uint32_t(kFoldTile), a.part);
}

PerDeviceFlags g_merge_attr[2];

cudaError_t fold_merge_launch(const FoldArgs& a, cudaStream_t st) {
  cudaError_t e;
  constexpr size_t full = TileGeom<kFoldE>::kSmem;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = set_smem_attr_once(fold_merge<false>, full, dev, g_merge_attr[0])) != cudaSuccess) return e;
  if ((e = set_smem_attr_once(fold_merge<true>, full, dev, g_merge_attr[1])) != cudaSuccess) return e;
  // the slots, plus the one chain buffer of the in-place chain (from three
  // sources): more CTAs fit per SM for the small folds
  using G = TileGeom<kFoldE>;
  const int S = a.src.count;
  const size_t smem = 2 * size_t(plain_slot_cap(uint32_t(S))) * sizeof(uint32_t) + (S >= 3 ? G::kChainBytes + kChainPad : 0);
  const uint64_t ntiles = fold_tiles(a.total);
  if (a.cleanup) {
    if ((e = cudaMemsetAsync(a.out_count, 0, sizeof(uint64_t), st)) != cudaSuccess) return e;
  }
  if (ntiles == 0) return cudaSuccess;
  if (a.cleanup) {
    if ((e = cudaMemsetAsync(a.lookback, 0, sizeof(uint64_t) * ntiles, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.tile_ctr, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    count_launches(1);
    fold_merge<true><<<unsigned(ntiles), kThreads, smem, st>>>(a.src, a.total, a.part, a.out_keys, a.out_vals,
                                                              nullptr, 16, a.status, a.lookback, a.tile_ctr,
                                                              a.out_count, uint32_t(ntiles));
  } else {
    count_launches(1);
    return launch_pdl(fold_merge<false>, dim3(unsigned(ntiles)), dim3(kThreads), smem, st, a.src, a.total,
                      static_cast<const uint32_t*>(a.part), a.out_keys, a.out_vals, a.out_fence, a.out_fshift,
                      a.status, static_cast<uint64_t*>(nullptr), static_cast<uint32_t*>(nullptr),
                      static_cast<uint64_t*>(nullptr), uint32_t(ntiles));
  }
  return cudaGetLastError();
}

cudaError_t fold_launch(const FoldArgs& a, cudaStream_t st) {
  cudaError_t e = fold_partition_launch(a, st);
  if (e != cudaSuccess) return e;
  return fold_merge_launch(a, st);
}

cudaError_t multi_prep_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st) {
  count_launches(1);
  multi_prep<<<1, 1024, 0, st>>>(ar, in);
  return cudaGetLastError();
}

cudaError_t multi_update_launch(const MultiArena& ar, const MultiBatch& in, cudaStream_t st) {
  cudaError_t e;
  if ((e = multi_sort_count_launch(ar, in, st)) != cudaSuccess) return e;
  if ((e = multi_prep_launch(ar, in, st)) != cudaSuccess) return e;
  if ((e = multi_sort_launch(ar, in, st)) != cudaSuccess) return e;
  return multi_fold_launch(ar, st);
}

static int g_merge_per_sm = 0;  // resident multi_merge CTAs per SM

cudaError_t multi_prepare_kernels() {
  cudaError_t e;
  if ((e = multi_sort_prepare()) != cudaSuccess) return e;
  constexpr size_t smem = TileGeom<8>::kSmem;
  if ((e = set_smem(multi_merge, smem)) != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, multi_merge, kThreads, smem)) != cudaSuccess)
    return e;
  g_merge_per_sm = per_sm < 1 ? 1 : per_sm;
  return cudaSuccess;
}

cudaError_t multi_fold_launch(const MultiArena& ar, cudaStream_t st) {
  cudaError_t e;
  if (g_merge_per_sm == 0 && (e = multi_prepare_kernels()) != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  count_launches(1);
  multi_partition<<<unsigned(sms) * 8u, 256, 0, st>>>(ar);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  count_launches(1);
  multi_merge<<<unsigned(sms) * unsigned(g_merge_per_sm), kThreads, TileGeom<8>::kSmem, st>>>(ar);
  return cudaGetLastError();
}

cudaError_t distribute_launch(const DistributeArgs& a, cudaStream_t st) {
  if (a.total == 0) return cudaSuccess;
  uint64_t blocks = (a.total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  distribute<<<unsigned(blocks), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t build_fence_launch(const uint32_t* keys, uint32_t n, uint32_t* fence, int fshift, cudaStream_t st) {
  uint64_t blocks = (uint64_t(n) + 1 + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_launches(1);
  build_fence<<<unsigned(blocks), 256, 0, st>>>(keys, n, fence, fshift);
  return cudaGetLastError();
}

}  // namespace gpulsm
