// Device-side helpers shared by the kernel translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lsm_kernels.h"

namespace gpulsm {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// launch_pdl may be scheduled while the kernel before it in the stream is
// still running; pdl_wait() blocks until that kernel has completed and its
// writes are visible (a no-op for a kernel launched without the attribute).
// pdl_trigger() lets the next kernel's blocks be scheduled once every block
// of this grid has executed it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Relaxed device-scope 64-bit load/store for look-back words: the word itself
// is the only datum exchanged, so no ordering beyond coherence is needed.
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Key of a key variable: the status bit dropped (§IV-A).
__device__ __forceinline__ uint32_t key_of(uint32_t kv) { return kv >> 1; }

// First index i in [lo, hi) with a[i] >= x (full 32-bit key variables), else hi.
// "a[i] >= (k << 1)" holds exactly for the elements whose key is >= k, whatever
// the status bits inside a segment, so this is a lower bound on the key.
__device__ __forceinline__ uint32_t lower_bound_kv(const uint32_t* __restrict__ a, uint32_t lo,
                                                   uint32_t hi, uint32_t x) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(a + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// First index i in [lo, hi) with key(a[i]) > k, else hi.
__device__ __forceinline__ uint32_t upper_bound_key(const uint32_t* __restrict__ a, uint32_t lo,
                                                    uint32_t hi, uint32_t k) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (key_of(__ldg(a + mid)) <= k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Entry P (0 .. 2^(32 - fshift)) of the prefix index of a sorted run of n
// elements: the number of elements whose bin is < P.  A table is written
// only inside its populated bin range: the two words after entry nbins hold
// bmin and bmax, the bins of the first and last element; below (and at)
// bmin the answer is 0, above bmax it is n.
// The answer is kept within [0, n], so that a search bounded by it stays
// inside the run even if the table were damaged.
__device__ __forceinline__ uint32_t fence_at(const uint32_t* f, int fshift, uint32_t n, uint32_t P) {
  const uint32_t nb = fence_bins(fshift);
  if (P <= __ldg(f + nb + 2)) return 0u;
  if (P > __ldg(f + nb + 3)) return n;
  return min(__ldg(f + P), n);
}

// Writing a prefix index from consecutive elements: the element at position
// pos with bin `bin` after an element with bin `pb` owns entries (pb, bin].
// Small gaps are written at once; gaps wider than kFenceDirect bins go to a
// per-CTA list that the whole CTA fills afterwards (fence_fill_gaps).
constexpr uint32_t kFenceDirect = 256;
constexpr int kFenceGapSlots = 64;
struct FenceGap {
  uint32_t lo, hi, val;
};

__device__ __forceinline__ void fence_write_gap(uint32_t* f, uint32_t pb, uint32_t bin, uint32_t pos,
                                                FenceGap* s_gaps, uint32_t* s_ngap) {
  if (bin - pb <= kFenceDirect) {
    for (uint32_t P = pb + 1; P <= bin; ++P) f[P] = pos;
    return;
  }
  const uint32_t slot = atomicAdd(s_ngap, 1u);
  if (slot < uint32_t(kFenceGapSlots)) {
    s_gaps[slot] = FenceGap{pb + 1, bin, pos};
  } else {
    for (uint32_t P = pb + 1; P <= bin; ++P) f[P] = pos;
  }
}

// Called by every thread of the CTA after a __syncthreads.
__device__ __forceinline__ void fence_fill_gaps(uint32_t* f, const FenceGap* s_gaps, uint32_t ngap) {
  if (ngap > uint32_t(kFenceGapSlots)) ngap = kFenceGapSlots;
  for (uint32_t g = 0; g < ngap; ++g) {
    const FenceGap gp = s_gaps[g];
    for (uint32_t P = gp.lo + threadIdx.x; P <= gp.hi; P += blockDim.x) f[P] = gp.val;
  }
}

// Largest i < n with prefix[i] <= w, for w < prefix[n] (prefix has n + 1
// non-decreasing entries, so the instance found owns item w even when
// instances with no items share its prefix value).
__device__ __forceinline__ uint32_t find_instance(const uint64_t* prefix, uint32_t n, uint64_t w) {
  uint32_t lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// Lanes of the warp whose value equals this lane's (values below 2^kBits):
// the intersection, over the bits, of the lanes that agree with this lane on
// that bit -- one ballot per bit, a fixed cost however many distinct values
// the warp holds.
template <int kBits>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < kBits; ++b) {
    const uint32_t bit = (d >> b) & 1u;
    const uint32_t m = __ballot_sync(0xffffffffu, bit != 0u);
    peers &= bit ? m : ~m;
  }
  return peers;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread over a block of NT threads
// (NT a multiple of 32, at most 1024).  s_warp holds NT/32 words.
template <int NT, typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* s_warp, T& total) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const T incl = warp_incl_scan(x);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  T before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) {
    const T t = s_warp[w];
    before += (w < (int)warp) ? t : T(0);
    tot += t;
  }
  __syncthreads();
  total = tot;
  return before + incl - x;
}

// ---------------------------------------------------------------- mbarrier --
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded spinning, shared by every wait of the library: a waiter calls
// spin_continue after each unsuccessful poll, with t0 = 0 before the first;
// once the wait has lasted limit_ns (globaltimer) it records kErrTimeout in
// *status and returns false, and the waiter stops waiting and carries on
// without the value (the call then reports LSM_ERR_TIMEOUT through the
// status word instead of hanging the GPU).
__device__ __forceinline__ bool spin_continue(uint64_t& t0, uint64_t limit_ns, uint32_t* status) {
  const uint64_t now = globaltimer_ns();
  if (t0 == 0) {
    t0 = now | 1u;  // never 0 once started
    return true;
  }
  if (now - t0 > limit_ns) {
    atomicOr(status, kErrTimeout);
    return false;
  }
  return true;
}

// Bounded wait on phase `parity`; false (and kErrTimeout) if it never completes.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status) {
  uint64_t t0 = 0;
  while (!mbar_try_wait(bar, parity))
    if (!spin_continue(t0, kWaitLimitNs, status)) return false;
  return true;
}

// 16-byte asynchronous copy global -> shared by this thread (both addresses
// 16-byte aligned); cp_async_wait_all() waits for all of this thread's.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One-dimensional bulk copy global -> shared (TMA engine, no tensor map).
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace gpulsm
