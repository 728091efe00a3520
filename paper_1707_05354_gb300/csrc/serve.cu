// Kernels of the serving engine (lsm_serve.cu): the ordered update batch,
// which lets requests that arrived one after another share one device batch,
// and the gather of request payload windows.
//
// Ordered batch.  The batch rules of §III-A resolve several ops on one key
// within a batch with the delete winning (rule 6), which is not the order
// the ops were issued in when they come from different requests.  Giving
// every op on a key the content of the LAST op on that key (in input order)
// makes the batch mean what applying its ops one by one means: all copies of
// a delete leave the key deleted, all copies of an insert leave its value.
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

__global__ void __launch_bounds__(256) resolve_last(const uint32_t* __restrict__ sk, const uint32_t* __restrict__ sv,
                                                    uint32_t n, const uint32_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ vals,
                                                    const uint8_t* __restrict__ del, uint32_t* __restrict__ out_k,
                                                    uint32_t* __restrict__ out_v, uint8_t* __restrict__ out_d) {
  for (uint32_t i = blockIdx.x * 256u + threadIdx.x; i < n; i += gridDim.x * 256u) {
    const uint32_t key = __ldg(sk + i);
    // last index e >= i holding this key (equal keys are contiguous, the
    // stable sort keeps them in input order)
    uint32_t e = i;
    if (i + 1 < n && __ldg(sk + i + 1) == key) {
      uint32_t lo = i + 1, hi = n;  // first index with a larger key
      while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(sk + mid) <= key) lo = mid + 1; else hi = mid;
      }
      e = lo - 1;
    }
    const uint32_t w = __ldg(sv + e), p = __ldg(sv + i);
    out_k[p] = key;
    out_v[p] = vals ? __ldg(vals + w) : 0u;
    out_d[p] = del ? __ldg(del + w) : uint8_t(0);
  }
}

// Request j of the n descriptors owns output positions [dst_off[j],
// dst_off[j] + size[j]); dst_off ascending.  Largest j with dst_off[j] <= g.
__device__ __forceinline__ uint32_t owner(const uint64_t* __restrict__ dst_off, uint32_t n, uint64_t g) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(dst_off + mid) <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// One thread per output element (requests are found by bisection of the
// output offsets), so a few large windows still spread over the GPU.
__global__ void __launch_bounds__(256) gather_windows(const uint32_t* __restrict__ src_a,
                                                      const uint32_t* __restrict__ src_b,
                                                      const uint64_t* __restrict__ start,
                                                      const uint64_t* __restrict__ dst_off, uint32_t nreq,
                                                      uint64_t total, uint32_t* __restrict__ dst_a,
                                                      uint32_t* __restrict__ dst_b) {
  for (uint64_t g = blockIdx.x * 256ull + threadIdx.x; g < total; g += uint64_t(gridDim.x) * 256ull) {
    const uint32_t j = owner(dst_off, nreq, g);
    const uint64_t s = __ldg(start + j) + (g - __ldg(dst_off + j));
    dst_a[g] = __ldg(src_a + s);
    if (src_b) dst_b[g] = __ldg(src_b + s);
  }
}

// Update requests into a batch: keys from pool_k, values from pool_v (0 for
// a delete request), the request's delete flag per op.
__global__ void __launch_bounds__(256) gather_update(const uint32_t* __restrict__ pool_k,
                                                     const uint32_t* __restrict__ pool_v,
                                                     const uint64_t* __restrict__ start,
                                                     const uint64_t* __restrict__ dst_off,
                                                     const uint8_t* __restrict__ is_del, uint32_t nreq,
                                                     uint64_t total, uint32_t* __restrict__ out_k,
                                                     uint32_t* __restrict__ out_v, uint8_t* __restrict__ out_d) {
  for (uint64_t g = blockIdx.x * 256ull + threadIdx.x; g < total; g += uint64_t(gridDim.x) * 256ull) {
    const uint32_t j = owner(dst_off, nreq, g);
    const uint64_t s = __ldg(start + j) + (g - __ldg(dst_off + j));
    const uint8_t del = __ldg(is_del + j);
    out_k[g] = __ldg(pool_k + s);
    out_v[g] = del ? 0u : __ldg(pool_v + s);
    out_d[g] = del;
  }
}

}  // namespace

cudaError_t gather_update_launch(const uint32_t* pool_k, const uint32_t* pool_v, const uint64_t* start,
                                 const uint64_t* dst_off, const uint8_t* is_del, uint32_t nreq, uint64_t total,
                                 uint32_t* out_k, uint32_t* out_v, uint8_t* out_d, cudaStream_t st) {
  if (nreq == 0 || total == 0) return cudaSuccess;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  gather_update<<<unsigned(blocks), 256, 0, st>>>(pool_k, pool_v, start, dst_off, is_del, nreq, total, out_k, out_v,
                                                  out_d);
  return cudaGetLastError();
}

cudaError_t resolve_last_launch(const uint32_t* sk, const uint32_t* sv, uint32_t n, const uint32_t* keys,
                                const uint32_t* vals, const uint8_t* del, uint32_t* out_k, uint32_t* out_v,
                                uint8_t* out_d, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint32_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  count_launches(1);
  resolve_last<<<blocks, 256, 0, st>>>(sk, sv, n, keys, vals, del, out_k, out_v, out_d);
  return cudaGetLastError();
}

cudaError_t gather_windows_launch(const uint32_t* src_a, const uint32_t* src_b, const uint64_t* start,
                                  const uint64_t* dst_off, uint32_t nreq, uint64_t total, uint32_t* dst_a,
                                  uint32_t* dst_b, cudaStream_t st) {
  if (nreq == 0 || total == 0) return cudaSuccess;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  count_launches(1);
  gather_windows<<<unsigned(blocks), 256, 0, st>>>(src_a, src_b, start, dst_off, nreq, total, dst_a, dst_b);
  return cudaGetLastError();
}

}  // namespace gpulsm
