// Fault injection entry points for tests (gpulsm.h, "Fault injection").
//
// Neither has a counterpart in the paper.  They let the tests drive the
// library's error paths without a real out-of-memory condition and without
// faulting or hanging a GPU: an allocation failure is simulated on the host
// (alloc_gate, lsm_api.cu), and a device wait that runs out is a bounded spin
// on a word that nothing writes, which gives up and reports a timeout while
// the context stays usable.
#include "gpulsm.h"
#include "lsm_device.cuh"

namespace gpulsm {
namespace {

// One thread spins on *flag with the library's bounded spin (spin_continue,
// the helper every look-back and bulk-copy wait uses); a wait that gives up
// leaves kErrTimeout in *status.
__global__ void debug_wait_flag(const uint32_t* flag, uint32_t* status, uint64_t limit_ns) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const volatile uint32_t* f = flag;
  uint64_t t0 = 0;
  while (*f == 0u)
    if (!spin_continue(t0, limit_ns, status)) return;
}

}  // namespace

void debug_fail_allocs(uint64_t skip, uint64_t count);

}  // namespace gpulsm

extern "C" lsm_status lsm_debug_fail_allocs(uint64_t skip, uint64_t count) {
  gpulsm::debug_fail_allocs(skip, count);
  return LSM_OK;
}

extern "C" lsm_status lsm_debug_wait_flag(const uint32_t* d_flag, uint32_t* d_status, uint64_t limit_ns,
                                          void* stream) {
  using namespace gpulsm;
  if (!d_flag || !d_status || limit_ns == 0 || limit_ns > 10000000000ull) return LSM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) {
    count_launches(1);
    debug_wait_flag<<<1, 32, 0, st>>>(d_flag, d_status, limit_ns);
    e = cudaGetLastError();
  }
  uint32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LSM_ERR_CUDA;
  }
  return (h & kErrTimeout) ? LSM_ERR_TIMEOUT : LSM_OK;
}
