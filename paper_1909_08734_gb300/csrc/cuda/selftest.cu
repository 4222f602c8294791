// Expiry of the bounded waits, exercised on purpose: one thread waits on an mbarrier phase
// that nothing completes and on a flag that nothing sets, both with a short time limit, then
// latches CPM_ERR_TIMEOUT in the handle's status word exactly as an expired wait in the
// solve or factorisation kernels does.  Nothing faults: the kernel returns normally.
#include "common.cuh"
#include "kernels.h"

namespace cpmdev {

__global__ void bounded_wait_selftest_kernel(uint64_t limit_ns, const uint32_t* never, int* status, int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);                       // no thread ever arrives: phase 0 never completes
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const bool phase_done = mbar_wait_bounded(&bar, 0, limit_ns);
  bool flag_seen = false;
  const uint64_t t0 = global_ns();
  while (!(flag_seen = ld_acquire(never) != 0u) && global_ns() - t0 <= limit_ns) {
  }
  if (!phase_done || !flag_seen) atomicOr(status, ST_TIMEOUT);
  out[0] = phase_done ? 1 : 0;
  out[1] = flag_seen ? 1 : 0;
}

cudaError_t launch_bounded_wait_selftest(uint64_t limit_ns, const uint32_t* never, int* status, int* out,
                                         cudaStream_t s) {
  bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(limit_ns, never, status, out);
  return cudaGetLastError();
}

}  // namespace cpmdev
