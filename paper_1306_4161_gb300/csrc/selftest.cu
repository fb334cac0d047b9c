// Self-test of the failure handling every kernel of the library relies on: a
// bounded wait that runs out.  One block waits on a shared-memory barrier that
// nothing arrives on, gives up after the caller's limit, records
// HSUMMA_ERR_TIMEOUT in the device status word through the same path as the
// GEMM kernels, and returns; hsumma_sync then reports and clears it.  Nothing
// faults, traps or hangs, and the context stays usable.
#include "internal.h"
#include "ptx.cuh"
#include "../../include/hsumma.h"

namespace hs {
namespace {

constexpr int kSiteSelfTest = 6;

__global__ void wait_runs_out_kernel(unsigned long long limit_ns, int *status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
  __syncthreads();
  const unsigned long long t0 = globaltimer();
  bool done = false;
  while (!(done = mbar_try_wait(smem_u32(&bar), 0))) {
    if (globaltimer() - t0 > limit_ns) break;
  }
  if (!done && threadIdx.x == 0) record_error(status, HSUMMA_ERR_TIMEOUT, kSiteSelfTest);
}

}  // namespace
}  // namespace hs

using namespace hs;

extern "C" int hsumma_selftest_timeout(long long limit_ns, void *stream) {
  if (state().device < 0) {
    set_error("hsumma_init has not been called");
    return HSUMMA_ERR_NOT_INIT;
  }
  if (limit_ns < 0 || limit_ns > 1000000000ll) {
    set_error("self-test wait limit must be in 0..1e9 ns (got %lld)", limit_ns);
    return HSUMMA_ERR_ARG;
  }
  wait_runs_out_kernel<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      (unsigned long long)limit_ns, state().d_status);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HSUMMA_OK : cuda_fail(e, "launch self-test wait");
}
