// Failure-path self test: a bounded mbarrier wait that nothing completes. The wait
// gives up after the given time, latches the timeout bit in the plan's device error
// word and returns, exactly as a stalled pipeline stage of the tensor-core kernels
// would; the host sees FTK_ERR_TIMEOUT at the next ftk_stream_check and the context
// stays usable. No fault, trap or unbounded loop is involved.
#include <cuda_runtime.h>

#include "ftk_internal.h"
#include "tc_ptx.cuh"

namespace {

__global__ void k_wait_nobody(int* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    ftk::tc::mbar_init(&bar, 1);
    abort_flag = 0;
    ftk::tc::fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) ftk::tc::mbar_wait(&bar, 0, &abort_flag, err, limit_ns);  // never arrived on
  __syncthreads();
}

}  // namespace

extern "C" ftk_status ftk_selftest_timeout(ftk_plan_t p, unsigned int limit_us, void* stream) {
  if (!p || limit_us == 0 || limit_us > 2000000u) return FTK_ERR_ARG;
  k_wait_nobody<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(p->d_err, 1000ull * limit_us);
  return cudaGetLastError() == cudaSuccess ? FTK_OK : FTK_ERR_CUDA;
}
