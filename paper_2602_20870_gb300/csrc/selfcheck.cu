// Failure-path check of the bounded device waits.
//
// Every kernel of the library that waits on an mbarrier gives up after FG_WAIT_LIMIT_NS,
// records FG_STATUS_WAIT_TIMEOUT in the plan's status word and returns, so a stalled
// producer never hangs the device.  This entry point runs that path on purpose: one
// thread waits, through the same bounded helper, on an mbarrier that nothing arrives on.
// The wait runs out, the status bit is set and the kernel returns normally; nothing
// faults and the context stays usable.
#include "internal.h"

namespace {

__global__ void wait_runs_out_kernel(uint32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival that never comes
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) (void)mbar_wait(&bar, 0, status);
}

}  // namespace

extern "C" int fgfrft_check_wait_timeout(fgfrft_plan p, void* stream) {
  if (!p) return FGFRFT_ERR_INVALID_ARG;
  wait_runs_out_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(p->dstatus);
  if (cudaGetLastError() != cudaSuccess) return FGFRFT_ERR_CUDA;
  return FGFRFT_OK;
}
