// Failure-path check of the bounded device waits (rt_selftest_wait_timeout,
// declared in include/rt.h).  Not a step of the method: it exercises the
// path every bounded wait of the library takes when its phase never
// completes -- give up after a bounded number of polls, record RT_TIMEOUT in
// the context's status word, return -- without any fault or hang.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "../../include/rt.h"
#include "rt_ctx.h"

namespace m1rt {

// One block that waits, at most `polls` polls, on an mbarrier phase that no
// arrival completes, and records the timeout.  No copy is in flight, so the
// block can leave at once.
__global__ void k_selftest_wait(int* status, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  bool done = false;
  for (uint32_t n = 0; n < polls && !done; ++n) done = mbar_try_wait(&bar, 0);
  if (!done && threadIdx.x == 0) atomicOr(status, kStTimeout);
}

}  // namespace m1rt

extern "C" rt_status rt_selftest_wait_timeout(rt_ctx* ctx, uint32_t polls) {
  if (!ctx) return RT_INVALID_ARG;
  if (!ctx->mesh_ready) {
    ctx->err = "rt_init_mesh has not succeeded";
    return RT_NOT_READY;
  }
  if (polls < 1 || polls > 65536) {
    ctx->err = "polls must lie in 1..65536";
    return RT_INVALID_ARG;
  }
  m1rt::k_selftest_wait<<<1, 32, 0, ctx->stream>>>(ctx->status, polls);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "selftest: %s", cudaGetErrorString(e));
    ctx->err = buf;
    return RT_CUDA;
  }
  return RT_OK;
}
