// dsr_diag.cu -- self-check of the device runtime's bounded waits.
#include <cuda_runtime.h>

#include "dsr.h"
#include "dsr_ctx.h"
#include "dsr_diag.h"
#include "dsr_runtime.cuh"

namespace {

// One thread: an mbarrier expecting 16 bytes that no copy delivers, waited
// on by the same bounded wait the fills use.
__global__ void bounded_wait_check(uint64_t timeout_ns, uint64_t *result) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  dsr::mbar_init(&bar, 1);
  dsr::mbar_init_fence();
  dsr::mbar_expect_tx(&bar, 16);  // the one arrival, and 16 bytes still owed
  const uint64_t t0 = dsr::globaltimer();
  const bool done = dsr::mbar_wait(&bar, 0, timeout_ns);
  result[1] = dsr::globaltimer() - t0;
  result[0] = static_cast<uint64_t>(done ? DSR_OK : DSR_ERR_TIMEOUT);
}

}  // namespace

extern "C" int32_t dsr_check_bounded_wait(dsr_ctx *ctx, uint64_t timeout_ns, uint64_t *result_dev,
                                          void *stream) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!result_dev) return dsr_fail(ctx, DSR_ERR_INVALID, "null result");
  if (timeout_ns > 10000000000ull)
    return dsr_fail(ctx, DSR_ERR_INVALID, "timeout %llu ns is over 10 s",
                    static_cast<unsigned long long>(timeout_ns));
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) {
    bounded_wait_check<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(timeout_ns, result_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "bounded-wait check");
  return DSR_OK;
}
