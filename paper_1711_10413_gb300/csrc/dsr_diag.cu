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

// The team stack's push and pop (Sec. 5.2's allocation on the shared stack,
// the global fallback, and the LIFO release), misused on purpose by one
// master warp, each outcome recorded by lane 0 in order (see dsr_diag.h).
constexpr uint32_t kCheckSlab = 96, kCheckOvf = 64, kCheckWords = 25;

__global__ void stack_check(uint8_t *ovf, uint64_t *r) {
  using namespace dsr;
  Stack s;
  uint32_t n = 0;
  auto put = [&](uint64_t v) {
    if (lane_id() == 0) r[n] = v;
    ++n;
  };
  // team 1: two frames in the slab and one in the overflow slab, then a pop
  // of a frame that is not the top, then the pops in order
  team_setup(s, kCheckSlab, ovf, kCheckOvf, 1000000ull, true);
  bool sm1 = false, sm2 = false, sm3 = false;
  uint8_t *f1 = push(s, 48, &sm1);
  uint8_t *f2 = push(s, 40, &sm2);
  uint8_t *f3 = push(s, 64, &sm3);
  put(f1 && sm1);
  put(f2 && sm2);
  put(f3 && !sm3);
  put(s.sp);
  put(s.gsp);
  put(static_cast<uint32_t>(pop(s, f2, 40)));
  put(s.depth());
  put(s.sp);
  put(s.gsp);
  put(static_cast<uint32_t>(pop(s, f3, 64)));
  put(static_cast<uint32_t>(pop(s, f2, 40)));
  put(static_cast<uint32_t>(pop(s, f1, 48)));
  put(s.depth());
  put(s.sp);
  put(s.gsp);
  put(static_cast<uint32_t>(s.status()));
  put(s.hwm);
  put(s.spill);
  // team 2: a push that fits neither slab, then a pop of the right frame
  // with the wrong size
  team_setup(s, kCheckSlab, ovf, kCheckOvf, 1000000ull, false);
  push(s, 48);
  push(s, 48);
  uint8_t *g3 = push(s, 64);
  uint8_t *g4 = push(s, 16);
  put(static_cast<uint32_t>(s.status()));
  put(g4 == nullptr);
  put(s.depth());
  put(static_cast<uint32_t>(pop(s, g3, 32)));
  // team 3: sixteen-byte frames until the frame table is full
  team_setup(s, kCheckSlab, ovf, kCheckOvf, 1000000ull, false);
  uint32_t pushed = 0;
  for (uint32_t i = 0; i < DSR_MAX_FRAMES + 1u; ++i) pushed += push(s, 16) != nullptr;
  put(pushed);
  put(static_cast<uint32_t>(s.status()));
  put(s.depth());
}

}  // namespace

extern "C" int32_t dsr_check_stack(dsr_ctx *ctx, uint64_t *result_dev, uint32_t n_result,
                                   void *scratch_dev, uint64_t scratch_bytes, void *stream) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!result_dev || n_result < kCheckWords)
    return dsr_fail(ctx, DSR_ERR_INVALID, "the result needs %u words", kCheckWords);
  if (!scratch_dev || scratch_bytes < kCheckOvf || (reinterpret_cast<uintptr_t>(scratch_dev) & 15u))
    return dsr_fail(ctx, DSR_ERR_INVALID, "scratch must be %u bytes, 16-byte aligned", kCheckOvf);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) {
    stack_check<<<1, 32, dsr::kCtrlBytes + kCheckSlab, static_cast<cudaStream_t>(stream)>>>(
        static_cast<uint8_t *>(scratch_dev), result_dev);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "stack check");
  return DSR_OK;
}

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
