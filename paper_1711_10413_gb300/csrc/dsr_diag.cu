// dsr_diag.cu -- self-checks of the device runtime (bounded waits, stack
// misuse) and the measured shared-memory bandwidth probe.
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

// Shared-memory bandwidth: each thread loads 16-byte vectors from a 32 KiB
// buffer, a warp's 32 lanes reading 512 consecutive bytes (4 wavefronts,
// no bank conflict), 8 loads per round from 8 different 4 KiB parts of the
// buffer, the window moving by one warp's 512 bytes each round; the loads
// are volatile so none is hoisted or merged, and their XOR goes to a sink
// the host never reads.
constexpr uint32_t kProbeThreads = 1024, kProbeVecs = 2048, kProbeUnroll = 8;

__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

__global__ void __launch_bounds__(kProbeThreads) smem_probe(uint32_t reps, uint64_t *r) {
  __shared__ uint4 buf[kProbeVecs];
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < kProbeVecs; i += blockDim.x)
    buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
  __syncthreads();
  const uint32_t base = dsr::smem_u32(buf);
  uint4 acc = make_uint4(0, 0, 0, 0);
  const uint64_t c0 = clock64(), t0 = dsr::globaltimer();
  for (uint32_t it = 0; it < reps; ++it) {
#pragma unroll
    for (uint32_t u = 0; u < kProbeUnroll; ++u) {
      const uint32_t v = (tid + u * (kProbeVecs / kProbeUnroll) + it * 32u) & (kProbeVecs - 1u);
      const uint4 x = ld_shared_v4(base + 16u * v);
      acc.x ^= x.x;
      acc.y ^= x.y;
      acc.z ^= x.z;
      acc.w ^= x.w;
    }
  }
  const uint64_t c1 = clock64(), t1 = dsr::globaltimer();
  __syncthreads();
  if (tid == 0) {
    atomicMax(reinterpret_cast<unsigned long long *>(&r[1]), c1 - c0);
    atomicMax(reinterpret_cast<unsigned long long *>(&r[2]), t1 - t0);
  }
  if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9e3779b9u) atomicXor(
      reinterpret_cast<unsigned long long *>(&r[0]), 1ull);
}

}  // namespace

extern "C" int32_t dsr_probe_smem_bandwidth(dsr_ctx *ctx, uint32_t reps, uint64_t *scratch_dev,
                                            void *stream, dsr_smem_probe *out) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!scratch_dev || !out) return dsr_fail(ctx, DSR_ERR_INVALID, "null scratch or output");
  if (reps == 0 || reps > (1u << 20))
    return dsr_fail(ctx, DSR_ERR_INVALID, "reps must be in [1, 2^20]");
  if (int32_t rc = dsr_check_device(ctx)) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_probe,
                                                                kProbeThreads, 0);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "probe occupancy");
  const uint32_t ctas = static_cast<uint32_t>(ctx->sm_count * (per_sm > 0 ? per_sm : 1));
  cudaEvent_t a = nullptr, z = nullptr;
  uint64_t h[4] = {0, 0, 0, 0};
  float ms = 0.0f;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  if (e == cudaSuccess) {
    smem_probe<<<ctas, kProbeThreads, 0, s>>>(reps / 8u + 1u, scratch_dev);  // warm-up
    e = cudaMemsetAsync(scratch_dev, 0, 4 * sizeof(uint64_t), s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    smem_probe<<<ctas, kProbeThreads, 0, s>>>(reps, scratch_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(z, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, scratch_dev, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "shared-memory probe");
  out->bytes = static_cast<uint64_t>(ctas) * kProbeThreads * reps * kProbeUnroll * 16ull;
  out->ms = ms;
  out->gbs = ms > 0 ? out->bytes / (ms * 1e-3) / 1e9 : 0.0;
  out->sm_mhz = h[2] ? static_cast<double>(h[1]) / static_cast<double>(h[2]) * 1e3 : 0.0;
  out->bytes_per_clk_sm =
      out->sm_mhz > 0 ? out->gbs * 1e9 / (ctx->sm_count * out->sm_mhz * 1e6) : 0.0;
  out->ctas = ctas;
  out->threads = kProbeThreads;
  return DSR_OK;
}

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
