// dsr_runtime.cuh -- device side of the generic-mode data-sharing runtime.
//
// One team = one CTA of N threads. Threads 0..W-1 (W = N - 32) are workers;
// the last warp is the master warp and its lane 0 the master (Sec. 4: "the
// last 32 threads are reserved for the master thread region", the first of
// them is the master). Lanes 1..31 of the master warp stay resident: they
// take part in every barrier and help with runtime-owned copies, so no
// thread of a barrier's warp count has exited.
//
// Handoff (Sec. 4, Fig. "codegen-master" / "codegen-worker"): workers wait
// at the fork barrier while the master runs sequential code; the master
// publishes the work (body id, thread count, argument) and the frame table,
// arrives at the fork barrier, and waits at the join barrier until the
// workers finish the body. Named barriers (Sec. 4: "named barriers are used
// to control the execution of master and worker threads") keep fork and
// join apart: bar.sync kForkBar / kJoinBar with the team's thread count.
// Workers beyond the region's thread count skip the body but still reach
// the join (the exec_status test of Fig. "codegen-worker").
//
// Shared locals (Sec. 5.1-5.3): the master pushes a frame per call level on
// a LIFO stack. The stack pointers (slab and overflow; the paper's shared
// stack pointer register of Sec. 5.3, %SPSH / VRShared) live in the team's
// control block in shared memory, where every master-warp lane reads them
// and lane 0 updates them, which keeps the kernels within 32 registers.
// A frame goes to the team's shared-memory slab when it fits, otherwise to
// the team's global overflow slab (the global-memory safety net of Sec. 5.2
// and the runtime-managed global stack of Sec. 7); a frame never straddles
// the two. The frame table in the control block is the list of references
// the master hands to the workers (Sec. 5.1-5.2): one generic pointer per
// live frame, valid for shared and global frames alike.
#pragma once

#include <cstdint>

#include "dsr.h"

namespace dsr {

constexpr uint32_t kForkBar = 1;
constexpr uint32_t kJoinBar = 2;
constexpr uint32_t kTerminate = 0xFFFFFFFFu;
constexpr uint32_t kCtrlBytes = 256;  // control block, slab starts after it

struct FrameEnt {
  uint8_t *ptr;      // generic address of the frame (shared or global)
  uint32_t bytes;    // requested size
  uint32_t in_smem;  // 1 = slab, 0 = overflow slab
};

struct __align__(16) Ctrl {
  // handoff: written by the master before the fork barrier, read by workers
  uint32_t work;      // body id of the current parallel region or kTerminate
  uint32_t nthreads;  // threads of the current parallel region
  uint32_t arg;       // per-region argument (level, region index)
  uint32_t task;      // batched launch: current task
  // the team's stack (master warp only; every lane reads, lane 0 writes)
  uint32_t sp;        // slab bytes reserved
  uint32_t depth;     // live frames
  uint32_t hwm;       // peak reserved bytes, slab + overflow
  uint32_t spill;     // peak reserved overflow bytes
  uint64_t gsp;       // overflow-slab bytes reserved
  int32_t status;
  uint32_t phase;     // parity of the fill mbarrier
  uint64_t mbar;      // mbarrier completing bulk-copy fills
  uint32_t slab_bytes;
  uint32_t pad0;
  uint8_t *ovf;       // this team's overflow slab
  uint64_t ovf_bytes;
  uint64_t timeout_ns;
  uint32_t chk[DSR_MAX_DEPTH];
  FrameEnt frames[DSR_MAX_FRAMES];
};
static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block too large");

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void named_bar(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after timeout_ns of
// %globaltimer and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 31u) == 0 && globaltimer() - t0 > timeout_ns) return false;
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Non-tensor bulk copy global -> this CTA's shared memory, completing on
// `bar` (dst, src 16-byte aligned; bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 32-bit finaliser of MurmurHash3 (Appleby, public domain).
__device__ __forceinline__ uint32_t mix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Per-team environment
// ---------------------------------------------------------------------------
extern __shared__ __align__(128) uint8_t dsr_smem[];

__device__ __forceinline__ Ctrl *ctrl() { return reinterpret_cast<Ctrl *>(dsr_smem); }
__device__ __forceinline__ uint8_t *slab_base() { return dsr_smem + kCtrlBytes; }
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t team_threads() { return blockDim.x; }
__device__ __forceinline__ uint32_t team_workers() { return blockDim.x - 32u; }

struct Env {
  const dsr_region_desc *d;  // the region (kernel parameter space or global)
  const uint8_t *images;
  uint8_t *out;
  uint32_t team;             // team number (omp_get_team_num)
};

// Team setup (master warp): the stack starts empty.
__device__ __forceinline__ void team_setup(uint32_t slab_bytes, uint8_t *ovf, uint64_t ovf_bytes,
                                           uint64_t timeout_ns, bool first) {
  Ctrl *c = ctrl();
  if (lane_id() == 0) {
    c->sp = 0;
    c->depth = 0;
    c->hwm = 0;
    c->spill = 0;
    c->gsp = 0;
    c->status = DSR_OK;
    c->slab_bytes = slab_bytes;
    c->ovf = ovf;
    c->ovf_bytes = ovf_bytes;
    c->timeout_ns = timeout_ns;
#pragma unroll
    for (int k = 0; k < DSR_MAX_DEPTH; ++k) c->chk[k] = 0;
    if (first) {
      c->phase = 0;
      mbar_init(&c->mbar, 1);
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void set_status(int32_t st) {
  __syncwarp();
  if (lane_id() == 0 && ctrl()->status == DSR_OK) ctrl()->status = st;
  __syncwarp();
}

__device__ __forceinline__ bool team_ok() { return ctrl()->status == DSR_OK; }

// Push `bytes` (whole master warp). Returns the frame's generic address, or
// nullptr with status OVERFLOW when neither slab has room or the frame table
// is full.
__device__ __forceinline__ uint8_t *push(uint32_t bytes, bool *in_smem = nullptr) {
  Ctrl *c = ctrl();
  const uint32_t fp = (bytes + 15u) & ~15u;
  if (c->status != DSR_OK) return nullptr;
  const uint32_t sp = c->sp, depth = c->depth;
  const uint64_t gsp = c->gsp;
  uint8_t *p = nullptr;
  uint32_t sm = 0;
  if (depth < DSR_MAX_FRAMES) {
    if (sp + fp <= c->slab_bytes) {
      p = slab_base() + sp;
      sm = 1;
    } else if (gsp + fp <= c->ovf_bytes) {
      p = c->ovf + gsp;
    }
  }
  if (!p) {
    set_status(DSR_ERR_OVERFLOW);
    return nullptr;
  }
  __syncwarp();
  if (lane_id() == 0) {
    const uint32_t nsp = sm ? sp + fp : sp;
    const uint64_t ngsp = sm ? gsp : gsp + fp;
    c->sp = nsp;
    c->gsp = ngsp;
    c->depth = depth + 1;
    c->frames[depth].ptr = p;
    c->frames[depth].bytes = bytes;
    c->frames[depth].in_smem = sm;
    const uint64_t live = static_cast<uint64_t>(nsp) + ngsp;
    if (live > c->hwm) c->hwm = static_cast<uint32_t>(live);
    if (ngsp > c->spill) c->spill = static_cast<uint32_t>(ngsp);
  }
  __syncwarp();
  if (in_smem) *in_smem = sm != 0;
  return p;
}

// Pop `p`, which must be the top frame (else status LIFO, nothing popped).
__device__ __forceinline__ int32_t pop(const uint8_t *p) {
  Ctrl *c = ctrl();
  const uint32_t depth = c->depth;
  if (depth == 0 || c->frames[depth - 1].ptr != p) {
    set_status(DSR_ERR_LIFO);
    return DSR_ERR_LIFO;
  }
  const FrameEnt f = c->frames[depth - 1];
  const uint32_t fp = (f.bytes + 15u) & ~15u;
  __syncwarp();
  if (lane_id() == 0) {
    if (f.in_smem)
      c->sp -= fp;
    else
      c->gsp -= fp;
    c->depth = depth - 1;
  }
  __syncwarp();
  return DSR_OK;
}

// Fill a frame from a global image, word by word XOR `key` (master warp).
// Shared-memory frames with 16-byte aligned source and size take one bulk
// copy issued by the master (a single thread moves the whole frame) and are
// then keyed in place; other frames are copied by the 32 lanes with 16-byte
// vector accesses where alignment allows.
__device__ __forceinline__ void fill(uint8_t *dst, bool dst_smem, const uint8_t *src,
                                     uint32_t bytes, uint32_t key) {
  const uint32_t lane = lane_id();
  Ctrl *c = ctrl();
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | bytes) & 15u) == 0;
  if (dst_smem && aligned && bytes >= 64) {
    uint64_t *bar = &c->mbar;
    const uint32_t phase = c->phase;
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_expect_tx(bar, bytes);
      for (uint32_t off = 0; off < bytes; off += 32768u) {
        const uint32_t n = bytes - off < 32768u ? bytes - off : 32768u;
        bulk_g2s(dst + off, src + off, n, bar);
      }
    }
    __syncwarp();
    const uint64_t tmo = c->timeout_ns;
    if (!mbar_wait(bar, phase, tmo)) {
      // the copy is still in flight: wait for it (bounded again) before the
      // slab can be reused or the CTA ends
      mbar_wait(bar, phase, tmo);
      set_status(DSR_ERR_TIMEOUT);
    }
    __syncwarp();
    if (lane == 0) c->phase = phase ^ 1u;
    if (key != 0) {
      uint4 *v = reinterpret_cast<uint4 *>(dst);
      for (uint32_t i = lane; i < bytes / 16u; i += 32u) {
        uint4 x = v[i];
        x.x ^= key;
        x.y ^= key;
        x.z ^= key;
        x.w ^= key;
        v[i] = x;
      }
    }
  } else if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const uint32_t nv = bytes / 16u;
    const uint4 *sv = reinterpret_cast<const uint4 *>(src);
    uint4 *dv = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i = lane; i < nv; i += 64u) {
      uint4 x0 = __ldg(sv + i), x1 = make_uint4(0, 0, 0, 0);
      const bool two = i + 32u < nv;
      if (two) x1 = __ldg(sv + i + 32u);
      x0.x ^= key;
      x0.y ^= key;
      x0.z ^= key;
      x0.w ^= key;
      dv[i] = x0;
      if (two) {
        x1.x ^= key;
        x1.y ^= key;
        x1.z ^= key;
        x1.w ^= key;
        dv[i + 32u] = x1;
      }
    }
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(src);
    uint32_t *dw = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t w = nv * 4u + lane; w < bytes / 4u; w += 32u) dw[w] = __ldg(sw + w) ^ key;
  } else {
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(src);
    uint32_t *dw = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t w = lane; w < bytes / 4u; w += 32u) dw[w] = __ldg(sw + w) ^ key;
  }
  __syncwarp();
}

// Sum of the words [0, words) of a frame (master warp; wrap-around sum, so
// the lane split gives the same value as one thread summing in order).
__device__ __forceinline__ uint32_t frame_sum(const uint32_t *f, uint32_t words) {
  uint32_t v = 0;
  for (uint32_t w = lane_id(); w < words; w += 32u) v += f[w];
  return warp_sum(v);
}

// ---------------------------------------------------------------------------
// Fork / join (master side) and the worker state machine
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void parallel(const Env &e, uint32_t work, uint32_t nthreads,
                                         uint32_t arg) {
  if (team_workers() == 0) {
    // no workers: the master runs the region as a team of one
    __syncwarp();
    if (lane_id() == 0)
      for (uint32_t v = 0; v < nthreads; ++v) P::body(e, work, v, nthreads, arg);
    __syncwarp();
    return;
  }
  if (lane_id() == 0) {
    Ctrl *c = ctrl();
    c->work = work;
    c->nthreads = nthreads;
    c->arg = arg;
  }
  named_bar(kForkBar, team_threads());  // release the workers
  named_bar(kJoinBar, team_threads());  // resume when they are done
}

// The worker state machine (Fig. "codegen-worker"): wait for work at the
// fork barrier, leave on terminate, run the body if selected, join.
template <class P>
__device__ __forceinline__ void worker_loop(const Env &e) {
  const uint32_t W = team_workers();
  for (;;) {
    named_bar(kForkBar, team_threads());
    const Ctrl *c = ctrl();
    const uint32_t work = c->work;
    if (work == kTerminate) break;
    const uint32_t n = c->nthreads, arg = c->arg;
    for (uint32_t v = threadIdx.x; v < n; v += W) P::body(e, work, v, n, arg);
    named_bar(kJoinBar, team_threads());
  }
}

__device__ __forceinline__ void terminate_workers() {
  if (team_workers() == 0) return;
  if (lane_id() == 0) ctrl()->work = kTerminate;
  named_bar(kForkBar, team_threads());
}

// Team exit (master warp): unwind what an error left live, then report.
__device__ __forceinline__ void team_report(const Env &e, dsr_team_status *st) {
  Ctrl *c = ctrl();
  const int32_t status = c->status;
  if (status != DSR_OK) {
    while (c->depth) {
      pop(c->frames[c->depth - 1].ptr);
    }
  }
  __syncwarp();
  if (lane_id() == 0) {
    dsr_team_status r;
    r.status = status;
    r.depth_final = c->depth;
    r.hwm_bytes = c->hwm;
    r.spill_bytes = c->spill;
#pragma unroll
    for (int k = 0; k < DSR_MAX_DEPTH; ++k) r.chk[k] = status == DSR_OK ? c->chk[k] : 0u;
    st[e.d->status_index + e.team] = r;
  }
}

__device__ __forceinline__ uint32_t region_width(const dsr_region_desc &d) {
  const uint32_t w = d.threads > 32u ? d.threads - 32u : 1u;
  return d.width ? d.width : w;
}

}  // namespace dsr
