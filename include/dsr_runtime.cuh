// dsr_runtime.cuh -- device side of the generic-mode data-sharing runtime.
//
// One team = one CTA of N threads: one warp of 32 threads holds the master
// thread (its lane 0) and the other W = N - 32 threads are the workers, as
// in Sec. 4, which sets a whole warp aside for the master so that the
// master's sequential code never diverges a warp that workers share. As
// there, the master warp is the CTA's last warp and the workers are threads
// 0..W-1. (Warp 0 as the master warp was measured: 8.20 -> 8.34 us per
// launch of the nested program, the batched form 1 % slower.) Lanes 1..31
// of the master warp stay resident: they take part in every barrier and
// help with runtime-owned copies, so no thread of a barrier's warp count has
// exited.
//
// Handoff (Sec. 4, Fig. "codegen-master" / "codegen-worker"): workers wait
// at the fork barrier while the master runs sequential code; the master
// publishes the work (body id, thread count, argument) and the frame table,
// arrives at the fork barrier, and waits at the join barrier until the
// workers finish the body. Named barriers (Sec. 4 drives the master and the
// workers with them) keep fork and join apart, each used as a
// producer/consumer pair with the team's thread
// count: at the fork the master arrives (bar.arrive, it need not wait) and
// the workers wait (bar.sync); at the join the workers arrive and the
// master waits. Workers beyond the region's thread count skip the body but
// still reach the join (the exec_status test of Fig. "codegen-worker").
//
// Shared locals (Sec. 5.1-5.3): the master pushes a frame per call level on
// a LIFO stack. The stack pointers (slab and overflow) live in registers of
// the master warp, identical in all 32 lanes, as the paper's shared stack
// pointer register does (Sec. 5.3, %SPSH / VRShared); lane 0 records each
// frame in the control block's frame table. A frame goes to the team's shared-memory slab when it fits, otherwise to
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
constexpr uint32_t kWorkerBar = 3;  // the workers alone, inside a region the runtime runs
constexpr uint32_t kTerminate = 0xFFFFFFFFu;
constexpr uint32_t kCopyWork = 0xFFFFFFF0u;  // runtime-internal: workers copy a frame image
constexpr uint32_t kCtrlBytes = 384;  // control block, slab starts after it
constexpr uint32_t kParallelCopyBytes = 2048;  // frames filled by the workers from this size
constexpr uint32_t kStreamChunks = 8;          // mbarriers of a streamed fill
constexpr uint32_t kStreamMinBytes = 16384;    // slab frames streamed from this size
// The persistent kernels (batched, served) give every CTA, after its slab, a
// region-wide accumulator of one word per thread a region may have
// (programs whose regions reduce into per-thread sums use it).
constexpr uint32_t kAccBytes = 4u * DSR_MAX_THREADS;
constexpr uint32_t kAccArea = 1u << 25;  // Stack::bits: this CTA has that area

struct FrameEnt {
  uint8_t *ptr;      // generic address of the frame (shared or global)
  uint32_t bytes;    // requested size
  uint32_t in_smem;  // 1 = slab, 0 = overflow slab
};

struct __align__(16) Ctrl {
  // handoff: written by the master before the fork, read by the workers
  uint32_t work;      // body id of the current parallel region or kTerminate
  uint32_t nthreads;  // threads of the current parallel region
  uint32_t arg;       // per-region argument (level, region index)
  uint32_t acc;       // a wrap-around sum the workers of a region add up (reset by the master)
  uint64_t mbar;      // mbarrier completing bulk-copy fills
  uint64_t timeout_ns;
  uint8_t *ovf;       // this team's overflow slab
  uint64_t ovf_bytes;
  uint32_t slab_bytes;  // capacity of the shared-memory slab
  uint32_t team;        // batched launch: the current task's team
  uint32_t whwm;    // worker-level stacks: sum of the warp stacks' peak bytes
  uint32_t wspill;  // ... and of their peak overflow bytes
  FrameEnt frames[DSR_MAX_FRAMES];
  dsr_region_desc desc;  // batched launch: the current task's region
  const uint8_t *copy_src;  // kCopyWork arguments
  uint8_t *copy_dst;
  uint32_t copy_bytes;
  uint32_t copy_key;
  // streamed fill: chunk k of the frame completes on chunk_bar[k]
  uint64_t chunk_bar[kStreamChunks];
  uint32_t stream_shift;  // log2 of the chunk size
  uint16_t stream_phase;  // parity the chunk barriers complete with this fill
  uint16_t stream_err;    // a worker's wait for a chunk ran out
  // worker-level stacks: each worker warp's share of what the team's slab
  // and overflow slab have left (set by the master before the fork)
  uint32_t wstack_off;   // shared-memory offset of warp 0's slab share
  uint32_t wslab;        // slab bytes per warp (a multiple of 16)
  uint8_t *wovf;         // warp 0's overflow share
  uint64_t wovf_bytes;   // overflow bytes per warp (a multiple of 16)
  uint32_t wfail;        // a worker frame fitted neither share
  uint32_t copy_x0;      // kCopyWork: XOR of word 0 on top of copy_key
};
static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block too large");

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void named_bar(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void named_arrive(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
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
}

// Makes mbarrier initialisations visible before their first use.
__device__ __forceinline__ void mbar_init_fence() {
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

// Hint: pull [src, src + bytes) into L2 (bulk prefetch; src 16-byte
// aligned, bytes a multiple of 16). Issued by one thread; no completion.
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
  if (((reinterpret_cast<uintptr_t>(src) | bytes) & 15u) != 0) return;
  const uint8_t *p = static_cast<const uint8_t *>(src);
  for (uint32_t off = 0; off < bytes; off += 65536u) {
    const uint32_t n = bytes - off < 65536u ? bytes - off : 65536u;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + off), "r"(n) : "memory");
  }
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

// Sum over the warp (wrap-around), in every lane: one warp reduction.
__device__ __forceinline__ uint32_t warp_sum(uint32_t v) { return __reduce_add_sync(0xffffffffu, v); }

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

// The master warp's stack state, in registers, identical in all 32 lanes.
// Nothing here is read back from memory on the handoff path: a load issued
// right after the join barrier waits for the workers' outstanding stores,
// so push and pop work from registers alone (the frame table in the control
// block is written for the workers, never read by the master's pop).
struct Stack {
  uint32_t slab_bytes;  // capacity of the shared-memory slab
  uint32_t sp;          // slab bytes reserved
  uint32_t gsp;         // overflow-slab bytes reserved
  uint32_t hwm;         // peak reserved bytes, slab + overflow
  uint32_t spill;       // peak reserved overflow bytes
  uint32_t chk;         // lane k < DSR_MAX_DEPTH: the program's check word k
  uint32_t bits;        // status (bits 0-7) | fill-mbarrier parity (bit 8) |
                        // staged copy pending (bit 9) | streamed-fill parity
                        // (bit 10) | streamed fill pending (bit 11) | live
                        // depth (bits 12-15) | frame k in the slab (bit 16 + k)
                        // | streamed-fill mbarriers initialised (bit 24)
                        // | accumulator area after the slab (bit 25)

  __device__ __forceinline__ int32_t status() const { return static_cast<int32_t>(bits & 0xffu); }
  __device__ __forceinline__ uint32_t phase() const { return (bits >> 8) & 1u; }
  __device__ __forceinline__ uint32_t depth() const { return (bits >> 12) & 0xfu; }
};

// Programmatic dependent launch (an attribute of the plain form's launch):
// the next grid in the stream may be dispatched once every CTA of this grid
// has signalled, so its CTAs are placed and set up while this grid drains;
// every thread of a grid waits for the grids before it to complete, their
// memory visible, before its first global-memory access. In a grid launched
// without the attribute both are no-ops.
__device__ __forceinline__ void signal_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void wait_prerequisites() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Team setup (master warp): the stack starts empty. `first` initialises the
// fill mbarrier (once per CTA).
__device__ __forceinline__ void team_setup(Stack &s, uint32_t slab_bytes, uint8_t *ovf,
                                           uint64_t ovf_bytes, uint64_t timeout_ns, bool first) {
  Ctrl *c = ctrl();
  if (lane_id() == 0) {
    c->ovf = ovf;
    c->ovf_bytes = ovf_bytes;
    c->timeout_ns = timeout_ns;
    c->slab_bytes = slab_bytes;
    if (first) {
      mbar_init(&c->mbar, 1);
      mbar_init_fence();
    }
  }
  // the mbarriers' parities (fill: bit 8, streamed fill: bit 10) and the
  // streamed fill's set-up flag (bit 24) and the accumulator area (bit 25)
  // carry over
  s.bits = first ? 0u : (s.bits & 0x3000500u);
  s.slab_bytes = slab_bytes;
  s.sp = 0;
  s.gsp = 0;
  s.hwm = 0;
  s.spill = 0;
  s.chk = 0;
  __syncwarp();
}

// Record the program's check word k (the same value in every lane): lane k
// keeps it in a register until the team reports.
__device__ __forceinline__ void set_chk(Stack &s, uint32_t k, uint32_t v) {
  if (lane_id() == k) s.chk = v;
}

__device__ __forceinline__ void set_status(Stack &s, int32_t st) {
  if (s.status() == DSR_OK) s.bits = (s.bits & ~0xffu) | static_cast<uint32_t>(st);
}

// Push `bytes` (whole master warp). Returns the frame's generic address, or
// nullptr with status OVERFLOW when neither slab has room or the frame table
// is full.
__device__ __forceinline__ uint8_t *push(Stack &s, uint32_t bytes, bool *in_smem = nullptr) {
  const uint32_t fp = (bytes + 15u) & ~15u;
  if (s.status() != DSR_OK) return nullptr;
  const uint32_t depth = s.depth();
  uint8_t *p = nullptr;
  uint32_t sm = 0;
  if (depth < DSR_MAX_FRAMES) {
    if (s.sp + fp <= s.slab_bytes) {
      p = slab_base() + s.sp;
      sm = 1;
    } else {
      const Ctrl *c = ctrl();  // overflow path: read the team's overflow slab
      if (static_cast<uint64_t>(s.gsp) + fp <= c->ovf_bytes) p = c->ovf + s.gsp;
    }
  }
  if (!p) {
    set_status(s, DSR_ERR_OVERFLOW);
    return nullptr;
  }
  if (sm)
    s.sp += fp;
  else
    s.gsp += fp;
  s.bits = (s.bits & ~0xf000u) | ((depth + 1u) << 12) | (sm << (16u + depth));
  if (lane_id() == 0) {
    Ctrl *c = ctrl();
    FrameEnt f;
    f.ptr = p;
    f.bytes = bytes;
    f.in_smem = sm;
    c->frames[depth] = f;
  }
  s.hwm = max(s.hwm, s.sp + s.gsp);
  s.spill = max(s.spill, s.gsp);
  if (in_smem) *in_smem = sm != 0;
  return p;
}

// Pop the top frame `p` of `bytes` bytes. A frame's address is unique while
// it is live, so `p` is the top frame exactly when it ends at the stack
// pointer of the slab the top frame was placed in; anything else is LIFO
// misuse (status LIFO, nothing popped).
__device__ __forceinline__ int32_t pop(Stack &s, const uint8_t *p, uint32_t bytes) {
  const uint32_t fp = (bytes + 15u) & ~15u;
  const uint32_t depth = s.depth();
  bool ok = depth != 0;
  uint32_t sm = 0;
  if (ok) {
    sm = (s.bits >> (16u + depth - 1u)) & 1u;
    if (sm) {
      ok = fp <= s.sp && p == slab_base() + (s.sp - fp);
    } else {
      const Ctrl *c = ctrl();  // overflow path
      ok = fp <= s.gsp && p == c->ovf + (s.gsp - fp);
    }
  }
  if (!ok) {
    set_status(s, DSR_ERR_LIFO);
    return DSR_ERR_LIFO;
  }
  if (sm)
    s.sp -= fp;
  else
    s.gsp -= fp;
  s.bits = (s.bits & ~(0xf000u | (1u << (16u + depth - 1u)))) | ((depth - 1u) << 12);
  return DSR_OK;
}

// Pop whatever is on top (error unwinding; reads the frame table).
__device__ __forceinline__ void pop_top(Stack &s) {
  __syncwarp();
  const FrameEnt f = ctrl()->frames[s.depth() - 1];
  const int32_t keep = s.status();
  s.bits &= ~0xffu;
  pop(s, f.ptr, f.bytes);
  s.bits = (s.bits & ~0xffu) | static_cast<uint32_t>(keep);
}

// kDepth 16-byte loads in flight for one thread's vectors i, i + nthr, ...
// below nv, then their stores XOR key; returns the first vector not copied.
template <uint32_t kDepth>
__device__ __forceinline__ uint32_t copy_xor_batches(uint4 *dv, const uint4 *sv, uint32_t nv,
                                                     uint32_t key, uint32_t i, uint32_t nthr) {
  for (; i + (kDepth - 1u) * nthr < nv; i += kDepth * nthr) {
    uint4 x[kDepth];
#pragma unroll
    for (uint32_t u = 0; u < kDepth; ++u) x[u] = __ldg(sv + i + u * nthr);
#pragma unroll
    for (uint32_t u = 0; u < kDepth; ++u) {
      x[u].x ^= key;
      x[u].y ^= key;
      x[u].z ^= key;
      x[u].w ^= key;
      dv[i + u * nthr] = x[u];
    }
  }
  return i;
}

// dst[w] = src[w] ^ key for the words of `bytes` (a multiple of 4), split
// over `nthr` threads (this one is `idx`); 16-byte vectors when aligned.
// Up to kDepth vector loads are in flight per thread before their stores:
// a copy between two global buffers is bound by the bytes in flight. Rounds
// of kDepth, then of 4, then single vectors, so that frames too small for a
// full round of kDepth still keep several loads in flight. Each step of
// depth costs four registers (1 in kernels held to 32).
template <uint32_t kDepth>
__device__ __forceinline__ void copy_xor(uint8_t *dst, const uint8_t *src, uint32_t bytes,
                                         uint32_t key, uint32_t idx, uint32_t nthr) {
  uint32_t w0 = 0;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const uint32_t nv = bytes / 16u;
    const uint4 *sv = reinterpret_cast<const uint4 *>(src);
    uint4 *dv = reinterpret_cast<uint4 *>(dst);
    uint32_t i = idx;
    if (kDepth > 4u) i = copy_xor_batches<(kDepth > 4u ? kDepth : 4u)>(dv, sv, nv, key, i, nthr);
    if (kDepth > 1u) i = copy_xor_batches<(kDepth > 1u ? 4u : 1u)>(dv, sv, nv, key, i, nthr);
    i = copy_xor_batches<1u>(dv, sv, nv, key, i, nthr);
    w0 = nv * 4u;
  }
  const uint32_t *sw = reinterpret_cast<const uint32_t *>(src);
  uint32_t *dw = reinterpret_cast<uint32_t *>(dst);
  for (uint32_t w = w0 + idx; w < bytes / 4u; w += nthr) dw[w] = __ldg(sw + w) ^ key;
}

// Fill a frame from a global image, word by word XOR `key`, word 0 also XOR
// `x0` (master warp). Shared-memory frames with 16-byte aligned source and
// size take one bulk copy issued by the master (a single thread moves the
// whole frame) and are then keyed in place; other frames are copied by the
// 32 lanes, with 16-byte vector accesses where alignment allows (kWide) or
// word by word (the register-lean form used by kernels held to 32
// registers), or by the workers when large. Word 0 is XORed by the thread
// that copies it, so a frame in global memory takes no extra round trip.
template <bool kWide>
__device__ __forceinline__ void fill(Stack &s, uint8_t *dst, bool dst_smem, const uint8_t *src,
                                     uint32_t bytes, uint32_t key, uint32_t x0 = 0) {
  const uint32_t lane = lane_id();
  const bool aligned = ((reinterpret_cast<uintptr_t>(src) | bytes) & 15u) == 0;
  if (dst_smem && aligned && bytes >= 64) {
    Ctrl *c = ctrl();
    uint64_t *bar = &c->mbar;
    const uint32_t phase = s.phase();
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
      set_status(s, DSR_ERR_TIMEOUT);
    }
    s.bits ^= 0x100u;
    if (key != 0 || x0 != 0) {
      uint4 *v = reinterpret_cast<uint4 *>(dst);
      for (uint32_t i = lane; i < bytes / 16u; i += 32u) {
        uint4 x = v[i];
        x.x ^= key ^ (i == 0 ? x0 : 0u);
        x.y ^= key;
        x.z ^= key;
        x.w ^= key;
        v[i] = x;
      }
    }
  } else if (bytes >= kParallelCopyBytes) {
    // a large frame outside the slab: the workers copy it (a runtime-owned
    // initialisation between two fork/join barriers, no user code runs)
    if (lane == 0) {
      Ctrl *c = ctrl();
      c->work = kCopyWork;
      c->copy_src = src;
      c->copy_dst = dst;
      c->copy_bytes = bytes;
      c->copy_key = key;
      c->copy_x0 = x0;
    }
    named_arrive(kForkBar, team_threads());
    named_bar(kJoinBar, team_threads());
  } else if (kWide &&
             ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const uint32_t nv = bytes / 16u;
    const uint4 *sv = reinterpret_cast<const uint4 *>(src);
    uint4 *dv = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i = lane; i < nv; i += 64u) {
      uint4 y0 = __ldg(sv + i), x1 = make_uint4(0, 0, 0, 0);
      const bool two = i + 32u < nv;
      if (two) x1 = __ldg(sv + i + 32u);
      y0.x ^= key ^ (i == 0 ? x0 : 0u);
      y0.y ^= key;
      y0.z ^= key;
      y0.w ^= key;
      dv[i] = y0;
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
    for (uint32_t w = nv * 4u + lane; w < bytes / 4u; w += 32u)
      dw[w] = __ldg(sw + w) ^ key ^ (w == 0 ? x0 : 0u);
  } else {
    const uint32_t *sw = reinterpret_cast<const uint32_t *>(src);
    uint32_t *dw = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t w = lane; w < bytes / 4u; w += 32u)
      dw[w] = __ldg(sw + w) ^ key ^ (w == 0 ? x0 : 0u);
  }
  __syncwarp();
}

// Eager staging. When the frames a team will push next all fit in the
// slab, their addresses are known before the pushes (the slab is a bump
// allocator and frames are pushed in order), so the master can start one
// bulk copy per frame image at once, into those future slots, and pay the
// memory latency once instead of once per level. stage() issues the copy
// (source 16-byte aligned, size a multiple of 16) and returns whether it
// did. The images must lie in memory as the frames will in the slab: in
// push order, each padded to 16 bytes, so one contiguous copy stages them
// all. wait_staged() waits for the copy (once, before the first staged
// frame is used); key_in_place() then completes each frame's fill.
__device__ __forceinline__ bool stage(Stack &s, const uint8_t *src, uint32_t total) {
  if (((reinterpret_cast<uintptr_t>(src) | total) & 15u) || total == 0 ||
      s.sp + total > s.slab_bytes || s.status() != DSR_OK)
    return false;
  if (lane_id() == 0) {
    Ctrl *c = ctrl();
    fence_proxy_async_smem();
    mbar_expect_tx(&c->mbar, total);
    for (uint32_t off = 0; off < total; off += 32768u) {
      const uint32_t n = total - off < 32768u ? total - off : 32768u;
      bulk_g2s(slab_base() + s.sp + off, src + off, n, &c->mbar);
    }
  }
  s.bits |= 0x200u;
  __syncwarp();
  return true;
}

__device__ __forceinline__ void wait_staged(Stack &s) {
  if (!(s.bits & 0x200u)) return;
  s.bits &= ~0x200u;
  Ctrl *c = ctrl();
  const uint32_t phase = s.phase();
  const uint64_t tmo = c->timeout_ns;
  if (!mbar_wait(&c->mbar, phase, tmo)) {
    mbar_wait(&c->mbar, phase, tmo);
    set_status(s, DSR_ERR_TIMEOUT);
  }
  s.bits ^= 0x100u;
}

// XOR every word of a staged frame with `key` (master warp). The frame's
// slot is reserved in 16-byte units, so the whole slot is keyed (the words
// past `bytes` are the slot's padding).
__device__ __forceinline__ void key_in_place(uint8_t *dst, uint32_t bytes, uint32_t key) {
  if (key != 0) {
    uint4 *v = reinterpret_cast<uint4 *>(dst);
    for (uint32_t i = lane_id(); i < (bytes + 15u) / 16u; i += 32u) {
      uint4 x = v[i];
      x.x ^= key;
      x.y ^= key;
      x.z ^= key;
      x.w ^= key;
      v[i] = x;
    }
  }
  __syncwarp();
}

// Streamed fill. A large slab frame's image is copied in up to
// kStreamChunks power-of-two chunks, chunk k completing on chunk_bar[k],
// and the master forks right away: the parallel region starts while the
// image is still arriving, and a worker waits for a chunk only when its
// reads first reach it (stream_ready). Every element is still read after
// it has landed, so the region sees the frame the master filled; the
// copy's latency overlaps the region instead of preceding it. The source
// must be 16-byte aligned and the size a multiple of 16 (else false: use
// fill()). stream_finish() (master, after the join) waits for every chunk
// before the frame may be popped.
__device__ __forceinline__ bool fill_streamed(Stack &s, uint8_t *dst, const uint8_t *src,
                                              uint32_t bytes) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | bytes) & 15u) ||
      bytes == 0 || (s.bits & 0x800u) || s.status() != DSR_OK)
    return false;
  uint32_t shift = 12;
  while ((kStreamChunks << shift) < bytes) ++shift;
  if (shift > 15) return false;  // chunks above 32 KiB: not streamed
  if (lane_id() == 0) {
    Ctrl *c = ctrl();
    if (!(s.bits & 0x1000000u)) {  // first streamed fill of this CTA
      for (uint32_t k = 0; k < kStreamChunks; ++k) mbar_init(&c->chunk_bar[k], 1);
      mbar_init_fence();
    }
    fence_proxy_async_smem();
    // every chunk barrier completes one phase per streamed fill (chunks past
    // the frame's end with no bytes), so one parity serves them all
    for (uint32_t k = 0; k < kStreamChunks; ++k) {
      const uint32_t off = k << shift;
      const uint32_t n = off < bytes ? min(bytes - off, 1u << shift) : 0u;
      mbar_expect_tx(&c->chunk_bar[k], n);
      if (n) bulk_g2s(dst + off, src + off, n, &c->chunk_bar[k]);
    }
    c->stream_shift = shift;
    c->stream_phase = static_cast<uint16_t>((s.bits >> 10) & 1u);
    c->stream_err = 0;
  }
  s.bits |= 0x1000800u;
  __syncwarp();
  return true;
}

// Worker side: make sure bytes [0, byte_end) of the streamed frame have
// landed, given that [0, ready) are known to have. Returns the new bound
// (a chunk boundary at or past byte_end). A wait that runs out flags the
// fill (the master reports TIMEOUT) and goes on.
__device__ __forceinline__ uint32_t stream_ready(uint32_t byte_end, uint32_t ready) {
  Ctrl *c = ctrl();
  const uint32_t shift = c->stream_shift, ph = c->stream_phase;
  const uint32_t last = (byte_end - 1u) >> shift;
  for (uint32_t k = ready >> shift; k <= last; ++k)
    if (!mbar_wait(&c->chunk_bar[k], ph, c->timeout_ns)) c->stream_err = 1;
  return (last + 1u) << shift;
}

// Master warp, after the join: wait (bounded) for every chunk of a
// streamed fill, then flip the parity for the next one.
__device__ __forceinline__ void stream_finish(Stack &s) {
  if (!(s.bits & 0x800u)) return;
  s.bits &= ~0x800u;
  Ctrl *c = ctrl();
  const uint32_t ph = (s.bits >> 10) & 1u;
  bool ok = c->stream_err == 0;
  for (uint32_t k = 0; k < kStreamChunks; ++k) {
    if (!mbar_wait(&c->chunk_bar[k], ph, c->timeout_ns)) {
      mbar_wait(&c->chunk_bar[k], ph, c->timeout_ns);  // copies still in flight
      ok = false;
    }
  }
  if (!ok) set_status(s, DSR_ERR_TIMEOUT);
  s.bits ^= 0x400u;
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Fork / join (master side) and the worker state machine
// ---------------------------------------------------------------------------
// Every launch gives a team at least one worker warp: a team declared with
// no workers (32 threads) runs with one extra warp and a region width of 1,
// which is the team of one such a region has. The master never runs a body.
// fork() publishes the work and releases the workers; join() waits for
// them. parallel() is the two back to back; a master that has runtime work
// of its own (filling frames it will push later) does it between them.
template <class P>
__device__ __forceinline__ void fork(const Env &e, uint32_t work, uint32_t nthreads,
                                     uint32_t arg) {
  if (lane_id() == 0) {
    Ctrl *c = ctrl();
    c->work = work;
    c->nthreads = nthreads;
    c->arg = arg;
  }
  named_arrive(kForkBar, team_threads());  // release the workers
}

__device__ __forceinline__ void join() {
  named_bar(kJoinBar, team_threads());  // resume when the workers are done
}

template <class P>
__device__ __forceinline__ void parallel(const Env &e, uint32_t work, uint32_t nthreads,
                                         uint32_t arg) {
  fork<P>(e, work, nthreads, arg);
  join();
}

// The worker state machine (Fig. "codegen-worker"): wait for work at the
// fork barrier, leave on terminate, run the body if selected, join. A
// region wider than the CTA's workers runs its threads round robin on them
// (thread v on worker v mod W); the bodies have no barriers, so any order
// of a worker's threads is one of the region's schedules. In a batched
// launch (kBatched) the region and team change from task to task and are
// read from the control block at every fork.
template <class P, bool kBatched = false>
__device__ __forceinline__ void worker_loop(const Env &e0) {
  const uint32_t W = team_workers();
  Env e = e0;
  for (;;) {
    named_bar(kForkBar, team_threads());
    const Ctrl *c = ctrl();
    const uint32_t work = c->work;
    if (work == kTerminate) break;
    if (work == kCopyWork) {
      copy_xor<P::kDense ? 1u : kBatched ? 4u : 8u>(c->copy_dst, c->copy_src, c->copy_bytes,
                                                   c->copy_key, threadIdx.x, W);
      // worker 0 copied word 0 (the first vector, or the first word): its
      // extra XOR, read back from the thread's own store
      if (threadIdx.x == 0 && c->copy_x0)
        reinterpret_cast<uint32_t *>(c->copy_dst)[0] ^= c->copy_x0;
      named_arrive(kJoinBar, team_threads());
      continue;
    }
    const uint32_t n = c->nthreads, arg = c->arg;
    if (kBatched) {
      e.d = &c->desc;
      e.team = c->team;
    }
    P::run(e, work, threadIdx.x, W, n, arg);
    named_arrive(kJoinBar, team_threads());
  }
}

// A worker's share of a parallel region: its virtual threads v = first,
// first + W, ... below n, each running the body. Programs may provide their
// own `run` that hoists per-region values out of the loop over v.
template <class P>
__device__ __forceinline__ void run_threads(const Env &e, uint32_t work, uint32_t first,
                                            uint32_t W, uint32_t n, uint32_t arg) {
  for (uint32_t v = first; v < n; v += W) P::body(e, work, v, n, arg);
}

__device__ __forceinline__ void terminate_workers() {
  if (lane_id() == 0) ctrl()->work = kTerminate;
  named_arrive(kForkBar, team_threads());
}

// Team exit (master warp): unwind what an error left live, then report.
__device__ __forceinline__ void team_report(const Env &e, Stack &s, dsr_team_status *st) {
  wait_staged(s);  // no bulk copy may still be landing in the slab
  stream_finish(s);
  const int32_t status = s.status();
  if (status != DSR_OK) {
    while (s.depth()) pop_top(s);
  }
  __syncwarp();
  // the check words come from lanes 0..DSR_MAX_DEPTH-1 (no memory read
  // after the last join)
  uint32_t chk[DSR_MAX_DEPTH];
#pragma unroll
  for (int k = 0; k < DSR_MAX_DEPTH; ++k) chk[k] = __shfl_sync(0xffffffffu, s.chk, k);
  if (lane_id() == 0) {
    dsr_team_status r;
    r.status = status;
    r.depth_final = s.depth();
    r.hwm_bytes = s.hwm;
    r.spill_bytes = s.spill;
#pragma unroll
    for (int k = 0; k < DSR_MAX_DEPTH; ++k) r.chk[k] = status == DSR_OK ? chk[k] : 0u;
    st[e.d->status_index + e.team] = r;
  }
}

// Shared-memory offset of the CTA's accumulator area (0: none).
__device__ __forceinline__ uint32_t acc_area(const Stack &s) {
  return (s.bits & kAccArea) ? kCtrlBytes + s.slab_bytes : 0u;
}

__device__ __forceinline__ uint32_t region_width(const dsr_region_desc &d) {
  const uint32_t w = d.threads > 32u ? d.threads - 32u : 1u;
  return d.width ? d.width : w;
}

}  // namespace dsr
