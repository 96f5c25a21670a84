/*
 * dsr_serve_kernel.cuh -- the served launch form's server kernel (device
 * side), a template over the region program so that the library's
 * built-in programs and user-written ones (dsr_device.cuh,
 * dsr_serve_start_user) run the same server.
 *
 * A persistent kernel keeps every CTA's team stack live on the GPU and runs
 * region instances as the host submits them (continuous batching; the
 * paper's runtime launches one kernel per target region, Sec. 4). Block 0,
 * the doorbell, copies each new request's descriptor from the pinned
 * submit ring (host memory mapped into the device) into a device ring and
 * publishes the host's tail and stop flag in device memory. The other CTAs
 * claim runs of teams of the oldest requests in flight with a 64-bit
 * compare-and-swap on each request slot's claim word (request sequence <<
 * 32 | next team), run them through the program's master code and worker
 * state machine, count finished teams per slot and, at a request's last
 * team, recycle its slot and write a completion record {sequence + 1,
 * worst status} to the mapped completion ring. Every wait is bounded: a CTA
 * with no work for idle_timeout_ns leaves. The host side of the protocol
 * (rings, admission, restart after an idle exit) is in the library
 * (dsr_serve_start, dsr_serve_submit, dsr_serve_poll, dsr_serve_stop).
 */
#ifndef DSR_SERVE_KERNEL_CUH_
#define DSR_SERVE_KERNEL_CUH_

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "dsr.h"
#include "dsr_kernels.cuh"

namespace dsr {

struct alignas(16) CompRec {
  unsigned long long marker;  // request sequence + 1; 0 = empty
  int status;
  unsigned int pad;
};

struct HostShared {  // pinned, mapped
  unsigned long long tail;  // requests published
  unsigned long long stop;  // 1 = drain and exit
  unsigned long long pad[14];
};

static_assert(offsetof(dsr_region_desc, teams) == 4, "the doorbell reads teams as word 1");

struct alignas(32) SlotState {
  unsigned long long claim;  // (sequence << 32) | next team to hand out
  unsigned int teams;        // the request's teams (written by the doorbell)
  unsigned int done;         // teams finished
  int status;                // worst team status
  unsigned int pad[3];
};

struct ServeWs {  // device workspace header
  unsigned long long head;       // oldest request that may still have unclaimed teams
  unsigned long long comp_tail;  // completion records written
  unsigned long long tail;       // the doorbell's copy of the host's tail
  unsigned long long stop;       // the doorbell's copy of the host's stop flag
  unsigned int idle_exits;       // CTAs that left after the idle timeout
  unsigned int errors;           // teams rejected on the device
  unsigned int pad[22];
};

struct ServeArgs {
  const dsr_region_desc *ring;  // device view of the submit ring (host memory)
  dsr_region_desc *dring;       // device copy of the submit ring
  HostShared *hs;               // device view
  CompRec *comp;                // device view of the completion ring
  ServeWs *ws;
  SlotState *slots;
  const uint8_t *images;
  uint8_t *out;
  dsr_team_status *status;
  uint8_t *pool;
  uint64_t image_bytes;
  uint64_t out_bytes;
  uint64_t n_status;
  uint64_t ovf_per_cta;
  uint64_t timeout_ns;       // bound on fills
  uint64_t idle_timeout_ns;  // leave after this long without work
  uint32_t capacity;         // submit-ring slots (completion ring: same)
  uint32_t slab_bytes;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Claim a run of teams of request r if it has teams left (lane 0): about
// a sixteenth of what is left, at most kChunk, at least one. `advance` reports
// that r has no team left to hand out (all claimed, or r is done). Runs of
// two: longer runs hold a request's completion back behind one CTA working
// through several heavy teams in turn, one-team runs contend on the claim
// word (measured on the hetero distribution: p99 at 50k requests/s 322 us
// with runs of four, 228 us with two; runs of one lost throughput).
constexpr uint32_t kChunk = 2;

__device__ __forceinline__ bool claim_in(const ServeArgs &a, unsigned long long r,
                                         uint32_t *team, uint32_t *count, bool *advance) {
  const uint32_t slot = static_cast<uint32_t>(r % a.capacity);
  SlotState *st = a.slots + slot;
  const uint32_t T = *reinterpret_cast<volatile const unsigned int *>(&st->teams);
  unsigned long long w = ld_relaxed_gpu(&st->claim);
  *advance = false;
  for (int cas = 0; cas < 4; ++cas) {
    if ((w >> 32) != (r & 0xffffffffull) || static_cast<uint32_t>(w) >= T) {
      *advance = true;
      return false;
    }
    const uint32_t left = T - static_cast<uint32_t>(w);
    const uint32_t g = min(kChunk, max(1u, left / 16u));
    const unsigned long long prev = atomicCAS(&st->claim, w, w + g);
    if (prev == w) {
      *team = static_cast<uint32_t>(w);
      *count = g;
      return true;
    }
    w = prev;
  }
  return false;
}

// Claim teams of a submitted request (master warp). Returns false when
// no team is available now. The CTA first tries the request it ran last
// (`hint`). Then the warp looks at the kWindow oldest requests in flight at
// once, kWindow / 32 per lane, so their claim words are read in one round
// trip rather than one after another; lane 0 tries those with teams left,
// starting at one that depends on its block index so that claims spread
// over the window, and moves the head past every leading request that has
// no team left to hand out. (Closed-loop capacity on the hetero
// distribution, 128-thread CTAs: 423k requests/s with a window of 32, 633k
// with 64, 688k with 128.)
constexpr uint32_t kWindow = 128;  // requests looked at per try
constexpr uint32_t kWinPer = kWindow / 32;

__device__ __forceinline__ bool claim(const ServeArgs &a, unsigned long long hint,
                                      unsigned long long *seq, uint32_t *team, uint32_t *count) {
  const uint32_t lane = lane_id();
  unsigned long long out_seq = 0;
  uint32_t out_team = 0, out_count = 0, got = 0;
  if (lane == 0 && hint != ~0ull) {
    bool adv;
    if (claim_in(a, hint, &out_team, &out_count, &adv)) {
      got = 1;
      out_seq = hint;
    }
  }
  got = __shfl_sync(0xffffffffu, got, 0);
  for (uint32_t tries = 0; tries < 8 && !got; ++tries) {
    unsigned long long h = 0, tail = 0;
    if (lane == 0) {
      h = ld_relaxed_gpu(&a.ws->head);
      tail = ld_acquire_gpu(&a.ws->tail);  // the doorbell's slot writes before it
    }
    h = __shfl_sync(0xffffffffu, h, 0);
    tail = __shfl_sync(0xffffffffu, tail, 0);
    __syncwarp();  // orders lane 0's acquire before the other lanes' slot reads
    if (h >= tail) break;
    const uint32_t n = static_cast<uint32_t>(min(tail - h, static_cast<unsigned long long>(kWindow)));
    // lane l looks at requests h + 32k + l, all its loads issued first
    uint32_t T[kWinPer];
    unsigned long long w[kWinPer];
#pragma unroll
    for (uint32_t k = 0; k < kWinPer; ++k) {
      T[k] = 0;
      w[k] = 0;
      if (32u * k + lane < n) {
        const SlotState *st = a.slots + static_cast<uint32_t>((h + 32u * k + lane) % a.capacity);
        T[k] = *reinterpret_cast<volatile const unsigned int *>(&st->teams);
        w[k] = ld_relaxed_gpu(&st->claim);
      }
    }
    uint32_t avail_m[kWinPer], spent_m[kWinPer];
#pragma unroll
    for (uint32_t k = 0; k < kWinPer; ++k) {
      const uint32_t idx = 32u * k + lane;
      const unsigned long long r = h + idx;
      // teams left when the slot still holds r and not all are handed out;
      // otherwise r has none left (all handed out, or r done and its slot
      // passed on to a later request)
      const bool avail = idx < n && (w[k] >> 32) == (r & 0xffffffffull) &&
                         static_cast<uint32_t>(w[k]) < T[k];
      avail_m[k] = __ballot_sync(0xffffffffu, avail);
      spent_m[k] = __ballot_sync(0xffffffffu, idx < n && !avail);
    }
    if (lane == 0) {
      // the head passes every leading request with no team left
      uint32_t lead = 0;
      for (uint32_t k = 0; k < kWinPer; ++k) {
        const uint32_t run = ~spent_m[k] ? static_cast<uint32_t>(__ffs(~spent_m[k])) - 1u : 32u;
        lead += run;
        if (run < 32u) break;
      }
      if (lead) atomicCAS(&a.ws->head, h, h + lead);
      const uint32_t start = (blockIdx.x * 7u + tries) % n;
      for (uint32_t p = 0; p < n && !got; ++p) {
        const uint32_t idx = start + p < n ? start + p : start + p - n;
        if (!((avail_m[idx >> 5] >> (idx & 31u)) & 1u)) continue;
        bool adv;
        if (claim_in(a, h + idx, &out_team, &out_count, &adv)) {
          got = 1;
          out_seq = h + idx;
        }
      }
    }
    got = __shfl_sync(0xffffffffu, got, 0);
  }
  *seq = __shfl_sync(0xffffffffu, out_seq, 0);
  *team = __shfl_sync(0xffffffffu, out_team, 0);
  *count = __shfl_sync(0xffffffffu, out_count, 0);
  return got != 0;
}

template <class P, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) serve_kernel(const __grid_constant__ ServeArgs a) {
  Env e;
  e.d = nullptr;
  e.images = a.images;
  e.out = a.out;
  e.team = 0;
  if (threadIdx.x < team_workers()) {
    worker_loop<P, true>(e);
    return;
  }
  const uint32_t lane = lane_id();
  if (blockIdx.x == 0) {
    // The doorbell (block 0, the first to be scheduled): the main reader of
    // host memory. For every new request it copies the descriptor into the
    // device ring (the warp's lanes copy 16 bytes each), then publishes the
    // new tail (and a stop) in device memory, where the other CTAs poll. It
    // leaves on stop or after idle_timeout_ns without a new request.
    unsigned long long last = ld_relaxed_gpu(&a.ws->tail);
    uint64_t idle_since = globaltimer();
    for (;;) {
      unsigned long long stop = 0, t = 0;
      if (lane == 0) {
        stop = ld_acquire_sys(&a.hs->stop);
        t = ld_acquire_sys(&a.hs->tail);
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t > last) {
        for (unsigned long long r = last + lane / 4u; r < t; r += 8u) {
          const uint32_t slot = static_cast<uint32_t>(r % a.capacity);
          const uint4 q = reinterpret_cast<const uint4 *>(a.ring + slot)[lane & 3u];
          reinterpret_cast<uint4 *>(a.dring + slot)[lane & 3u] = q;
          if ((lane & 3u) == 0) a.slots[slot].teams = q.y;  // dsr_region_desc::teams
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicMax(&a.ws->tail, t);
        last = t;
        idle_since = globaltimer();
      }
      if (stop) {
        if (lane == 0) atomicExch(&a.ws->stop, 1ull);
        break;
      }
      if (globaltimer() - idle_since > a.idle_timeout_ns) {
        if (lane == 0) atomicAdd(&a.ws->idle_exits, 1u);
        break;
      }
      __nanosleep(256);
    }
    __syncwarp();
    terminate_workers();
    return;
  }
  Ctrl *c = ctrl();
  Stack s;
  uint8_t *ovf = a.ovf_per_cta ? a.pool + static_cast<uint64_t>(blockIdx.x) * a.ovf_per_cta : nullptr;
  bool first = true;
  uint64_t idle_since = globaltimer();
  uint32_t backoff = 256;
  unsigned long long hint = ~0ull;
  unsigned long long cached = ~0ull;  // request whose descriptor is in the control block
  bool cached_ok = false;
  for (;;) {
    unsigned long long seq;
    uint32_t team0, count;
    if (!claim(a, hint, &seq, &team0, &count)) {
      hint = ~0ull;
      // nothing to run: leave when asked to stop (all submitted work has
      // been claimed) or after the idle timeout; otherwise back off
      unsigned long long stop = 0;
      if (lane == 0) {
        stop = ld_acquire_gpu(&a.ws->stop);
        // a few CTAs also look at the host's stop flag now and then, so a
        // stop is seen even when the doorbell has left
        if (!stop && (blockIdx.x & 63u) == 1u && backoff >= 4096 &&
            ld_acquire_sys(&a.hs->stop))
          atomicExch(&a.ws->stop, 1ull);
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (stop) break;
      if (globaltimer() - idle_since > a.idle_timeout_ns) {
        if (lane == 0) atomicAdd(&a.ws->idle_exits, 1u);
        break;
      }
      __nanosleep(backoff);
      backoff = backoff < 4096 ? backoff * 2 : 4096;
      continue;
    }
    backoff = 256;
    hint = seq;
    idle_since = globaltimer();
    const uint32_t slot = static_cast<uint32_t>(seq % a.capacity);
    if (seq != cached) {
      __syncwarp();
      if (lane < 4)
        reinterpret_cast<uint4 *>(&c->desc)[lane] =
            reinterpret_cast<const uint4 *>(a.dring + slot)[lane];
      __syncwarp();
      cached = seq;
      cached_ok = program_fits<P>(c->desc, a.image_bytes, a.out_bytes, a.n_status);
    }
    const dsr_region_desc &d = c->desc;
    int32_t worst = DSR_OK;
    for (uint32_t team = team0; team < team0 + count; ++team) {
      if (lane == 0) c->team = team;
      e.d = &c->desc;
      e.team = team;
      team_setup(s, a.slab_bytes, ovf, a.ovf_per_cta, a.timeout_ns, first);
      if (first) s.bits |= kAccArea;
      first = false;
      int32_t st;
      if (!cached_ok) {
        st = DSR_ERR_INVALID;
        if (lane == 0) {
          atomicAdd(&a.ws->errors, 1u);
          const uint64_t si = static_cast<uint64_t>(d.status_index) + team;
          if (si < a.n_status) {
            dsr_team_status r = {};
            r.status = DSR_ERR_INVALID;
            a.status[si] = r;
          }
        }
      } else {
        P::master(e, s);
        st = s.status();
        team_report(e, s, a.status);
      }
      worst = max(worst, st);
    }
    if (lane == 0) {
      __threadfence();  // these teams' outputs before their completion count
      if (worst != DSR_OK) atomicMax(&a.slots[slot].status, worst);
      const uint32_t done = atomicAdd(&a.slots[slot].done, count) + count;
      if (done == d.teams) {
        // the request's last team: recycle the slot for request seq +
        // capacity, then publish the completion to the host
        __threadfence();
        const int rst = atomicAdd(&a.slots[slot].status, 0);
        a.slots[slot].done = 0;
        a.slots[slot].status = 0;
        __threadfence();
        atomicExch(&a.slots[slot].claim, ((seq + a.capacity) & 0xffffffffull) << 32);
        const unsigned long long pos = atomicAdd(&a.ws->comp_tail, 1ull);
        CompRec *r = a.comp + (pos % a.capacity);
        r->status = rst;
        __threadfence_system();
        st_release_sys(&r->marker, seq + 1);
      }
    }
    __syncwarp();
  }
  terminate_workers();
}

using ServeFn = void (*)(ServeArgs);

template <class P>
ServeFn pick_serve(uint32_t threads) {
  if (threads <= 128) return serve_kernel<P, 128, 8>;
  if (threads <= 256) return serve_kernel<P, 256, 4>;
  return serve_kernel<P, 1024, 1>;
}

}  // namespace dsr

#endif  // DSR_SERVE_KERNEL_CUH_
