// dsr_kernels.cuh -- the kernels every region program runs in: the plain
// per-region kernel (one CTA per team) and the persistent batched kernel
// (a fixed grid pulling (instance, team) tasks). Both are templates over a
// program P, so the library's built-in programs and programs a user writes
// against dsr_device.cuh are launched by the same code.
//
// A program P provides:
//   static constexpr uint32_t kProgram;  the id its descriptors carry
//   static constexpr bool kDense;        teams fill the GPU: 32 registers
//   __device__ static void master(const Env &, Stack &);    sequential code
//   __device__ static void run(const Env &, uint32_t work, uint32_t first,
//                              uint32_t W, uint32_t n, uint32_t arg);
//                                        a worker's share of a region
// and, when its buffer extents are not those of a built-in program
// (user-written programs), kUser = true and
//   __host__ __device__ static void extent(const dsr_region_desc &,
//                                          uint64_t *image_bytes,
//                                          uint64_t *out_bytes);
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <type_traits>
#include <vector>

#include "dsr.h"
#include "dsr_check.cuh"
#include "dsr_runtime.cuh"

namespace dsr {

// ---------------------------------------------------------------------------
// Program traits
// ---------------------------------------------------------------------------
template <class P, class = void>
struct is_user : std::false_type {};
template <class P>
struct is_user<P, std::void_t<decltype(P::kUser)>> : std::bool_constant<P::kUser> {};

template <class P, class = void>
struct wide_regs : std::false_type {};
template <class P>
struct wide_regs<P, std::void_t<decltype(P::kWideRegs)>> : std::bool_constant<P::kWideRegs> {};

// Programs whose teams' input ranges follow from the descriptor alone name
// them in P::prefetch_inputs(e), which the plain kernel issues as L2
// prefetches before it waits for the previous launch: a prefetch is a hint
// with no effect on what any load returns, so it may run before the inputs
// are final, and the team's first reads then come from L2.
template <class P, class = void>
struct has_prefetch : std::false_type {};
template <class P>
struct has_prefetch<P, std::void_t<decltype(&P::prefetch_inputs)>> : std::true_type {};

// Images, outputs and statuses of a well-formed descriptor of program P.
template <class P>
DSR_HD void program_extent(const dsr_region_desc &d, uint64_t *ib, uint64_t *ob, uint64_t *ns) {
  if constexpr (is_user<P>::value) {
    P::extent(d, ib, ob);
    *ns = d.teams;
  } else {
    extent(d, ib, ob, ns);
  }
}

// The descriptor is well formed for P and fits the buffers it indexes.
template <class P>
DSR_HD bool program_fits(const dsr_region_desc &d, uint64_t image_bytes, uint64_t out_bytes,
                         uint64_t n_status) {
  if (d.program != P::kProgram || shape_error(d) != 0) return false;
  uint64_t ib, ob, ns;
  program_extent<P>(d, &ib, &ob, &ns);
  if (ib && (d.image_offset > image_bytes || ib > image_bytes - d.image_offset)) return false;
  if (d.out_offset > out_bytes || ob > out_bytes - d.out_offset) return false;
  return static_cast<uint64_t>(d.status_index) + ns <= n_status;
}

// ---------------------------------------------------------------------------
// Plain kernel: one CTA per team (Sec. 4: a target region compiles to one
// kernel with a fixed number of teams and threads; team = threadblock).
// MAXT/MINB bound the registers so that teams of MAXT threads can reach
// MINB resident CTAs per SM.
// ---------------------------------------------------------------------------
template <class P, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
    plain_kernel(const __grid_constant__ dsr_region_desc d, const uint8_t *__restrict__ images,
                 uint8_t *__restrict__ out, dsr_team_status *__restrict__ st,
                 uint8_t *__restrict__ pool, uint64_t ovf_per_team, uint32_t slab_bytes,
                 uint64_t timeout_ns) {
  Env e;
  e.d = &d;
  e.images = images;
  e.out = out;
  e.team = blockIdx.x;
  if (threadIdx.x == 0) signal_dependents();
  if (threadIdx.x < team_workers()) {
    wait_prerequisites();
    worker_loop<P>(e);
    return;
  }
  Stack s;
  team_setup(s, slab_bytes,
             ovf_per_team ? pool + static_cast<uint64_t>(blockIdx.x) * ovf_per_team : nullptr,
             ovf_per_team, timeout_ns, true);
  if constexpr (has_prefetch<P>::value) {
    if (lane_id() == 0) P::prefetch_inputs(e);
  }
  wait_prerequisites();  // the set-up above touches shared memory only
  P::master(e, s);
  terminate_workers();
  team_report(e, s, st);
}

using PlainFn = void (*)(dsr_region_desc, const uint8_t *, uint8_t *, dsr_team_status *,
                         uint8_t *, uint64_t, uint32_t, uint64_t);

// Balanced residency of a plain launch. A launch of T teams on N SMs needs
// at most ceil(T / N) teams on any SM, but the block scheduler fills an SM
// up to the kernel's occupancy (with programmatic dependent launch, the SMs
// the previous grid frees first take the most), and the launch ends with
// its fullest SM. Dynamic shared memory asked for beyond what the program
// uses caps the CTAs an SM can hold, so the launch asks for the least that
// leaves room for ceil(T / N) CTAs and no more. Returns the dynamic shared
// memory to launch kernel k with: `base` (control block and slab) when the
// teams are no more than the SMs, when ceil(T / N) CTAs per SM is already
// the occupancy or beyond it, or when the occupancy calculator does not
// confirm exactly the cap at the padded size (which it then also allows in
// the kernel's attributes). Host code; results are kept per (kernel, block,
// base, T, device).
inline uint32_t balanced_smem(const void *k, uint32_t block, uint32_t base, uint32_t teams,
                              int device, uint32_t max_dyn) {
  struct Entry {
    const void *k;
    uint32_t block, base, teams;
    int device;
    uint32_t smem;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  {
    std::lock_guard<std::mutex> g(mu);
    for (const Entry &x : cache)
      if (x.k == k && x.block == block && x.base == base && x.teams == teams && x.device == device)
        return x.smem;
  }
  uint32_t smem = base;
  int sms = 0, per_sm_smem = 0, reserved = 0, occ = 0;
  cudaFuncAttributes fa{};
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess &&
      cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) ==
          cudaSuccess &&
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) ==
          cudaSuccess &&
      cudaFuncGetAttributes(&fa, k) == cudaSuccess && sms > 0 &&
      teams > static_cast<uint32_t>(sms) &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, static_cast<int>(block), base) ==
          cudaSuccess) {
    const uint32_t cap = (teams + sms - 1u) / static_cast<uint32_t>(sms);
    if (cap < static_cast<uint32_t>(occ)) {
      // (cap + 1) CTAs of this footprint exceed the SM's shared memory
      const int64_t want = static_cast<int64_t>(per_sm_smem) / (cap + 1) -
                           static_cast<int64_t>(fa.sharedSizeBytes) - reserved + 1;
      const uint32_t dyn = static_cast<uint32_t>((want + 15) & ~int64_t(15));
      int occ2 = 0;
      if (want > static_cast<int64_t>(base) && dyn <= max_dyn &&
          (static_cast<int>(dyn) <= fa.maxDynamicSharedSizeBytes ||
           cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(dyn)) == cudaSuccess) &&
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k, static_cast<int>(block), dyn) ==
              cudaSuccess &&
          occ2 == static_cast<int>(cap))
        smem = dyn;
    }
  }
  cudaGetLastError();  // a refused query leaves the launch at `base`
  std::lock_guard<std::mutex> g(mu);
  if (cache.size() >= 64) cache.erase(cache.begin());
  cache.push_back({k, block, base, teams, device, smem});
  return smem;
}

// The plain kernel instance for a CTA of `threads` threads. Programs whose
// launches fill the GPU with many teams (P::kDense) are held to 32
// registers, so 2048 threads per SM can be resident; those whose teams are
// few per SM anyway (kWideRegs) get up to 85; the others 64.
template <class P>
PlainFn pick_plain(uint32_t threads) {
  // resident CTAs of 256 threads the register budget is sized for
  constexpr int k = P::kDense ? 8 : wide_regs<P>::value ? 3 : 4;
  if (threads <= 128) return plain_kernel<P, 128, 2 * k>;
  if (threads <= 256) return plain_kernel<P, 256, k>;
  constexpr int k512 = k / 2 > 1 ? k / 2 : 1, k1024 = k / 4 > 1 ? k / 4 : 1;
  if (threads <= 512) return plain_kernel<P, 512, k512>;
  return plain_kernel<P, 1024, k1024>;
}

// ---------------------------------------------------------------------------
// Batched form: the workspace header and the persistent kernel
// ---------------------------------------------------------------------------
// The task list is dealt to kGroups parts round robin (part g holds
// positions g, g + kGroups, ...), each with its own cursor on its own
// 128-byte line, so the CTAs' grabs spread over kGroups addresses while
// every part still runs in longest-first order; a CTA starts on part
// (block mod kGroups) and moves on to the next part when its own is used up.
constexpr uint32_t kGroups = 32;
constexpr uint32_t kBuckets = 32;  // cost classes, log2 of a team's estimated cost

struct WsHeader {
  unsigned long long total;  // tasks counted by the scan
  unsigned int errors;       // tasks rejected on the device
  unsigned int abort;        // set by the host (dsr_batch_abort): take no more tasks
  unsigned int ran;          // tasks the CTAs ran (added up as they leave)
  unsigned int pad[27];
  unsigned long long bucket_fill[kBuckets];  // next free task slot of each cost class
  struct {
    unsigned long long next;  // tasks of this part handed out
    unsigned long long pad[15];
  } cursor[kGroups];
};
static_assert(sizeof(WsHeader) == 128 + 8 * kBuckets + 128 * kGroups, "workspace header");

// Dynamic shared memory of a persistent-kernel CTA with a slab of `slab`
// bytes: control block, slab, accumulator area.
constexpr uint32_t batch_smem(uint32_t slab) { return kCtrlBytes + slab + kAccBytes; }

// The persistent kernel's master warp pulls tasks in chunks of consecutive
// tasks (consecutive teams of one instance share its descriptor and images,
// which then hit in cache): chunks of 4 when every CTA has at least
// kLongBatch tasks to take, else 2. The tasks run longest first, so a CTA
// whose chunk holds several of the heaviest runs them in turn, and in a
// short batch those first chunks set the batch's end. Hetero instances on
// 128-thread CTAs (2,432 CTAs), chunks of 2 / 4: 10,000 instances (about 330
// tasks per CTA) 5.51 / 5.44 ms; 2,000 (66 per CTA) 1.69-1.74 / 2.28-2.74 ms;
// 500 0.73 / 1.25 ms. Chunks of 1 (5.65 ms), 8 (5.76-5.88) and 16 (6.7-7.0)
// were slower at 10,000.
constexpr uint32_t kLongBatch = 256;

struct Feeder {
  uint32_t g;        // current part
  uint32_t visited;  // parts found used up
  uint32_t grab;     // tasks per chunk (the same in every CTA of a launch)

  // Next chunk of tasks of the current part: positions [*start, *end) of
  // the part (task index = g + position * kGroups); *start == *end when no
  // task is left anywhere, or when the host has asked the batch to stop
  // (the flag is read with each grab, in the same round trip).
  __device__ __forceinline__ void next(WsHeader *hdr, uint32_t total, uint32_t *start,
                                       uint32_t *end) {
    while (visited < kGroups) {
      const uint32_t count = g < total ? (total - g + kGroups - 1) / kGroups : 0u;
      unsigned long long t = 0;
      uint32_t stop = 0;
      if (lane_id() == 0) {
        t = atomicAdd(&hdr->cursor[g].next, static_cast<unsigned long long>(grab));
        stop = *reinterpret_cast<volatile const unsigned int *>(&hdr->abort);
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      if (__shfl_sync(0xffffffffu, stop, 0)) {
        *start = *end = 0;
        visited = kGroups;
        return;
      }
      if (t < count) {
        *start = static_cast<uint32_t>(t);
        *end = min(*start + grab, count);
        return;
      }
      g = (g + 1) % kGroups;
      ++visited;
    }
    *start = *end = 0;
  }
  __device__ __forceinline__ uint32_t task_index(uint32_t pos) const { return g + pos * kGroups; }
};

// The persistent kernel. Each task runs as one team of its instance: the
// descriptor is copied into the control block and checked once per
// instance (a bad one gives its teams INVALID). The next chunk's grab and
// the next task's entry are issued before the current task runs, so their
// latency overlaps it.
template <class P, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) batch_kernel(const __grid_constant__ dsr_batch_plan a) {
  Env e;
  e.d = nullptr;
  e.images = static_cast<const uint8_t *>(a.images);
  e.out = static_cast<uint8_t *>(a.out);
  e.team = 0;
  if (threadIdx.x < team_workers()) {
    worker_loop<P, true>(e);
    return;
  }
  Ctrl *c = ctrl();
  Stack s;
  WsHeader *hdr = static_cast<WsHeader *>(a.hdr);
  const uint2 *tasks = static_cast<const uint2 *>(a.tasks);
  const dsr_region_desc *descs = static_cast<const dsr_region_desc *>(a.descs);
  dsr_team_status *status = static_cast<dsr_team_status *>(a.status);
  uint8_t *ovf = a.ovf_per_cta ? static_cast<uint8_t *>(a.pool) +
                                     static_cast<uint64_t>(blockIdx.x) * a.ovf_per_cta
                               : nullptr;
  const uint32_t total = static_cast<uint32_t>(min(static_cast<uint64_t>(hdr->total), a.capacity));
  const uint32_t lane = lane_id();
  Feeder feed{blockIdx.x % kGroups, 0,
              total >= static_cast<uint64_t>(kLongBatch) * gridDim.x ? 4u : 2u};
  uint32_t cur, end;
  feed.next(hdr, total, &cur, &end);
  bool have = cur < end;
  uint2 task = have ? tasks[feed.task_index(cur)] : make_uint2(0, 0);
  uint32_t cached = 0xffffffffu;  // instance whose descriptor is in the control block
  bool cached_ok = false;
  bool first = true;
  uint32_t ran = 0;
  while (have) {
    // the next task: its chunk grab (at a chunk boundary) and its entry
    uint32_t nxt = cur + 1, nend = end;
    if (nxt >= end) feed.next(hdr, total, &nxt, &nend);
    const bool nhave = nxt < nend;
    const uint2 ntask = nhave ? tasks[feed.task_index(nxt)] : make_uint2(0, 0);

    if (task.x != cached) {
      __syncwarp();
      if (lane < 4)
        reinterpret_cast<uint4 *>(&c->desc)[lane] =
            reinterpret_cast<const uint4 *>(descs + task.x)[lane];
      __syncwarp();
      cached = task.x;
      cached_ok = program_fits<P>(c->desc, a.image_bytes, a.out_bytes, a.n_status);
    }
    if (lane == 0) c->team = task.y;
    e.d = &c->desc;
    e.team = task.y;
    team_setup(s, a.slab_bytes, ovf, a.ovf_per_cta, a.timeout_ns, first);
    if (first) s.bits |= kAccArea;
    first = false;
    if (!cached_ok || task.y >= c->desc.teams) {
      if (lane == 0) {
        atomicAdd(&hdr->errors, 1u);
        const uint64_t si = static_cast<uint64_t>(c->desc.status_index) + task.y;
        if (si < a.n_status) {
          dsr_team_status r = {};
          r.status = DSR_ERR_INVALID;
          status[si] = r;
        }
      }
    } else {
      P::master(e, s);
      team_report(e, s, status);
    }
    ++ran;
    cur = nxt;
    end = nend;
    task = ntask;
    have = nhave;
  }
  if (lane == 0 && ran) atomicAdd(&hdr->ran, ran);
  terminate_workers();
}

using BatchFn = void (*)(dsr_batch_plan);

// Register budgets: CTAs of up to 512 threads are held to 32 registers, so
// that 2048 threads (many teams in flight, or wide teams with many workers)
// fit an SM; 1024-thread CTAs get up to 64.
template <class P>
BatchFn pick_batch(uint32_t threads) {
  if (threads <= 128) return batch_kernel<P, 128, 16>;
  if (threads <= 256) return batch_kernel<P, 256, 8>;
  if (threads <= 512) return batch_kernel<P, 512, 4>;
  return batch_kernel<P, 1024, 1>;
}

}  // namespace dsr
