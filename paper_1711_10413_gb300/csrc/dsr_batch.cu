// dsr_batch.cu -- batched launch form and its autotuner.
//
// Thousands of heterogeneous region instances (uneven team counts, thread
// counts and frame sizes) run in one persistent kernel: a fixed grid of
// CTAs, each with a fixed thread count and shared-memory slab, pulls tasks
// -- (instance, team) pairs -- from a global cursor and runs each as a
// virtual team with the instance's width (a region wider than the CTA's
// workers runs its threads round robin on them). Three kernels make a batch:
// a scan of the instances' team counts, the expansion of the task list, and
// the persistent kernel; with use_graph they are captured once per
// argument set into a CUDA graph that later calls replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "dsr.h"
#include "dsr_check.cuh"
#include "dsr_ctx.h"
#include "dsr_programs.cuh"

using namespace dsr;

namespace {

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
  unsigned int pad[29];
  unsigned long long bucket_fill[kBuckets];  // next free task slot of each cost class
  struct {
    unsigned long long next;  // tasks of this part handed out
    unsigned long long pad[15];
  } cursor[kGroups];
};
static_assert(sizeof(WsHeader) == 128 + 8 * kBuckets + 128 * kGroups, "workspace header");

constexpr uint64_t kWsHeader = sizeof(WsHeader);

uint64_t pad256(uint64_t n) { return (n + 255u) & ~static_cast<uint64_t>(255u); }

uint64_t ws_tasks_off(uint32_t) { return pad256(kWsHeader); }
uint64_t ws_bytes(uint32_t n, uint64_t tasks) { return ws_tasks_off(n) + pad256(8ull * tasks); }

struct BatchArgs {
  const dsr_region_desc *descs;
  const uint2 *tasks;  // (instance, team)
  WsHeader *hdr;
  const uint8_t *images;
  uint8_t *out;
  dsr_team_status *status;
  uint8_t *pool;
  uint64_t capacity;  // task slots in the workspace
  uint64_t image_bytes;
  uint64_t out_bytes;
  uint64_t n_status;
  uint64_t ovf_per_cta;
  uint64_t timeout_ns;
  uint32_t n;
  uint32_t slab_bytes;
};

// A team's estimated cost, in word-operations: its frames' words (filled,
// updated and hashed once or twice each), its region width (one output per
// thread) and a fixed share per level for the handoff and the master's code.
__device__ __forceinline__ uint32_t cost_class(const dsr_region_desc &d) {
  uint64_t c = 1024ull * (d.depth < DSR_MAX_DEPTH ? d.depth : DSR_MAX_DEPTH) + desc_width(d);
  for (uint32_t k = 0; k < DSR_MAX_DEPTH; ++k)
    if (k < d.depth) c += d.frame_bytes[k] / 2u;
  const uint32_t b = 63u - static_cast<uint32_t>(__clzll(c));
  return b < kBuckets ? b : kBuckets - 1;
}

// Team totals per cost class, and where each class starts in the task list:
// the most expensive class first, so the cursors hand out the longest
// teams first (longest-processing-time order) and the batch does not end on
// a long team (one CTA).
__global__ void __launch_bounds__(1024) batch_scan(const dsr_region_desc *__restrict__ descs,
                                                   uint32_t n, WsHeader *hdr) {
  __shared__ unsigned long long count[kBuckets];
  const uint32_t tid = threadIdx.x;
  if (tid < kBuckets) count[tid] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < n; i += blockDim.x)
    atomicAdd(&count[cost_class(descs[i])], static_cast<unsigned long long>(descs[i].teams));
  __syncthreads();
  if (tid == 0) {
    unsigned long long base = 0;
    for (int b = kBuckets - 1; b >= 0; --b) {
      hdr->bucket_fill[b] = base;
      base += count[b];
    }
    hdr->total = base;
    hdr->errors = 0;
  }
  if (tid < kGroups) hdr->cursor[tid].next = 0;
}

// Task list: each instance claims a contiguous run of slots in its cost
// class and writes its teams there (one warp per instance). The order of
// instances inside a class depends on timing; which teams run is the same.
__global__ void __launch_bounds__(256) batch_expand(const dsr_region_desc *__restrict__ descs,
                                                    uint32_t n, WsHeader *hdr, uint2 *tasks,
                                                    uint64_t capacity) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x / 32u);
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) / 32u; i < n; i += warps) {
    const uint32_t T = descs[i].teams;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&hdr->bucket_fill[cost_class(descs[i])], static_cast<unsigned long long>(T));
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t t = lane; t < T && base + t < capacity; t += 32u)
      tasks[base + t] = make_uint2(i, t);
  }
}

// The persistent kernel. Its master warp pulls tasks in chunks of kGrab
// consecutive tasks (consecutive teams of one instance share its descriptor
// and images, which then hit in cache) and runs each as one team of its
// instance: the descriptor is copied into the control block and checked
// once per instance. The next chunk's grab and the next task's entry are
// issued before the current task runs, so their latency overlaps it.
constexpr uint32_t kGrab = 2;

struct Feeder {
  uint32_t g;        // current part
  uint32_t visited;  // parts found used up

  // Next chunk of tasks of the current part: positions [*start, *end) of
  // the part (task index = g + position * kGroups); *start == *end when no
  // task is left anywhere.
  __device__ __forceinline__ void next(const BatchArgs &a, uint32_t total, uint32_t *start,
                                       uint32_t *end) {
    while (visited < kGroups) {
      const uint32_t count = g < total ? (total - g + kGroups - 1) / kGroups : 0u;
      unsigned long long t = 0;
      if (lane_id() == 0) t = atomicAdd(&a.hdr->cursor[g].next, static_cast<unsigned long long>(kGrab));
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t < count) {
        *start = static_cast<uint32_t>(t);
        *end = min(*start + kGrab, count);
        return;
      }
      g = (g + 1) % kGroups;
      ++visited;
    }
    *start = *end = 0;
  }
  __device__ __forceinline__ uint32_t task_index(uint32_t pos) const { return g + pos * kGroups; }
};

template <class P, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) batch_kernel(const __grid_constant__ BatchArgs a) {
  Env e;
  e.d = nullptr;
  e.images = a.images;
  e.out = a.out;
  e.team = 0;
  if (threadIdx.x < team_workers()) {
    worker_loop<P, true>(e);
    return;
  }
  Ctrl *c = ctrl();
  Stack s;
  uint8_t *ovf = a.ovf_per_cta ? a.pool + static_cast<uint64_t>(blockIdx.x) * a.ovf_per_cta : nullptr;
  const uint32_t total =
      static_cast<uint32_t>(min(static_cast<uint64_t>(a.hdr->total), a.capacity));
  const uint32_t lane = lane_id();
  Feeder feed{blockIdx.x % kGroups, 0};
  uint32_t cur, end;
  feed.next(a, total, &cur, &end);
  bool have = cur < end;
  uint2 task = have ? a.tasks[feed.task_index(cur)] : make_uint2(0, 0);
  uint32_t cached = 0xffffffffu;  // instance whose descriptor is in the control block
  bool cached_ok = false;
  bool first = true;
  while (have) {
    // the next task: its chunk grab (at a chunk boundary) and its entry
    uint32_t nxt = cur + 1, nend = end;
    if (nxt >= end) feed.next(a, total, &nxt, &nend);
    const bool nhave = nxt < nend;
    const uint2 ntask = nhave ? a.tasks[feed.task_index(nxt)] : make_uint2(0, 0);

    if (task.x != cached) {
      __syncwarp();
      if (lane < 4)
        reinterpret_cast<uint4 *>(&c->desc)[lane] =
            reinterpret_cast<const uint4 *>(a.descs + task.x)[lane];
      __syncwarp();
      const dsr_region_desc &d = c->desc;
      cached = task.x;
      cached_ok = d.program == P::kProgram && shape_error(d) == 0 &&
                  fits(d, a.image_bytes, a.out_bytes, a.n_status);
    }
    if (lane == 0) c->team = task.y;
    e.d = &c->desc;
    e.team = task.y;
    team_setup(s, a.slab_bytes, ovf, a.ovf_per_cta, a.timeout_ns, first);
    first = false;
    if (!cached_ok || task.y >= c->desc.teams) {
      if (lane == 0) {
        atomicAdd(&a.hdr->errors, 1u);
        const uint64_t si = static_cast<uint64_t>(c->desc.status_index) + task.y;
        if (si < a.n_status) {
          dsr_team_status r = {};
          r.status = DSR_ERR_INVALID;
          a.status[si] = r;
        }
      }
    } else {
      P::master(e, s);
      team_report(e, s, a.status);
    }
    cur = nxt;
    end = nend;
    task = ntask;
    have = nhave;
  }
  terminate_workers();
}

using BatchFn = void (*)(BatchArgs);

// Three register budgets: small CTAs held to 32 registers so that many of
// them (many tasks in flight) fit an SM; the others up to 64.
template <class P>
BatchFn pick_batch(uint32_t threads) {
  if (threads <= 128) return batch_kernel<P, 128, 16>;
  if (threads <= 256) return batch_kernel<P, 256, 4>;
  return batch_kernel<P, 1024, 1>;
}

BatchFn batch_kernel_for(uint32_t program, uint32_t threads) {
  switch (program) {
    case DSR_PROG_PAPER_SCALARS: return pick_batch<ProgPaperScalars>(threads);
    case DSR_PROG_PAPER_ARRAYS: return pick_batch<ProgPaperArrays>(threads);
    case DSR_PROG_SCALARS: return pick_batch<ProgScalars>(threads);
    case DSR_PROG_NESTED: return pick_batch<ProgNested>(threads);
    case DSR_PROG_SWEEP: return pick_batch<ProgSweep>(threads);
    case DSR_PROG_HETERO: return pick_batch<ProgHetero>(threads);
    default: return nullptr;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Context state of the batched form
// ---------------------------------------------------------------------------
struct GraphKey {
  const void *descs, *images, *out, *status, *ws;
  uint64_t n, tasks, image_bytes, out_bytes, n_status, ws_bytes;
  uint32_t program, threads, slab, grid;
  bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct dsr_batch_state {
  cudaStream_t capture = nullptr;
  struct Entry {
    GraphKey key;
    cudaGraphExec_t exec;
  };
  std::vector<Entry> graphs;
  bool attrs_set = false;
};

static void drop_graphs(dsr_batch_state *b) {
  for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

void dsr_ctx_release(dsr_ctx *ctx) {
  if (ctx->batch) {
    drop_graphs(ctx->batch);
    if (ctx->batch->capture) cudaStreamDestroy(ctx->batch->capture);
    delete ctx->batch;
    ctx->batch = nullptr;
  }
  dsr_serve_release(ctx);
}

int32_t dsr_ctx_stack_changed(dsr_ctx *ctx, uint32_t) {
  // graphs baked in the old overflow pool
  if (ctx->batch) drop_graphs(ctx->batch);
  return DSR_OK;
}

static dsr_batch_state *batch_state(dsr_ctx *ctx) {
  if (!ctx->batch) ctx->batch = new dsr_batch_state();
  return ctx->batch;
}

static int32_t set_batch_attrs(dsr_ctx *ctx) {
  dsr_batch_state *b = batch_state(ctx);
  if (b->attrs_set) return DSR_OK;
  for (uint32_t p = DSR_PROG_PAPER_SCALARS; p <= DSR_PROG_HETERO; ++p)
    for (uint32_t t : {128u, 256u, 1024u}) {
      const void *k = reinterpret_cast<const void *>(batch_kernel_for(p, t));
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           ctx->max_smem_optin);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "cudaFuncSetAttribute (batch)");
    }
  b->attrs_set = true;
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Host entry points
// ---------------------------------------------------------------------------
extern "C" uint64_t dsr_batch_workspace_bytes(uint32_t n, uint64_t total_teams) {
  return ws_bytes(n, total_teams);
}

extern "C" int32_t dsr_batch_count(const dsr_region_desc *descs_host, uint32_t n,
                                   uint64_t image_bytes, uint64_t out_bytes, uint64_t n_status,
                                   uint64_t *total_teams) {
  if (!descs_host || !total_teams) return dsr_fail(nullptr, DSR_ERR_INVALID, "null argument");
  uint64_t total = 0;
  for (uint32_t i = 0; i < n; ++i) {
    int32_t rc = dsr_validate_region(descs_host + i, image_bytes, out_bytes, n_status);
    if (rc != DSR_OK)
      return dsr_fail(nullptr, rc, "descriptor %u: %s", i, dsr_last_error_string(nullptr));
    total += descs_host[i].teams;
  }
  *total_teams = total;
  return DSR_OK;
}

namespace {

struct BatchCall {
  const dsr_region_desc *descs;
  uint32_t n;
  uint32_t program;
  uint64_t tasks;
  const void *images;
  uint64_t image_bytes;
  void *out;
  uint64_t out_bytes;
  dsr_team_status *status;
  uint64_t n_status;
  void *ws;
  uint64_t ws_bytes;
};

int32_t resolve_tuning(dsr_ctx *ctx, const BatchCall &c, const dsr_batch_tuning *t_in,
                       uint32_t *threads, uint32_t *slab, uint32_t *grid) {
  dsr_batch_tuning t = {256, 16384, 0, 0};
  if (t_in) t = *t_in;
  if (t.threads < 64 || t.threads > DSR_MAX_THREADS || t.threads % 32)
    return dsr_fail(ctx, DSR_ERR_INVALID, "batch threads must be a multiple of 32 in [64, 1024]");
  if (t.slab_bytes % 16 || kCtrlBytes + t.slab_bytes > static_cast<uint32_t>(ctx->max_smem_optin))
    return dsr_fail(ctx, DSR_ERR_INVALID, "batch slab must be a multiple of 16 fitting a CTA");
  BatchFn k = batch_kernel_for(c.program, t.threads);
  if (!k) return dsr_fail(ctx, DSR_ERR_INVALID, "unknown program %u", c.program);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, reinterpret_cast<const void *>(k), static_cast<int>(t.threads),
      kCtrlBytes + t.slab_bytes);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "occupancy query");
  if (occ < 1) return dsr_fail(ctx, DSR_ERR_INVALID, "batch CTA shape does not fit an SM");
  const uint32_t per_sm = t.ctas_per_sm ? std::min<uint32_t>(t.ctas_per_sm, occ) : occ;
  uint64_t g = static_cast<uint64_t>(ctx->sm_count) * per_sm;
  g = std::min<uint64_t>(g, std::max<uint64_t>(c.tasks, 1));
  if (ctx->ovf_per_team) g = std::min<uint64_t>(g, ctx->max_teams);
  *threads = t.threads;
  *slab = t.slab_bytes;
  *grid = static_cast<uint32_t>(std::max<uint64_t>(g, 1));
  return DSR_OK;
}

int32_t enqueue_batch(dsr_ctx *ctx, const BatchCall &c, uint32_t threads, uint32_t slab,
                      uint32_t grid, cudaStream_t s) {
  uint8_t *ws = static_cast<uint8_t *>(c.ws);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
  auto *tasks = reinterpret_cast<uint2 *>(ws + ws_tasks_off(c.n));
  batch_scan<<<1, 1024, 0, s>>>(c.descs, c.n, hdr);
  const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((c.n + 7) / 8, 4096));
  batch_expand<<<blocks, 256, 0, s>>>(c.descs, c.n, hdr, tasks, c.tasks);
  BatchArgs a;
  a.descs = c.descs;
  a.tasks = tasks;
  a.hdr = hdr;
  a.images = static_cast<const uint8_t *>(c.images);
  a.out = static_cast<uint8_t *>(c.out);
  a.status = c.status;
  a.pool = ctx->pool;
  a.capacity = c.tasks;
  a.image_bytes = c.image_bytes;
  a.out_bytes = c.out_bytes;
  a.n_status = c.n_status;
  a.ovf_per_cta = ctx->ovf_per_team;
  a.timeout_ns = ctx->timeout_ns;
  a.n = c.n;
  a.slab_bytes = slab;
  batch_kernel_for(c.program, threads)<<<grid, threads, kCtrlBytes + slab, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "batch launch");
  return DSR_OK;
}

int32_t check_batch(dsr_ctx *ctx, const BatchCall &c) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  if (!c.descs || c.n == 0 || !c.out || !c.status || !c.ws)
    return dsr_fail(ctx, DSR_ERR_INVALID, "null batch argument or empty batch");
  if ((reinterpret_cast<uintptr_t>(c.descs) | reinterpret_cast<uintptr_t>(c.ws)) & 15u)
    return dsr_fail(ctx, DSR_ERR_INVALID, "descriptors and workspace must be 16-byte aligned");
  if (c.tasks >= 0xffffffffull)
    return dsr_fail(ctx, DSR_ERR_INVALID, "a batch holds fewer than 2^32 - 1 teams");
  if (c.ws_bytes < ws_bytes(c.n, c.tasks))
    return dsr_fail(ctx, DSR_ERR_BUDGET, "workspace of %llu bytes, %llu needed",
                    (unsigned long long)c.ws_bytes, (unsigned long long)ws_bytes(c.n, c.tasks));
  return set_batch_attrs(ctx);
}

}  // namespace

extern "C" int32_t dsr_launch_batch(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                                    uint32_t program, uint64_t total_teams,
                                    const void *images_dev, uint64_t image_bytes, void *out_dev,
                                    uint64_t out_bytes, dsr_team_status *status_dev,
                                    uint64_t n_status, void *workspace_dev,
                                    uint64_t workspace_bytes, const dsr_batch_tuning *tuning,
                                    void *stream, int use_graph) {
  BatchCall c{descs_dev, n, program, total_teams, images_dev, image_bytes, out_dev,
              out_bytes, status_dev, n_status, workspace_dev, workspace_bytes};
  int32_t rc = check_batch(ctx, c);
  if (rc != DSR_OK) return rc;
  uint32_t threads, slab, grid;
  if ((rc = resolve_tuning(ctx, c, tuning, &threads, &slab, &grid)) != DSR_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!use_graph) return enqueue_batch(ctx, c, threads, slab, grid, s);

  dsr_batch_state *b = batch_state(ctx);
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.descs = descs_dev;
  key.images = images_dev;
  key.out = out_dev;
  key.status = status_dev;
  key.ws = workspace_dev;
  key.n = n;
  key.tasks = total_teams;
  key.image_bytes = image_bytes;
  key.out_bytes = out_bytes;
  key.n_status = n_status;
  key.ws_bytes = workspace_bytes;
  key.program = program;
  key.threads = threads;
  key.slab = slab;
  key.grid = grid;
  cudaGraphExec_t exec = nullptr;
  for (auto &g : b->graphs)
    if (g.key == key) exec = g.exec;
  cudaError_t e;
  if (!exec) {
    if (!b->capture && (e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking)) !=
                           cudaSuccess)
      return dsr_cuda_fail(ctx, e, "capture stream");
    if ((e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return dsr_cuda_fail(ctx, e, "begin capture");
    rc = enqueue_batch(ctx, c, threads, slab, grid, b->capture);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->capture, &graph);
    if (rc != DSR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "end capture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "graph instantiate");
    if (b->graphs.size() >= 8) {
      cudaGraphExecDestroy(b->graphs.front().exec);
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back({key, exec});
  }
  if ((e = cudaGraphLaunch(exec, s)) != cudaSuccess) return dsr_cuda_fail(ctx, e, "graph launch");
  return DSR_OK;
}

extern "C" int32_t dsr_batch_errors(dsr_ctx *ctx, const void *workspace_dev, uint32_t *errors,
                                    uint64_t *tasks_counted, void *stream) {
  if (!ctx || !workspace_dev || !errors) return dsr_fail(ctx, DSR_ERR_INVALID, "null argument");
  WsHeader h;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h, workspace_dev, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "workspace read");
  *errors = h.errors;
  if (tasks_counted) *tasks_counted = h.total;
  return DSR_OK;
}

// Autotuner: time every candidate CTA shape x slab size on the real batch
// (outputs are the same for every candidate) and keep the fastest.
extern "C" int32_t dsr_autotune(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                                uint32_t program, uint64_t total_teams, const void *images_dev,
                                uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                                dsr_team_status *status_dev, uint64_t n_status,
                                void *workspace_dev, uint64_t workspace_bytes, void *stream,
                                dsr_batch_tuning *best, float *best_ms) {
  if (!best) return dsr_fail(ctx, DSR_ERR_INVALID, "null output");
  BatchCall c{descs_dev, n, program, total_teams, images_dev, image_bytes, out_dev,
              out_bytes, status_dev, n_status, workspace_dev, workspace_bytes};
  int32_t rc = check_batch(ctx, c);
  if (rc != DSR_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t a, z;
  cudaEventCreate(&a);
  cudaEventCreate(&z);
  float best_t = 1e30f;
  dsr_batch_tuning best_c = {256, 16384, 0, 0};
  const uint32_t kThreads[] = {64, 96, 128, 192, 256, 512};
  const uint32_t kSlabs[] = {2048, 4096, 8192, 16384, 32768};
  for (uint32_t th : kThreads)
    for (uint32_t sl : kSlabs) {
      dsr_batch_tuning t = {th, sl, 0, 0};
      uint32_t threads, slab, grid;
      if (resolve_tuning(ctx, c, &t, &threads, &slab, &grid) != DSR_OK) continue;
      if (enqueue_batch(ctx, c, threads, slab, grid, s) != DSR_OK) continue;  // warm
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(a, s);
        enqueue_batch(ctx, c, threads, slab, grid, s);
        cudaEventRecord(z, s);
        cudaEventSynchronize(z);
        float m = 0;
        cudaEventElapsedTime(&m, a, z);
        ms = std::min(ms, m);
      }
      if (ms < best_t) {
        best_t = ms;
        best_c = t;
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "autotune");
  if (best_t >= 1e29f) return dsr_fail(ctx, DSR_ERR_INVALID, "no batch shape fits this device");
  *best = best_c;
  if (best_ms) *best_ms = best_t;
  return DSR_OK;
}

// Per-region launches of host descriptors: the baseline the batched form is
// measured against (one kernel launch per region instance).
extern "C" int32_t dsr_launch_regions(dsr_ctx *ctx, const dsr_region_desc *descs_host, uint32_t n,
                                      const void *images_dev, uint64_t image_bytes,
                                      void *out_dev, uint64_t out_bytes,
                                      dsr_team_status *status_dev, uint64_t n_status,
                                      void *stream) {
  if (!descs_host) return dsr_fail(ctx, DSR_ERR_INVALID, "null descriptors");
  for (uint32_t i = 0; i < n; ++i) {
    int32_t rc = dsr_launch_region(ctx, descs_host + i, images_dev, image_bytes, out_dev,
                                   out_bytes, status_dev, n_status, stream);
    if (rc != DSR_OK) return rc;
  }
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Batched launch without allocation
//
// For callers that cannot allocate device memory -- code that must not call
// cudaMalloc/cudaFree (they can synchronise the device), or a host whose
// device memory is owned by another allocator -- the batch workspace can
// live in this fixed file-scope array instead of a caller buffer. Every GPU
// that loads this library keeps the array for the life of the process.
// ---------------------------------------------------------------------------
static constexpr uint64_t kStaticWsBytes = 8ull << 20;  // 8 MiB
static __device__ __align__(256) uint8_t g_static_ws[kStaticWsBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices];      // device address of g_static_ws, per device
bool g_static_attrs[kMaxDevices];     // batch kernels' shared-memory limit set

// Once per device, with that device current: the array's device address
// (the host-side symbol is only a stand-in for it) and the batch kernels'
// dynamic shared-memory limit.
int32_t static_setup(dsr_ctx *ctx, void **ws) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return dsr_fail(ctx, DSR_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[ctx->device] || !g_static_attrs[ctx->device]) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "cudaGetDevice");
    if (cur != ctx->device && (e = cudaSetDevice(ctx->device)) != cudaSuccess)
      return dsr_cuda_fail(ctx, e, "cudaSetDevice");
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e == cudaSuccess)
      for (uint32_t prog = DSR_PROG_PAPER_SCALARS; prog <= DSR_PROG_HETERO && e == cudaSuccess; ++prog)
        for (uint32_t t : {128u, 256u, 1024u}) {
          const void *k = reinterpret_cast<const void *>(batch_kernel_for(prog, t));
          e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   ctx->max_smem_optin);
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
          if (e != cudaSuccess) break;
        }
    if (cur != ctx->device) cudaSetDevice(cur);
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "static workspace set-up");
    g_static_ptr[ctx->device] = p;
    g_static_attrs[ctx->device] = true;
  }
  *ws = g_static_ptr[ctx->device];
  return DSR_OK;
}
}  // namespace

extern "C" uint64_t dsr_batch_static_capacity(void) { return kStaticWsBytes; }

extern "C" int32_t dsr_launch_batch_static(dsr_ctx *ctx, const dsr_region_desc *descs_dev,
                                           uint32_t n, uint32_t program, uint64_t total_teams,
                                           const void *images_dev, uint64_t image_bytes,
                                           void *out_dev, uint64_t out_bytes,
                                           dsr_team_status *status_dev, uint64_t n_status,
                                           const dsr_batch_tuning *tuning, void *stream) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  if (!descs_dev || n == 0 || !out_dev || !status_dev)
    return dsr_fail(ctx, DSR_ERR_INVALID, "null batch argument or empty batch");
  if (reinterpret_cast<uintptr_t>(descs_dev) & 15u)
    return dsr_fail(ctx, DSR_ERR_INVALID, "descriptors must be 16-byte aligned");
  if (total_teams >= 0xffffffffull || ws_bytes(n, total_teams) > kStaticWsBytes)
    return dsr_fail(ctx, DSR_ERR_BUDGET,
                    "a batch of %llu teams needs %llu workspace bytes; the static workspace "
                    "holds %llu (use dsr_launch_batch with a caller buffer)",
                    (unsigned long long)total_teams,
                    (unsigned long long)ws_bytes(n, total_teams),
                    (unsigned long long)kStaticWsBytes);
  void *ws = nullptr;
  int32_t rc = static_setup(ctx, &ws);
  if (rc != DSR_OK) return rc;
  BatchCall c{descs_dev, n, program, total_teams, images_dev, image_bytes, out_dev,
              out_bytes, status_dev, n_status, ws, kStaticWsBytes};
  uint32_t threads, slab, grid;
  if ((rc = resolve_tuning(ctx, c, tuning, &threads, &slab, &grid)) != DSR_OK) return rc;
  return enqueue_batch(ctx, c, threads, slab, grid, static_cast<cudaStream_t>(stream));
}
