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
// argument set into a CUDA graph that later calls replay. The persistent
// kernel itself (batch_kernel in dsr_kernels.cuh) is a template over the
// program, shared with programs written against dsr_device.cuh; this file
// launches the built-in programs' instances and prepares every batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "dsr.h"
#include "dsr_check.cuh"
#include "dsr_ctx.h"
#include "dsr_kernels.cuh"
#include "dsr_programs.cuh"

using namespace dsr;

namespace {

constexpr uint64_t kWsHeader = sizeof(WsHeader);

uint64_t pad256(uint64_t n) { return (n + 255u) & ~static_cast<uint64_t>(255u); }

uint64_t ws_tasks_off(uint32_t) { return pad256(kWsHeader); }
uint64_t ws_bytes(uint32_t n, uint64_t tasks) { return ws_tasks_off(n) + pad256(8ull * tasks); }

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
    hdr->abort = 0;
    hdr->ran = 0;
  }
  if (tid < kGroups) hdr->cursor[tid].next = 0;
}

// Task list: each instance claims a contiguous run of slots in its cost
// class and writes its teams there (one warp per instance). The order of
// instances inside a class depends on timing; which teams run is the same.
// A team with no slot (the caller's total_teams fell short of the
// instances' sum) never runs: its status says INVALID, where addressable,
// and it counts as a device-side error.
__global__ void __launch_bounds__(256) batch_expand(const dsr_region_desc *__restrict__ descs,
                                                    uint32_t n, WsHeader *hdr, uint2 *tasks,
                                                    uint64_t capacity, dsr_team_status *status,
                                                    uint64_t n_status) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x / 32u);
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) / 32u; i < n; i += warps) {
    const uint32_t T = descs[i].teams;
    unsigned long long base = 0;
    if (lane == 0)
      base = atomicAdd(&hdr->bucket_fill[cost_class(descs[i])], static_cast<unsigned long long>(T));
    base = __shfl_sync(0xffffffffu, base, 0);
    const uint64_t room = base < capacity ? capacity - static_cast<uint64_t>(base) : 0u;
    const uint64_t placed = T < room ? static_cast<uint64_t>(T) : room;
    for (uint32_t t = lane; t < placed; t += 32u) tasks[base + t] = make_uint2(i, t);
    if (placed < T) {
      if (lane == 0) atomicAdd(&hdr->errors, static_cast<unsigned int>(T - placed));
      const uint64_t si = descs[i].status_index;
      const uint64_t addressable = si < n_status ? n_status - si : 0u;
      const uint64_t stop = T < addressable ? static_cast<uint64_t>(T) : addressable;
      dsr_team_status r = {};
      r.status = DSR_ERR_INVALID;
      for (uint64_t t = placed + lane; t < stop; t += 32u) status[si + t] = r;
    }
  }
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
  uint32_t program, threads, slab, grid;  // grid: resident CTAs per SM
  bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};

struct dsr_batch_state {
  cudaStream_t capture = nullptr;
  cudaStream_t abort_stream = nullptr;  // carries abort flags while a batch holds the SMs
  unsigned int *abort_one = nullptr;    // pinned host word holding 1
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
    if (ctx->batch->abort_stream) cudaStreamDestroy(ctx->batch->abort_stream);
    if (ctx->batch->abort_one) cudaFreeHost(ctx->batch->abort_one);
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
    for (uint32_t t : {128u, 256u, 512u, 1024u}) {
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

// The CTA shape of a tuning (NULL: 256 threads, 16 KiB), checked.
int32_t check_tuning(dsr_ctx *ctx, const dsr_batch_tuning *t_in, dsr_batch_tuning *t) {
  *t = {256, 16384, 0, 0};
  if (t_in) *t = *t_in;
  if (t->threads < 64 || t->threads > DSR_MAX_THREADS || t->threads % 32)
    return dsr_fail(ctx, DSR_ERR_INVALID, "batch threads must be a multiple of 32 in [64, 1024]");
  if (t->slab_bytes % 16 || batch_smem(t->slab_bytes) > static_cast<uint32_t>(ctx->max_smem_optin))
    return dsr_fail(ctx, DSR_ERR_INVALID, "batch slab must be a multiple of 16 fitting a CTA");
  return DSR_OK;
}

// Resident CTAs per SM of a built-in program's persistent kernel in the
// tuning's shape (capped by the tuning's ctas_per_sm).
int32_t builtin_per_sm(dsr_ctx *ctx, uint32_t program, const dsr_batch_tuning &t,
                       uint32_t *per_sm) {
  BatchFn k = batch_kernel_for(program, t.threads);
  if (!k) return dsr_fail(ctx, DSR_ERR_INVALID, "unknown program %u", program);
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, reinterpret_cast<const void *>(k), static_cast<int>(t.threads),
      batch_smem(t.slab_bytes));
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "occupancy query");
  *per_sm = t.ctas_per_sm ? std::min<uint32_t>(t.ctas_per_sm, occ) : static_cast<uint32_t>(occ);
  return DSR_OK;
}

// Checks a batch, enqueues its scan and task-list expansion on s, and fills
// the persistent kernel's plan (grid: per_sm CTAs on every SM, at most one
// per task and one per overflow slab of the pool).
int32_t prepare(dsr_ctx *ctx, const BatchCall &c, uint32_t threads, uint32_t slab,
                uint32_t per_sm, cudaStream_t s, dsr_batch_plan *plan) {
  if (per_sm < 1) return dsr_fail(ctx, DSR_ERR_INVALID, "batch CTA shape does not fit an SM");
  uint64_t g = static_cast<uint64_t>(ctx->sm_count) * per_sm;
  g = std::min<uint64_t>(g, std::max<uint64_t>(c.tasks, 1));
  if (ctx->ovf_per_team) g = std::min<uint64_t>(g, ctx->max_teams);
  uint8_t *ws = static_cast<uint8_t *>(c.ws);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
  auto *tasks = reinterpret_cast<uint2 *>(ws + ws_tasks_off(c.n));
  batch_scan<<<1, 1024, 0, s>>>(c.descs, c.n, hdr);
  const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((c.n + 7) / 8, 4096));
  batch_expand<<<blocks, 256, 0, s>>>(c.descs, c.n, hdr, tasks, c.tasks, c.status, c.n_status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "batch scan launch");
  dsr_batch_plan &a = *plan;
  a.descs = c.descs;
  a.tasks = tasks;
  a.hdr = hdr;
  a.images = c.images;
  a.out = c.out;
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
  a.grid = static_cast<uint32_t>(std::max<uint64_t>(g, 1));
  a.threads = threads;
  return DSR_OK;
}

// A whole batch of a built-in program: prepare, then the persistent kernel.
int32_t enqueue_batch(dsr_ctx *ctx, const BatchCall &c, const dsr_batch_tuning &t,
                      uint32_t per_sm, cudaStream_t s) {
  dsr_batch_plan a;
  int32_t rc = prepare(ctx, c, t.threads, t.slab_bytes, per_sm, s, &a);
  if (rc != DSR_OK) return rc;
  batch_kernel_for(c.program, a.threads)<<<a.grid, a.threads, batch_smem(a.slab_bytes), s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "batch launch");
  return DSR_OK;
}

// Arguments every batched entry point checks, the workspace aside.
int32_t check_batch_args(dsr_ctx *ctx, const BatchCall &c) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  int32_t rc = dsr_check_device(ctx);
  if (rc != DSR_OK) return rc;
  if (!c.descs || c.n == 0 || !c.out || !c.status)
    return dsr_fail(ctx, DSR_ERR_INVALID, "null batch argument or empty batch");
  if (reinterpret_cast<uintptr_t>(c.descs) & 15u)
    return dsr_fail(ctx, DSR_ERR_INVALID, "descriptors must be 16-byte aligned");
  if (c.tasks >= 0xffffffffull)
    return dsr_fail(ctx, DSR_ERR_INVALID, "a batch holds fewer than 2^32 - 1 teams");
  return DSR_OK;
}

int32_t check_batch(dsr_ctx *ctx, const BatchCall &c) {
  int32_t rc = check_batch_args(ctx, c);
  if (rc != DSR_OK) return rc;
  if (!c.ws) return dsr_fail(ctx, DSR_ERR_INVALID, "null workspace");
  if (reinterpret_cast<uintptr_t>(c.ws) & 15u)
    return dsr_fail(ctx, DSR_ERR_INVALID, "workspace must be 16-byte aligned");
  if (c.ws_bytes < ws_bytes(c.n, c.tasks))
    return dsr_fail(ctx, DSR_ERR_BUDGET, "workspace of %llu bytes, %llu needed",
                    (unsigned long long)c.ws_bytes, (unsigned long long)ws_bytes(c.n, c.tasks));
  return DSR_OK;
}

// Check, tuning and resident CTAs of a built-in program's batch.
int32_t builtin_setup(dsr_ctx *ctx, const BatchCall &c, const dsr_batch_tuning *t_in,
                      dsr_batch_tuning *t, uint32_t *per_sm) {
  if (c.program >= DSR_PROG_USER)
    return dsr_fail(ctx, DSR_ERR_INVALID,
                    "program %u is user-written: launch it with dsr_launch_user_batch",
                    c.program);
  int32_t rc = check_tuning(ctx, t_in, t);
  if (rc == DSR_OK) rc = set_batch_attrs(ctx);
  if (rc == DSR_OK) rc = builtin_per_sm(ctx, c.program, *t, per_sm);
  return rc;
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
  dsr_batch_tuning t;
  uint32_t per_sm = 0;
  if ((rc = builtin_setup(ctx, c, tuning, &t, &per_sm)) != DSR_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!use_graph) return enqueue_batch(ctx, c, t, per_sm, s);

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
  key.threads = t.threads;
  key.slab = t.slab_bytes;
  key.grid = per_sm;
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
    rc = enqueue_batch(ctx, c, t, per_sm, b->capture);
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

// Stop a running batch: its CTAs take no task after their next grab. The
// flag goes in by a host-to-device copy on a stream of its own (a copy
// engine writes it while the persistent kernel holds every SM); the call
// does not wait for it.
static void *static_ws_of(dsr_ctx *ctx);

extern "C" int32_t dsr_batch_abort(dsr_ctx *ctx, void *workspace_dev) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  int32_t rc = dsr_check_device(ctx);
  if (rc != DSR_OK) return rc;
  void *ws = workspace_dev ? workspace_dev : static_ws_of(ctx);
  if (!ws) return dsr_fail(ctx, DSR_ERR_INVALID, "no workspace (no static batch has run)");
  dsr_batch_state *b = batch_state(ctx);
  cudaError_t e = cudaSuccess;
  if (!b->abort_stream) e = cudaStreamCreateWithFlags(&b->abort_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !b->abort_one) {
    e = cudaHostAlloc(&b->abort_one, sizeof(unsigned int), cudaHostAllocDefault);
    if (e == cudaSuccess) *b->abort_one = 1u;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&static_cast<WsHeader *>(ws)->abort, b->abort_one, sizeof(unsigned int),
                        cudaMemcpyHostToDevice, b->abort_stream);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "batch abort");
  return DSR_OK;
}

extern "C" int32_t dsr_batch_progress(dsr_ctx *ctx, const void *workspace_dev,
                                      uint64_t *tasks_taken, uint64_t *tasks_counted,
                                      void *stream) {
  if (!ctx || !tasks_taken) return dsr_fail(ctx, DSR_ERR_INVALID, "null argument");
  int32_t rc = dsr_check_device(ctx);
  if (rc != DSR_OK) return rc;
  const void *ws = workspace_dev ? workspace_dev : static_ws_of(ctx);
  if (!ws) return dsr_fail(ctx, DSR_ERR_INVALID, "no workspace (no static batch has run)");
  WsHeader h;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "workspace read");
  *tasks_taken = h.ran;
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
      const dsr_batch_tuning cand = {th, sl, 0, 0};
      dsr_batch_tuning t;
      uint32_t per_sm = 0;
      if (builtin_setup(ctx, c, &cand, &t, &per_sm) != DSR_OK) continue;
      if (enqueue_batch(ctx, c, t, per_sm, s) != DSR_OK) continue;  // warm
      float ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(a, s);
        enqueue_batch(ctx, c, t, per_sm, s);
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
void *g_static_ptr[kMaxDevices];  // device address of g_static_ws, per device

// Once per device, with that device current (every entry point requires the
// ctx's device to be current): the array's device address, for the host-side
// symbol is only a stand-in for it. The batch kernels' shared-memory limit
// is set per ctx, as for every batched launch.
int32_t static_setup(dsr_ctx *ctx, void **ws) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return dsr_fail(ctx, DSR_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[ctx->device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "static workspace address");
    g_static_ptr[ctx->device] = p;
  }
  *ws = g_static_ptr[ctx->device];
  return DSR_OK;
}
}  // namespace

extern "C" uint64_t dsr_batch_static_capacity(void) { return kStaticWsBytes; }

static void *static_ws_of(dsr_ctx *ctx) {
  std::lock_guard<std::mutex> g(g_static_mu);
  return ctx->device >= 0 && ctx->device < kMaxDevices ? g_static_ptr[ctx->device] : nullptr;
}

extern "C" int32_t dsr_launch_batch_static(dsr_ctx *ctx, const dsr_region_desc *descs_dev,
                                           uint32_t n, uint32_t program, uint64_t total_teams,
                                           const void *images_dev, uint64_t image_bytes,
                                           void *out_dev, uint64_t out_bytes,
                                           dsr_team_status *status_dev, uint64_t n_status,
                                           const dsr_batch_tuning *tuning, void *stream) {
  BatchCall c{descs_dev, n, program, total_teams, images_dev, image_bytes, out_dev,
              out_bytes, status_dev, n_status, nullptr, kStaticWsBytes};
  int32_t rc = check_batch_args(ctx, c);
  if (rc != DSR_OK) return rc;
  if (ws_bytes(n, total_teams) > kStaticWsBytes)
    return dsr_fail(ctx, DSR_ERR_BUDGET,
                    "a batch of %llu teams needs %llu workspace bytes; the static workspace "
                    "holds %llu (use dsr_launch_batch with a caller buffer)",
                    (unsigned long long)total_teams,
                    (unsigned long long)ws_bytes(n, total_teams),
                    (unsigned long long)kStaticWsBytes);
  if ((rc = static_setup(ctx, &c.ws)) != DSR_OK) return rc;
  dsr_batch_tuning t;
  uint32_t per_sm = 0;
  if ((rc = builtin_setup(ctx, c, tuning, &t, &per_sm)) != DSR_OK) return rc;
  return enqueue_batch(ctx, c, t, per_sm, static_cast<cudaStream_t>(stream));
}

extern "C" int32_t dsr_batch_static_errors(dsr_ctx *ctx, uint32_t *errors,
                                           uint64_t *tasks_counted, void *stream) {
  if (!ctx || !errors) return dsr_fail(ctx, DSR_ERR_INVALID, "null argument");
  int32_t rc = dsr_check_device(ctx);
  if (rc != DSR_OK) return rc;
  void *ws = nullptr;
  {
    std::lock_guard<std::mutex> g(g_static_mu);
    if (ctx->device >= 0 && ctx->device < kMaxDevices) ws = g_static_ptr[ctx->device];
  }
  if (!ws) return dsr_fail(ctx, DSR_ERR_INVALID, "no static batch has run on this device");
  return dsr_batch_errors(ctx, ws, errors, tasks_counted, stream);
}

// ---------------------------------------------------------------------------
// Batches of user-written programs (dsr_device.cuh): the library checks the
// batch, enqueues its scan and task list, and returns the plan the user's
// translation unit launches its own instance of the persistent kernel with.
// ---------------------------------------------------------------------------
extern "C" int32_t dsr_batch_prepare(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                                     uint32_t program, uint64_t total_teams,
                                     const void *images_dev, uint64_t image_bytes, void *out_dev,
                                     uint64_t out_bytes, dsr_team_status *status_dev,
                                     uint64_t n_status, void *workspace_dev,
                                     uint64_t workspace_bytes, uint32_t threads,
                                     uint32_t slab_bytes, uint32_t ctas_per_sm, void *stream,
                                     dsr_batch_plan *plan) {
  if (!plan) return dsr_fail(ctx, DSR_ERR_INVALID, "null plan");
  BatchCall c{descs_dev, n, program, total_teams, images_dev, image_bytes, out_dev,
              out_bytes, status_dev, n_status, workspace_dev, workspace_bytes};
  int32_t rc = check_batch(ctx, c);
  if (rc != DSR_OK) return rc;
  const dsr_batch_tuning in = {threads, slab_bytes, 0, 0};
  dsr_batch_tuning t;
  if ((rc = check_tuning(ctx, &in, &t)) != DSR_OK) return rc;
  return prepare(ctx, c, t.threads, t.slab_bytes, ctas_per_sm, static_cast<cudaStream_t>(stream),
                 plan);
}
