// dsr_serve.cu -- served launch form: a device-resident request loop.
//
// A persistent server kernel keeps every CTA's team stack live on the GPU
// and runs region instances as the host submits them, without a kernel
// launch per request: continuous batching. Requests that arrive while
// others run are picked up team by team as CTAs free up, so different
// requests' teams share the GPU at the same time.
//
// Host <-> device protocol, in pinned host memory mapped into the device:
//  * submit ring: `capacity` descriptor slots and a tail counter. The host
//    writes request s into slot s % capacity and then stores tail = s + 1
//    with release order; the device reads the tail with a system-scope
//    acquire load before it reads the slot.
//  * completion ring: records {s + 1, status} the device writes (payload
//    first, then the marker with a system-scope release store) at
//    positions it takes from a device counter; the host consumes them in
//    position order and clears each.
//  * stop flag: set by the host; the server drains what was submitted and
//    exits.
// Device workspace (caller-owned): the head of the request stream and, per
// slot, a claim word (request sequence << 32 | next team) and counters of
// finished teams and the worst team status. A CTA claims a run of teams with
// a 64-bit compare-and-swap on the claim word, which succeeds only while
// the sequence half still names the request it read, so a slot reused for a
// later request is never mistaken for an earlier one.
// One CTA, the doorbell, reads host memory: it copies every new request's
// descriptor into a device-memory ring and then the tail and the stop flag
// into device memory, where the other CTAs poll with backoff; the other CTAs
// never read host memory (a few do, rarely, when idle, so the server does
// not depend on the doorbell being resident). CTAs claim teams from a window
// of the oldest requests in flight, starting at different requests, so the
// claims do not all contend on one word.
// Every device-side wait is bounded: a CTA that finds no work for
// idle_timeout_ns leaves (the host restarts the server on the next submit
// or poll).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dsr.h"
#include "dsr_check.cuh"
#include "dsr_ctx.h"
#include "dsr_kernels.cuh"
#include "dsr_programs.cuh"
#include "dsr_serve_kernel.cuh"

using namespace dsr;

namespace {

ServeFn serve_kernel_for(uint32_t program, uint32_t threads) {
  switch (program) {
    case DSR_PROG_SCALARS: return pick_serve<ProgScalars>(threads);
    case DSR_PROG_NESTED: return pick_serve<ProgNested>(threads);
    case DSR_PROG_HETERO: return pick_serve<ProgHetero>(threads);
    default: return nullptr;
  }
}

uint64_t serve_ws_bytes(uint32_t capacity) {
  return sizeof(ServeWs) + (sizeof(SlotState) + sizeof(dsr_region_desc)) *
                               static_cast<uint64_t>(capacity);
}

__global__ void serve_init(ServeWs *ws, SlotState *slots, uint32_t capacity) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    ws->head = 0;
    ws->comp_tail = 0;
    ws->tail = 0;
    ws->stop = 0;
    ws->idle_exits = 0;
    ws->errors = 0;
  }
  if (i < capacity) {
    slots[i].claim = static_cast<unsigned long long>(i) << 32;
    slots[i].teams = 0;
    slots[i].done = 0;
    slots[i].status = 0;
  }
}

// Before a server starts again (after a stop or an idle exit): clear the
// stop copy; the head, tail copy and completion counters continue.
__global__ void serve_reopen(ServeWs *ws) {
  ws->stop = 0;
  ws->idle_exits = 0;
}

}  // namespace

struct dsr_serve_state {
  dsr_serve_cfg cfg{};
  bool is_user = false;       // a user-written program's server (hooks below)
  dsr_serve_program user{};
  uint32_t grid = 0;
  cudaStream_t stream = nullptr;
  bool running = false;
  bool launched = false;
  // pinned, mapped host memory
  dsr_region_desc *ring = nullptr;
  HostShared *hs = nullptr;
  CompRec *comp = nullptr;
  dsr_region_desc *ring_dev = nullptr;
  HostShared *hs_dev = nullptr;
  CompRec *comp_dev = nullptr;
  // device workspace (caller-owned)
  ServeWs *ws = nullptr;
  SlotState *slots = nullptr;
  dsr_region_desc *dring = nullptr;
  // host bookkeeping, per ring slot (ticket t uses slot t % capacity): no
  // map on the per-request path
  uint64_t next_seq = 0;       // next ticket
  uint64_t comp_pos = 0;       // next completion record to read
  uint64_t completed = 0;      // requests completed
  std::vector<uint8_t> slot_busy;        // slot holds an unfinished request
  std::vector<uint64_t> slot_reserved;   // its overflow bytes reserved
  std::vector<uint64_t> slot_done;       // ticket + 1 of a completion not yet reported, or 0
  std::vector<int32_t> slot_status;      // ... and its status
  std::unordered_map<uint64_t, int32_t> unreported;  // completions whose slot was reused first
  std::vector<uint64_t> just_done;       // tickets completed since the bench last looked
  bool collect_done = false;             // a bench run is collecting them
  uint64_t reserved_bytes = 0;
  uint64_t pool_budget = 0;
  uint64_t next_alive_check = 0;  // host time of the next server-exit check
};

void dsr_serve_release(dsr_ctx *ctx) {
  dsr_serve_state *sv = ctx->serve;
  if (!sv) return;
  if (sv->running) dsr_serve_stop(ctx);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  if (sv->ring) cudaFreeHost(sv->ring);
  if (sv->hs) cudaFreeHost(sv->hs);
  if (sv->comp) cudaFreeHost(sv->comp);
  delete sv;
  ctx->serve = nullptr;
}

namespace {

inline uint64_t now_ns() {
  return static_cast<uint64_t>(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                   std::chrono::steady_clock::now().time_since_epoch())
                                   .count());
}

// Has the server kernel left (idle timeout)? Asked of the driver at most
// once per millisecond: the query costs microseconds.
bool server_exited(dsr_serve_state *sv) {
  if (!sv->running) return true;
  const uint64_t t = now_ns();
  if (t < sv->next_alive_check) return false;
  sv->next_alive_check = t + 1000000;
  return cudaStreamQuery(sv->stream) == cudaSuccess;
}

int32_t launch_server(dsr_ctx *ctx, dsr_serve_state *sv) {
  if (sv->launched) serve_reopen<<<1, 1, 0, sv->stream>>>(sv->ws);
  sv->launched = true;
  ServeArgs a;
  a.ring = sv->ring_dev;
  a.dring = sv->dring;
  a.hs = sv->hs_dev;
  a.comp = sv->comp_dev;
  a.ws = sv->ws;
  a.slots = sv->slots;
  a.images = static_cast<const uint8_t *>(sv->cfg.images_dev);
  a.out = static_cast<uint8_t *>(sv->cfg.out_dev);
  a.status = sv->cfg.status_dev;
  a.pool = ctx->pool;
  a.image_bytes = sv->cfg.image_bytes;
  a.out_bytes = sv->cfg.out_bytes;
  a.n_status = sv->cfg.n_status;
  a.ovf_per_cta = ctx->ovf_per_team;
  a.timeout_ns = ctx->timeout_ns;
  a.idle_timeout_ns = sv->cfg.idle_timeout_ns ? sv->cfg.idle_timeout_ns : 2000000000ull;
  a.capacity = sv->cfg.capacity;
  a.slab_bytes = sv->cfg.slab_bytes;
  if (sv->is_user) {
    // the program's kernel lives in the user's translation unit
    if (sv->user.launch(&a, sv->grid, sv->cfg.threads, batch_smem(sv->cfg.slab_bytes),
                        sv->stream) != DSR_OK)
      return dsr_fail(ctx, DSR_ERR_CUDA, "server launch (user program): %s",
                      cudaGetErrorString(cudaGetLastError()));
  } else {
    serve_kernel_for(sv->cfg.program, sv->cfg.threads)<<<sv->grid, sv->cfg.threads,
                                                          batch_smem(sv->cfg.slab_bytes),
                                                          sv->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "server launch");
  }
  sv->running = true;
  return DSR_OK;
}

// Overflow bytes one team of `d` may hold at once, with the server's slab.
uint64_t team_spill(const dsr_region_desc &d, uint32_t slab) {
  uint64_t sp = 0, spill = 0;
  for (uint32_t k = 0; k < d.depth && k < DSR_MAX_DEPTH; ++k) {
    const uint64_t fp = pad16(d.frame_bytes[k]);
    if (sp + fp <= slab)
      sp += fp;
    else
      spill += fp;
  }
  return spill;
}

// Read new completion records (host side): free their slots and their
// overflow reservations, and keep each status for its ticket's poll.
void drain_completions(dsr_serve_state *sv) {
  for (;;) {
    CompRec *r = sv->comp + (sv->comp_pos % sv->cfg.capacity);
    const unsigned long long m = __atomic_load_n(&r->marker, __ATOMIC_ACQUIRE);
    if (m == 0) break;
    const uint64_t seq = m - 1;
    const uint32_t slot = static_cast<uint32_t>(seq % sv->cfg.capacity);
    sv->slot_done[slot] = seq + 1;
    sv->slot_status[slot] = r->status;
    __atomic_store_n(&r->marker, 0ull, __ATOMIC_RELAXED);
    ++sv->comp_pos;
    ++sv->completed;
    sv->slot_busy[slot] = 0;
    sv->reserved_bytes -= sv->slot_reserved[slot];
    sv->slot_reserved[slot] = 0;
    if (sv->collect_done) sv->just_done.push_back(seq);
  }
}

// Report ticket's completion once: *status, or false when it has none yet.
bool take_done(dsr_serve_state *sv, uint64_t ticket, int32_t *status) {
  const uint32_t slot = static_cast<uint32_t>(ticket % sv->cfg.capacity);
  if (sv->slot_done[slot] == ticket + 1) {
    *status = sv->slot_status[slot];
    sv->slot_done[slot] = 0;
    return true;
  }
  auto it = sv->unreported.find(ticket);
  if (it == sv->unreported.end()) return false;
  *status = it->second;
  sv->unreported.erase(it);
  return true;
}

}  // namespace

extern "C" uint64_t dsr_serve_workspace_bytes(uint32_t capacity) { return serve_ws_bytes(capacity); }

namespace {

// dsr_serve_start and dsr_serve_start_user: `user` null for a built-in program.
int32_t serve_start(dsr_ctx *ctx, const dsr_serve_cfg *cfg, void *workspace_dev,
                    uint64_t workspace_bytes, const dsr_serve_program *user) {
  if (!ctx || !cfg) return dsr_fail(ctx, DSR_ERR_INVALID, "null argument");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  if (int32_t rc = dsr_check_device(ctx)) return rc;
  if (ctx->serve && ctx->serve->running) return dsr_fail(ctx, DSR_ERR_INVALID, "already serving");
  if (user) {
    if (user->program < DSR_PROG_USER || cfg->program != user->program || !user->validate ||
        !user->prepare || !user->launch)
      return dsr_fail(ctx, DSR_ERR_INVALID,
                      "a user program's server needs its id (>= DSR_PROG_USER) in cfg and all hooks");
  } else if (!serve_kernel_for(cfg->program, cfg->threads)) {
    return dsr_fail(ctx, DSR_ERR_INVALID,
                    cfg->program >= DSR_PROG_USER
                        ? "a user-written program is served through dsr_serve_start_user"
                        : "the served form runs the scalars, nested and hetero programs");
  }
  if (cfg->threads < 64 || cfg->threads > DSR_MAX_THREADS || cfg->threads % 32 ||
      cfg->slab_bytes % 16 || batch_smem(cfg->slab_bytes) > static_cast<uint32_t>(ctx->max_smem_optin) ||
      cfg->capacity == 0 || cfg->capacity > (1u << 24) || !cfg->out_dev || !cfg->status_dev)
    return dsr_fail(ctx, DSR_ERR_INVALID, "bad serve configuration");
  if (!workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) & 15u) ||
      workspace_bytes < serve_ws_bytes(cfg->capacity))
    return dsr_fail(ctx, DSR_ERR_BUDGET, "serve workspace needs %llu bytes, 16-byte aligned",
                    (unsigned long long)serve_ws_bytes(cfg->capacity));
  dsr_serve_release(ctx);
  dsr_serve_state *sv = new dsr_serve_state();
  ctx->serve = sv;
  sv->cfg = *cfg;
  sv->is_user = user != nullptr;
  if (user) sv->user = *user;
  cudaError_t e;
  const unsigned fl = cudaHostAllocMapped | cudaHostAllocPortable;
  if ((e = cudaHostAlloc(&sv->ring, sizeof(dsr_region_desc) * cfg->capacity, fl)) != cudaSuccess ||
      (e = cudaHostAlloc(&sv->hs, sizeof(HostShared), fl)) != cudaSuccess ||
      (e = cudaHostAlloc(&sv->comp, sizeof(CompRec) * cfg->capacity, fl)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&sv->ring_dev, sv->ring, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&sv->hs_dev, sv->hs, 0)) != cudaSuccess ||
      (e = cudaHostGetDevicePointer(&sv->comp_dev, sv->comp, 0)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    int32_t rc = dsr_cuda_fail(ctx, e, "serve rings");
    dsr_serve_release(ctx);
    return rc;
  }
  std::memset(sv->ring, 0, sizeof(dsr_region_desc) * cfg->capacity);
  std::memset(sv->hs, 0, sizeof(HostShared));
  std::memset(sv->comp, 0, sizeof(CompRec) * cfg->capacity);
  sv->slot_busy.assign(cfg->capacity, 0);
  sv->slot_reserved.assign(cfg->capacity, 0);
  sv->slot_done.assign(cfg->capacity, 0);
  sv->slot_status.assign(cfg->capacity, 0);
  sv->ws = static_cast<ServeWs *>(workspace_dev);
  sv->slots = reinterpret_cast<SlotState *>(static_cast<uint8_t *>(workspace_dev) + sizeof(ServeWs));
  sv->dring = reinterpret_cast<dsr_region_desc *>(sv->slots + cfg->capacity);
  int occ = 0;
  if (user) {
    int32_t per_sm = 0;
    if (user->prepare(cfg->threads, batch_smem(cfg->slab_bytes), &per_sm) != DSR_OK) {
      int32_t rc = dsr_cuda_fail(ctx, cudaGetLastError(), "serve attributes (user program)");
      dsr_serve_release(ctx);
      return rc;
    }
    occ = per_sm;
  } else {
    ServeFn k = serve_kernel_for(cfg->program, cfg->threads);
    if ((e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ctx->max_smem_optin)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k),
                                  cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared)) != cudaSuccess) {
      int32_t rc = dsr_cuda_fail(ctx, e, "serve attributes");
      dsr_serve_release(ctx);
      return rc;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void *>(k),
                                                  cfg->threads, batch_smem(cfg->slab_bytes));
  }
  if (occ < 1) {
    dsr_serve_release(ctx);
    return dsr_fail(ctx, DSR_ERR_INVALID, "serve CTA shape does not fit an SM");
  }
  uint64_t g = static_cast<uint64_t>(ctx->sm_count) *
               (cfg->ctas_per_sm ? std::min<uint32_t>(cfg->ctas_per_sm, occ) : occ);
  if (ctx->ovf_per_team) g = std::min<uint64_t>(g, ctx->max_teams);
  if (g < 2) {
    dsr_serve_release(ctx);
    return dsr_fail(ctx, DSR_ERR_BUDGET, "a server needs two CTAs (the doorbell and one more)");
  }
  sv->grid = static_cast<uint32_t>(g);
  sv->pool_budget = ctx->ovf_per_team * g;
  serve_init<<<(cfg->capacity + 255) / 256, 256, 0, sv->stream>>>(sv->ws, sv->slots, cfg->capacity);
  int32_t rc = launch_server(ctx, sv);
  if (rc != DSR_OK) dsr_serve_release(ctx);
  return rc;
}

}  // namespace

extern "C" int32_t dsr_serve_start(dsr_ctx *ctx, const dsr_serve_cfg *cfg, void *workspace_dev,
                                   uint64_t workspace_bytes) {
  return serve_start(ctx, cfg, workspace_dev, workspace_bytes, nullptr);
}

extern "C" int32_t dsr_serve_start_user(dsr_ctx *ctx, const dsr_serve_cfg *cfg,
                                        void *workspace_dev, uint64_t workspace_bytes,
                                        const dsr_serve_program *prog) {
  if (!prog) return dsr_fail(ctx, DSR_ERR_INVALID, "null program");
  return serve_start(ctx, cfg, workspace_dev, workspace_bytes, prog);
}

extern "C" int32_t dsr_serve_submit(dsr_ctx *ctx, const dsr_region_desc *d, uint64_t *ticket) {
  if (!ctx || !ctx->serve || !d || !ticket) return dsr_fail(ctx, DSR_ERR_INVALID, "not serving");
  dsr_serve_state *sv = ctx->serve;
  if (d->program != sv->cfg.program) return dsr_fail(ctx, DSR_ERR_INVALID, "program mismatch");
  int32_t rc;
  if (sv->is_user) {
    if ((rc = sv->user.validate(d, sv->cfg.image_bytes, sv->cfg.out_bytes, sv->cfg.n_status)) !=
        DSR_OK)
      return dsr_fail(ctx, DSR_ERR_INVALID, "the program's check refused the descriptor");
  } else if ((rc = dsr_validate_region(d, sv->cfg.image_bytes, sv->cfg.out_bytes,
                                       sv->cfg.n_status)) != DSR_OK) {
    return dsr_fail(ctx, rc, "%s", dsr_last_error_string(nullptr));
  }
  const uint64_t spill = team_spill(*d, sv->cfg.slab_bytes);
  if (spill > ctx->ovf_per_team)
    return dsr_fail(ctx, DSR_ERR_OVERFLOW, "a team needs %llu overflow bytes, %llu per CTA",
                    (unsigned long long)spill, (unsigned long long)ctx->ovf_per_team);
  drain_completions(sv);
  // admission: the request's ring slot is free (its previous occupant has
  // completed), and its overflow reservation fits the pool
  if (sv->slot_busy[sv->next_seq % sv->cfg.capacity])
    return dsr_fail(ctx, DSR_ERR_BUDGET, "request ring full");
  const uint64_t want = spill * std::min<uint64_t>(d->teams, sv->grid);
  if (sv->reserved_bytes + want > sv->pool_budget)
    return dsr_fail(ctx, DSR_ERR_BUDGET, "overflow pool budget in use");
  // a server that left after its idle timeout is started again
  if (sv->running && server_exited(sv)) sv->running = false;
  if (!sv->running && (rc = launch_server(ctx, sv)) != DSR_OK) return rc;
  const uint64_t seq = sv->next_seq++;
  const uint32_t slot = static_cast<uint32_t>(seq % sv->cfg.capacity);
  if (sv->slot_done[slot]) {  // the slot's last completion was never polled: keep it
    sv->unreported[sv->slot_done[slot] - 1] = sv->slot_status[slot];
    sv->slot_done[slot] = 0;
  }
  sv->ring[slot] = *d;
  sv->slot_busy[slot] = 1;
  sv->slot_reserved[slot] = want;
  sv->reserved_bytes += want;
  __atomic_store_n(&sv->hs->tail, static_cast<unsigned long long>(seq + 1), __ATOMIC_RELEASE);
  *ticket = seq;
  return DSR_OK;
}

extern "C" int32_t dsr_serve_poll(dsr_ctx *ctx, uint64_t ticket, int32_t *status) {
  if (!ctx || !ctx->serve || !status) return dsr_fail(ctx, DSR_ERR_INVALID, "not serving");
  dsr_serve_state *sv = ctx->serve;
  drain_completions(sv);
  if (sv->running && sv->completed < sv->next_seq && server_exited(sv)) {
    // every CTA left after the idle timeout while work was published
    sv->running = false;
    int32_t rc = launch_server(ctx, sv);
    if (rc != DSR_OK) return rc;
  }
  if (!take_done(sv, ticket, status)) *status = DSR_PENDING;
  return DSR_OK;
}

extern "C" int32_t dsr_serve_stop(dsr_ctx *ctx) {
  if (!ctx || !ctx->serve) return DSR_OK;
  dsr_serve_state *sv = ctx->serve;
  __atomic_store_n(&sv->hs->stop, 1ull, __ATOMIC_RELEASE);
  // Every CTA leaves once the stop is seen and nothing is left to claim, or
  // after its idle timeout; wait for that, but not without end: a server
  // still running well past its idle timeout is reported, not waited on.
  const uint64_t idle = sv->cfg.idle_timeout_ns ? sv->cfg.idle_timeout_ns : 2000000000ull;
  const uint64_t deadline = now_ns() + 2 * idle + 30000000000ull;
  cudaError_t e;
  while ((e = cudaStreamQuery(sv->stream)) == cudaErrorNotReady) {
    if (now_ns() > deadline)
      return dsr_fail(ctx, DSR_ERR_TIMEOUT, "server did not drain within %.0f s of the stop",
                      (2 * idle + 30000000000ull) * 1e-9);
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  sv->running = false;
  __atomic_store_n(&sv->hs->stop, 0ull, __ATOMIC_RELEASE);
  drain_completions(sv);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "server stop");
  return DSR_OK;
}

extern "C" int32_t dsr_serve_stats(dsr_ctx *ctx, uint64_t *submitted, uint64_t *completed,
                                   uint32_t *idle_exits, uint32_t *errors) {
  if (!ctx || !ctx->serve) return dsr_fail(ctx, DSR_ERR_INVALID, "not serving");
  dsr_serve_state *sv = ctx->serve;
  drain_completions(sv);
  ServeWs w;
  cudaError_t e = cudaMemcpy(&w, sv->ws, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "serve stats");
  if (submitted) *submitted = sv->next_seq;
  if (completed) *completed = sv->completed;
  if (idle_exits) *idle_exits = w.idle_exits;
  if (errors) *errors = w.errors;
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Open-loop latency harnesses (host threads; the clock is CLOCK_MONOTONIC)
// ---------------------------------------------------------------------------
extern "C" int32_t dsr_serve_bench(dsr_ctx *ctx, const dsr_region_desc *descs, uint32_t n,
                                   const int64_t *arrival_ns, int64_t *latency_ns,
                                   int64_t *elapsed_ns) {
  if (!ctx || !ctx->serve || !descs || !arrival_ns || !latency_ns)
    return dsr_fail(ctx, DSR_ERR_INVALID, "not serving or null argument");
  dsr_serve_state *sv = ctx->serve;
  // the request of each ring slot's ticket (a slot holds one request at a time)
  std::vector<uint32_t> req_of_slot(sv->cfg.capacity, ~0u);
  std::vector<uint64_t> ticket_of_slot(sv->cfg.capacity, ~0ull);
  const uint64_t t0 = now_ns() + 1000000;  // start 1 ms from now
  uint32_t next = 0, finished = 0;
  sv->just_done.clear();
  sv->collect_done = true;
  struct Stop {  // stop collecting however the loop ends
    dsr_serve_state *sv;
    ~Stop() {
      sv->collect_done = false;
      sv->just_done.clear();
    }
  } stop_collecting{sv};
  for (uint32_t i = 0; i < n; ++i) latency_ns[i] = -1;
  const uint64_t deadline = t0 + static_cast<uint64_t>(arrival_ns[n ? n - 1 : 0]) + 30000000000ull;
  while (finished < n) {
    const uint64_t now = now_ns();
    if (now > deadline) return dsr_fail(ctx, DSR_ERR_TIMEOUT, "serve bench did not finish");
    // submit every request whose arrival time has come (open loop: a full
    // ring delays the submission, and that delay counts as latency)
    while (next < n && now >= t0 + static_cast<uint64_t>(arrival_ns[next])) {
      uint64_t tk;
      const int32_t rc = dsr_serve_submit(ctx, descs + next, &tk);
      if (rc == DSR_ERR_BUDGET) break;
      if (rc != DSR_OK) return rc;
      req_of_slot[tk % sv->cfg.capacity] = next;
      ticket_of_slot[tk % sv->cfg.capacity] = tk;
      ++next;
    }
    drain_completions(sv);
    if (!sv->just_done.empty()) {
      const uint64_t t_done = now_ns();
      for (const uint64_t tk : sv->just_done) {
        const uint32_t slot = static_cast<uint32_t>(tk % sv->cfg.capacity);
        if (ticket_of_slot[slot] != tk) continue;  // not one of this run's requests
        int32_t st = DSR_OK;
        take_done(sv, tk, &st);
        const uint32_t i = req_of_slot[slot];
        latency_ns[i] = static_cast<int64_t>(t_done - (t0 + arrival_ns[i]));
        if (st != DSR_OK) latency_ns[i] = -2 - st;
        ticket_of_slot[slot] = ~0ull;
        ++finished;
      }
      sv->just_done.clear();
    }
  }
  if (elapsed_ns) *elapsed_ns = static_cast<int64_t>(now_ns() - t0);
  return DSR_OK;
}

// The same open-loop arrivals served by one plain kernel launch per request
// on `stream`; completion is observed through an event per request.
extern "C" int32_t dsr_launch_bench(dsr_ctx *ctx, const dsr_region_desc *descs, uint32_t n,
                                    const int64_t *arrival_ns, int64_t *latency_ns,
                                    int64_t *elapsed_ns, const void *images_dev,
                                    uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                                    dsr_team_status *status_dev, uint64_t n_status,
                                    void *stream) {
  if (!ctx || !descs || !arrival_ns || !latency_ns)
    return dsr_fail(ctx, DSR_ERR_INVALID, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t kEvents = 4096;
  std::vector<cudaEvent_t> ev(kEvents);
  for (auto &x : ev) cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  std::deque<std::pair<uint32_t, uint32_t>> inflight;  // (request, event)
  uint32_t next = 0, finished = 0, ev_next = 0;
  const uint64_t t0 = now_ns() + 1000000;
  const uint64_t deadline = t0 + static_cast<uint64_t>(arrival_ns[n ? n - 1 : 0]) + 60000000000ull;
  int32_t rc = DSR_OK;
  while (finished < n && rc == DSR_OK) {
    const uint64_t now = now_ns();
    if (now > deadline) {
      rc = dsr_fail(ctx, DSR_ERR_TIMEOUT, "launch bench did not finish");
      break;
    }
    while (next < n && now >= t0 + static_cast<uint64_t>(arrival_ns[next]) &&
           inflight.size() < kEvents) {
      rc = dsr_launch_region(ctx, descs + next, images_dev, image_bytes, out_dev, out_bytes,
                             status_dev, n_status, stream);
      if (rc != DSR_OK) break;
      cudaEventRecord(ev[ev_next], s);
      inflight.emplace_back(next, ev_next);
      ev_next = (ev_next + 1) % kEvents;
      ++next;
    }
    while (!inflight.empty() && cudaEventQuery(ev[inflight.front().second]) == cudaSuccess) {
      const uint32_t i = inflight.front().first;
      latency_ns[i] = static_cast<int64_t>(now_ns() - (t0 + arrival_ns[i]));
      inflight.pop_front();
      ++finished;
    }
  }
  cudaStreamSynchronize(s);
  for (auto &x : ev) cudaEventDestroy(x);
  if (elapsed_ns) *elapsed_ns = static_cast<int64_t>(now_ns() - t0);
  return rc;
}
