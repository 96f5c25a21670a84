// dsr_capi.cu -- plain per-region launch and the host side of the C ABI:
// context, stack configuration, descriptor checks, footprint model. The
// plain kernel itself (plain_kernel in dsr_kernels.cuh) is a template over
// the program, shared with programs written against dsr_device.cuh.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "dsr.h"
#include "dsr_check.cuh"
#include "dsr_ctx.h"
#include "dsr_kernels.cuh"
#include "dsr_programs.cuh"

using namespace dsr;

namespace {

using KernelFn = PlainFn;

KernelFn plain_kernel_for(uint32_t program, uint32_t threads, uint32_t param = 0) {
  switch (program) {
    case DSR_PROG_PAPER_SCALARS: return pick_plain<ProgPaperScalars>(threads);
    case DSR_PROG_PAPER_ARRAYS: return pick_plain<ProgPaperArrays>(threads);
    case DSR_PROG_SCALARS: return pick_plain<ProgScalars>(threads);
    case DSR_PROG_NESTED: return pick_plain<ProgNested>(threads);
    case DSR_PROG_SWEEP: return pick_plain<ProgSweep>(threads);
    case DSR_PROG_HETERO: return pick_plain<ProgHetero>(threads);
    case DSR_PROG_WORKERS:
      return param == 1 ? pick_plain<ProgWorkersSmem>(threads) : pick_plain<ProgWorkers>(threads);
    default: return nullptr;
  }
}

std::mutex g_err_mu;
std::string g_last_err;

}  // namespace

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
int32_t dsr_fail(dsr_ctx *ctx, int32_t code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  std::lock_guard<std::mutex> g(g_err_mu);
  g_last_err = buf;
  return code;
}

int32_t dsr_cuda_fail(dsr_ctx *ctx, cudaError_t e, const char *what) {
  return dsr_fail(ctx, DSR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int32_t dsr_check_device(dsr_ctx *ctx) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "cudaGetDevice");
  if (cur != ctx->device)
    return dsr_fail(ctx, DSR_ERR_INVALID,
                    "the calling thread's current device is %d, the context's is %d "
                    "(cudaSetDevice(%d) first)",
                    cur, ctx->device, ctx->device);
  return DSR_OK;
}

extern "C" int32_t dsr_report_error(dsr_ctx *ctx, int32_t code, const char *msg) {
  return dsr_fail(ctx, code, "%s", msg ? msg : "");
}

extern "C" const char *dsr_last_error_string(const dsr_ctx *ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> g(g_err_mu);
  thread_local std::string copy;
  copy = g_last_err;
  return copy.c_str();
}

// ---------------------------------------------------------------------------
// Descriptor checks (host side of dsr_check.cuh)
// ---------------------------------------------------------------------------
int32_t dsr_check_shape(const dsr_region_desc *d, const char **why) {
  static const char *const kWhy[] = {
      "",
      "shape out of range (teams >= 1, threads a multiple of 32 in [32, 1024], "
      "depth 1..4, width <= workers)",
      "frame sizes must be positive multiples of 4",
      "image/out offsets must be 16-byte aligned",
      "frame sizes do not match the program's layout",
      "unknown program"};
  *why = "";
  if (!d) return (*why = "null descriptor"), DSR_ERR_INVALID;
  const int e = dsr::shape_error(*d);
  *why = kWhy[e];
  return e ? DSR_ERR_INVALID : DSR_OK;
}

extern "C" int32_t dsr_region_extent(const dsr_region_desc *d, uint64_t *image_bytes,
                                     uint64_t *out_bytes, uint64_t *n_status) {
  const char *why;
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(nullptr, DSR_ERR_INVALID, "%s", why);
  uint64_t ib, ob, ns;
  dsr::extent(*d, &ib, &ob, &ns);
  if (image_bytes) *image_bytes = ib;
  if (out_bytes) *out_bytes = ob;
  if (n_status) *n_status = ns;
  return DSR_OK;
}

extern "C" int32_t dsr_validate_region(const dsr_region_desc *d, uint64_t image_bytes,
                                       uint64_t out_bytes, uint64_t n_status) {
  uint64_t ib, ob, ns;
  int32_t rc = dsr_region_extent(d, &ib, &ob, &ns);
  if (rc != DSR_OK) return rc;
  if (!dsr::fits(*d, image_bytes, out_bytes, n_status))
    return dsr_fail(nullptr, DSR_ERR_INVALID,
                    "region needs images [%llu, +%llu) of %llu, outputs [%llu, +%llu) of %llu, "
                    "statuses [%u, +%llu) of %llu",
                    (unsigned long long)d->image_offset, (unsigned long long)ib,
                    (unsigned long long)image_bytes, (unsigned long long)d->out_offset,
                    (unsigned long long)ob, (unsigned long long)out_bytes, d->status_index,
                    (unsigned long long)ns, (unsigned long long)n_status);
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Footprint / occupancy model (GB300 SM): the counterpart of the paper's
// per-team footprint (Sec. 6.2.1) and teams-per-SM arithmetic (Sec. 6.2.2).
// ---------------------------------------------------------------------------
namespace {
constexpr uint32_t kSmemPerSm = 233472;      // 228 KB
constexpr uint32_t kSmemReservedPerCta = 1024;
constexpr uint32_t kMaxSmemPerCta = 232448;  // 227 KB opt-in
constexpr uint32_t kWarpsPerSm = 64;
constexpr uint32_t kCtasPerSm = 32;
constexpr uint32_t kRegsPerSm = 65536;
}  // namespace

extern "C" int32_t dsr_footprint_model(const dsr_region_desc *d, uint32_t slab_bytes,
                                       uint32_t regs, dsr_footprint *out) {
  const char *why;
  if (!out) return dsr_fail(nullptr, DSR_ERR_INVALID, "null output");
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(nullptr, DSR_ERR_INVALID, "%s", why);
  if (slab_bytes % 16 || slab_bytes + kCtrlBytes > kMaxSmemPerCta)
    return dsr_fail(nullptr, DSR_ERR_INVALID, "slab must be a multiple of 16 and fit a CTA");
  if (regs == 0) regs = 64;
  if (regs > 255) return dsr_fail(nullptr, DSR_ERR_INVALID, "regs > 255");
  // frames of one team are all live at the deepest point: place them in
  // push order, first fit into the slab, else the overflow slab
  const uint64_t spill = dsr::spill_bytes(*d, slab_bytes);
  const uint32_t warps = d->threads / 32;
  const uint32_t smem = kCtrlBytes + slab_bytes;
  const uint32_t by_threads = kWarpsPerSm / warps;
  const uint32_t by_smem = kSmemPerSm / (smem + kSmemReservedPerCta);
  const uint32_t regs_per_warp = ((regs + 7u) & ~7u) * 32u;
  const uint32_t by_regs = (kRegsPerSm / regs_per_warp) / warps;
  uint32_t best = kCtasPerSm, limit = 4;
  if (by_threads < best) best = by_threads, limit = 1;
  if (by_smem < best) best = by_smem, limit = 2;
  if (by_regs < best) best = by_regs, limit = 3;
  out->smem_per_team = smem;
  out->ctrl_bytes = kCtrlBytes;
  out->slab_bytes = slab_bytes;
  out->teams_per_sm = best;
  out->limit = limit;
  out->spill_bytes = static_cast<uint32_t>(spill);
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Lifecycle and stacks
// ---------------------------------------------------------------------------
extern "C" int32_t dsr_create(dsr_ctx **out, const dsr_config *cfg) {
  if (!out) return dsr_fail(nullptr, DSR_ERR_INVALID, "null output handle");
  *out = nullptr;
  dsr_config c{};
  if (cfg) c = *cfg;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return dsr_fail(nullptr, DSR_ERR_CUDA, "no CUDA device: %s",
                    e == cudaSuccess ? "count is 0" : cudaGetErrorString(e));
  }
  if (c.device < 0 || c.device >= n) return dsr_fail(nullptr, DSR_ERR_INVALID, "bad device");
  dsr_ctx *ctx = new dsr_ctx();
  ctx->device = c.device;
  ctx->timeout_ns = c.wait_timeout_ns ? c.wait_timeout_ns : 1000000000ull;
  if ((e = cudaSetDevice(c.device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, c.device)) !=
          cudaSuccess ||
      (e = cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  c.device)) != cudaSuccess) {
    int32_t rc = dsr_cuda_fail(nullptr, e, "device query");
    delete ctx;
    return rc;
  }
  *out = ctx;
  return DSR_OK;
}

extern "C" int32_t dsr_destroy(dsr_ctx *ctx) {
  if (!ctx) return DSR_OK;
  dsr_ctx_release(ctx);
  delete ctx;
  return DSR_OK;
}

// Every plain kernel instance may take all the dynamic shared memory a CTA
// can opt in to (less its own static shared memory), with the carveout
// preferring shared memory to L1.
static int32_t set_smem_attr(dsr_ctx *ctx) {
  static const uint32_t kThreads[] = {128, 256, 512, 1024};
  for (uint32_t p = DSR_PROG_PAPER_SCALARS; p <= DSR_PROG_WORKERS + 1; ++p)
    for (uint32_t t : kThreads) {
      // the last round: the worker program's shared-memory-table variant
      const void *k = reinterpret_cast<const void *>(
          p <= DSR_PROG_WORKERS ? plain_kernel_for(p, t) : plain_kernel_for(DSR_PROG_WORKERS, t, 1));
      // a kernel with static shared memory of its own can take that much
      // less dynamic shared memory (a larger slab then fails at launch)
      cudaFuncAttributes fa{};
      cudaError_t e = cudaFuncGetAttributes(&fa, k);
      if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "cudaFuncGetAttributes");
      // the ceiling is all a CTA may take: a plain launch asks for its slab
      // or, to balance residency, a padded size (balanced_smem), and a
      // ceiling set to one slab would refuse another's
      const uint32_t room = static_cast<uint32_t>(ctx->max_smem_optin) -
                            static_cast<uint32_t>(fa.sharedSizeBytes);
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(room));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
  return DSR_OK;
}

extern "C" int32_t dsr_region_footprint(const dsr_region_desc *d, uint64_t *stack_bytes,
                                        uint64_t *slab_bytes) {
  const char *why;
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(nullptr, DSR_ERR_INVALID, "%s", why);
  uint64_t st, sl;
  dsr::footprint(*d, &st, &sl);
  if (stack_bytes) *stack_bytes = st;
  if (slab_bytes) *slab_bytes = sl;
  return DSR_OK;
}

uint32_t dsr_plain_slab(const dsr_ctx *ctx, const dsr_region_desc *d) {
  if (!ctx->slab_auto) return ctx->slab_bytes;
  uint64_t st, sl;
  dsr::footprint(*d, &st, &sl);
  return static_cast<uint32_t>(sl < ctx->slab_bytes ? dsr::pad16(sl) : ctx->slab_bytes);
}

extern "C" int32_t dsr_stack_init(dsr_ctx *ctx, uint32_t smem_slab_bytes,
                                  uint64_t overflow_bytes_per_team, uint32_t max_teams,
                                  void *overflow_pool_dev, uint64_t pool_bytes) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  const bool slab_auto = smem_slab_bytes == DSR_SLAB_AUTO;
  if (slab_auto)  // the cap: what one CTA can hold next to the control block
    smem_slab_bytes = (static_cast<uint32_t>(ctx->max_smem_optin) - kCtrlBytes) & ~15u;
  if (smem_slab_bytes % 16 || overflow_bytes_per_team % 16)
    return dsr_fail(ctx, DSR_ERR_INVALID, "slab sizes must be multiples of 16");
  if (kCtrlBytes + smem_slab_bytes > static_cast<uint32_t>(ctx->max_smem_optin))
    return dsr_fail(ctx, DSR_ERR_INVALID, "slab %u + control %u exceeds %d bytes per CTA",
                    smem_slab_bytes, kCtrlBytes, ctx->max_smem_optin);
  if (overflow_bytes_per_team) {
    if (!overflow_pool_dev || reinterpret_cast<uintptr_t>(overflow_pool_dev) % 16)
      return dsr_fail(ctx, DSR_ERR_INVALID, "overflow pool must be a 16-byte aligned pointer");
    if (max_teams == 0 || static_cast<double>(max_teams) * overflow_bytes_per_team > 1.8e19 ||
        max_teams * overflow_bytes_per_team > pool_bytes)
      return dsr_fail(ctx, DSR_ERR_BUDGET, "pool of %llu bytes cannot hold %u x %llu bytes",
                      (unsigned long long)pool_bytes, max_teams,
                      (unsigned long long)overflow_bytes_per_team);
  }
  int32_t rc = set_smem_attr(ctx);
  if (rc != DSR_OK) return rc;
  rc = dsr_ctx_stack_changed(ctx, kCtrlBytes + smem_slab_bytes);
  if (rc != DSR_OK) return rc;
  ctx->slab_bytes = smem_slab_bytes;
  ctx->slab_auto = slab_auto;
  ctx->ovf_per_team = overflow_bytes_per_team;
  ctx->max_teams = overflow_bytes_per_team ? max_teams : 0xffffffffu;
  ctx->pool = static_cast<uint8_t *>(overflow_pool_dev);
  ctx->pool_bytes = pool_bytes;
  ctx->stack_ready = true;
  ++ctx->stack_gen;
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Plain launch
// ---------------------------------------------------------------------------
uint32_t dsr_plain_launch_smem(dsr_ctx *ctx, const dsr_region_desc *d) {
  const uint32_t block = d->threads > 32u ? d->threads : 64u;
  const void *k = reinterpret_cast<const void *>(plain_kernel_for(d->program, block, d->param));
  return balanced_smem(k, block, kCtrlBytes + dsr_plain_slab(ctx, d), d->teams, ctx->device,
                       static_cast<uint32_t>(ctx->max_smem_optin));
}

int32_t dsr_launch_plain(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                         void *out_dev, dsr_team_status *status_dev, cudaStream_t s) {
  // a team without workers gets one worker warp (its region width is 1)
  const uint32_t block = d->threads > 32u ? d->threads : 64u;
  KernelFn k = plain_kernel_for(d->program, block, d->param);
  const uint32_t slab = dsr_plain_slab(ctx, d);
  // programmatic stream serialisation: this grid may be dispatched while the
  // kernel before it in the stream drains (its threads wait for that kernel
  // before touching global memory); consecutive regions overlap a launch's
  // CTA placement with the previous region's tail
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(d->teams);
  cfg.blockDim = dim3(block);
  // at most ceil(teams / SMs) CTAs per SM when fewer than the occupancy
  cfg.dynamicSmemBytes = dsr_plain_launch_smem(ctx, d);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(
      &cfg, k, *d, static_cast<const uint8_t *>(images_dev), static_cast<uint8_t *>(out_dev),
      status_dev, ctx->pool, ctx->ovf_per_team, slab, ctx->timeout_ns);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "plain launch");
  return DSR_OK;
}

// Checks every plain launch makes, built-in or user-written program.
static int32_t check_launch_common(dsr_ctx *ctx, const dsr_region_desc *d, const void *out_dev,
                                   const void *status_dev) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  int32_t rc = dsr_check_device(ctx);
  if (rc != DSR_OK) return rc;
  const char *why;
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(ctx, DSR_ERR_INVALID, "%s", why);
  if (!out_dev || !status_dev) return dsr_fail(ctx, DSR_ERR_INVALID, "null output or status");
  if (ctx->ovf_per_team && d->teams > ctx->max_teams)
    return dsr_fail(ctx, DSR_ERR_BUDGET, "%u teams exceed the %u overflow slabs", d->teams,
                    ctx->max_teams);
  return DSR_OK;
}

static int32_t check_launch(dsr_ctx *ctx, const dsr_region_desc *d, const void *out_dev,
                            const void *status_dev) {
  int32_t rc = check_launch_common(ctx, d, out_dev, status_dev);
  if (rc == DSR_OK && d->program >= DSR_PROG_USER)
    return dsr_fail(ctx, DSR_ERR_INVALID,
                    "program %u is user-written: launch it with dsr_launch_user_region",
                    d->program);
  return rc;
}

// ---------------------------------------------------------------------------
// Plain launches of user-written programs (dsr_device.cuh): the checks and
// the ctx's stack configuration; the user's translation unit launches its
// own instance of the plain kernel with them.
// ---------------------------------------------------------------------------
extern "C" int32_t dsr_user_plain_config(dsr_ctx *ctx, const dsr_region_desc *d,
                                         uint64_t image_need, uint64_t out_need,
                                         uint64_t image_bytes, uint64_t out_bytes,
                                         uint64_t n_status, const void *out_dev,
                                         const void *status_dev, dsr_plain_config *cfg) {
  if (!cfg) return dsr_fail(ctx, DSR_ERR_INVALID, "null output");
  int32_t rc = check_launch_common(ctx, d, out_dev, status_dev);
  if (rc != DSR_OK) return rc;
  if (d->program < DSR_PROG_USER)
    return dsr_fail(ctx, DSR_ERR_INVALID, "program %u is built in: use dsr_launch_region",
                    d->program);
  if (image_need && (d->image_offset > image_bytes || image_need > image_bytes - d->image_offset))
    return dsr_fail(ctx, DSR_ERR_INVALID, "region needs images [%llu, +%llu) of %llu",
                    (unsigned long long)d->image_offset, (unsigned long long)image_need,
                    (unsigned long long)image_bytes);
  if (d->out_offset > out_bytes || out_need > out_bytes - d->out_offset)
    return dsr_fail(ctx, DSR_ERR_INVALID, "region needs outputs [%llu, +%llu) of %llu",
                    (unsigned long long)d->out_offset, (unsigned long long)out_need,
                    (unsigned long long)out_bytes);
  if (static_cast<uint64_t>(d->status_index) + d->teams > n_status)
    return dsr_fail(ctx, DSR_ERR_INVALID, "region needs statuses [%u, +%u) of %llu",
                    d->status_index, d->teams, (unsigned long long)n_status);
  cfg->pool_dev = ctx->pool;
  cfg->ovf_per_team = ctx->ovf_per_team;
  cfg->timeout_ns = ctx->timeout_ns;
  cfg->slab_bytes = dsr_plain_slab(ctx, d);
  cfg->ctrl_bytes = kCtrlBytes;
  cfg->device = ctx->device;
  cfg->max_smem = static_cast<uint32_t>(ctx->max_smem_optin);
  return DSR_OK;
}

int32_t dsr_check_region_launch(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                                uint64_t image_bytes, const void *out_dev, uint64_t out_bytes,
                                const void *status_dev, uint64_t n_status) {
  int32_t rc = check_launch(ctx, d, out_dev, status_dev);
  if (rc != DSR_OK) return rc;
  if ((rc = dsr_validate_region(d, image_bytes, out_bytes, n_status)) != DSR_OK)
    return dsr_fail(ctx, rc, "%s", dsr_last_error_string(nullptr));
  uint64_t ib = 0;
  dsr_region_extent(d, &ib, nullptr, nullptr);
  if (ib && !images_dev) return dsr_fail(ctx, DSR_ERR_INVALID, "null images");
  return DSR_OK;
}

extern "C" int32_t dsr_launch_region(dsr_ctx *ctx, const dsr_region_desc *d,
                                     const void *images_dev, uint64_t image_bytes,
                                     void *out_dev, uint64_t out_bytes,
                                     dsr_team_status *status_dev, uint64_t n_status,
                                     void *stream) {
  int32_t rc = dsr_check_region_launch(ctx, d, images_dev, image_bytes, out_dev, out_bytes,
                                       status_dev, n_status);
  if (rc != DSR_OK) return rc;
  return dsr_launch_plain(ctx, d, images_dev, out_dev, status_dev,
                          static_cast<cudaStream_t>(stream));
}

extern "C" int32_t dsr_region_occupancy(dsr_ctx *ctx, const dsr_region_desc *d,
                                        dsr_occupancy *out) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!out) return dsr_fail(ctx, DSR_ERR_INVALID, "null output");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  const char *why;
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(ctx, DSR_ERR_INVALID, "%s", why);
  const uint32_t block = d->threads > 32u ? d->threads : 64u;
  const void *k = reinterpret_cast<const void *>(plain_kernel_for(d->program, block, d->param));
  const uint32_t slab = dsr_plain_slab(ctx, d);
  const uint32_t smem = kCtrlBytes + slab;
  cudaFuncAttributes a{};
  int per_sm = 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k);
  // resident CTAs of the launch as made: the balanced dynamic shared memory
  const uint32_t launch_smem =
      e == cudaSuccess ? balanced_smem(k, block, smem, d->teams, ctx->device,
                                       static_cast<uint32_t>(ctx->max_smem_optin))
                       : smem;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, static_cast<int>(block),
                                                      static_cast<size_t>(launch_smem));
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "occupancy query");
  const uint64_t spill = dsr::spill_bytes(*d, slab);
  out->threads = block;
  out->regs_per_thread = static_cast<uint32_t>(a.numRegs);
  out->smem_per_team = smem;
  out->ctas_per_sm = static_cast<uint32_t>(per_sm);
  out->sm_count = static_cast<uint32_t>(ctx->sm_count);
  out->spill_bytes = static_cast<uint32_t>(spill);
  return DSR_OK;
}

extern "C" int32_t dsr_enqueue_region_host(dsr_ctx *ctx, const dsr_region_desc *d,
                                           const void *images_host, uint64_t image_bytes,
                                           void *out_host, uint64_t out_bytes,
                                           dsr_team_status *status_host, void *images_dev,
                                           void *out_dev, dsr_team_status *status_dev,
                                           void *stream) {
  int32_t rc = check_launch(ctx, d, out_dev, status_dev);
  if (rc != DSR_OK) return rc;
  if (!out_host || !status_host) return dsr_fail(ctx, DSR_ERR_INVALID, "null host buffers");
  rc = dsr_validate_region(d, image_bytes, out_bytes, static_cast<uint64_t>(d->status_index) +
                                                         d->teams);
  if (rc != DSR_OK) return dsr_fail(ctx, rc, "%s", dsr_last_error_string(nullptr));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (image_bytes) {
    if (!images_host || !images_dev) return dsr_fail(ctx, DSR_ERR_INVALID, "null images");
    e = cudaMemcpyAsync(images_dev, images_host, image_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "image upload");
  }
  const bool in_place =
      d->program == DSR_PROG_PAPER_SCALARS || d->program == DSR_PROG_PAPER_ARRAYS;
  if (in_place && (e = cudaMemcpyAsync(out_dev, out_host, out_bytes, cudaMemcpyHostToDevice,
                                       s)) != cudaSuccess)
    return dsr_cuda_fail(ctx, e, "output upload");
  rc = dsr_launch_plain(ctx, d, images_dev, out_dev, status_dev, s);
  if (rc != DSR_OK) return rc;
  if ((e = cudaMemcpyAsync(out_host, out_dev, out_bytes, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(status_host + d->status_index, status_dev + d->status_index,
                           sizeof(dsr_team_status) * d->teams, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess)
    return dsr_cuda_fail(ctx, e, "download");
  return DSR_OK;
}

extern "C" int32_t dsr_run_region_host(dsr_ctx *ctx, const dsr_region_desc *d,
                                       const void *images_host, uint64_t image_bytes,
                                       void *out_host, uint64_t out_bytes,
                                       dsr_team_status *status_host, void *images_dev,
                                       void *out_dev, dsr_team_status *status_dev,
                                       void *stream) {
  int32_t rc = dsr_enqueue_region_host(ctx, d, images_host, image_bytes, out_host, out_bytes,
                                       status_host, images_dev, out_dev, status_dev, stream);
  if (rc != DSR_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "sync");
  return DSR_OK;
}
