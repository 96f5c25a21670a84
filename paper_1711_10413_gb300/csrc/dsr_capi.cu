// dsr_capi.cu -- plain per-region launch and the host side of the C ABI:
// context, stack configuration, descriptor checks, footprint model.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "dsr.h"
#include "dsr_ctx.h"
#include "dsr_programs.cuh"

using namespace dsr;

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
  if (threadIdx.x < team_workers()) {
    worker_loop<P>(e);
    return;
  }
  team_setup(slab_bytes,
             ovf_per_team ? pool + static_cast<uint64_t>(blockIdx.x) * ovf_per_team : nullptr,
             ovf_per_team, timeout_ns, true);
  P::master(e);
  terminate_workers();
  team_report(e, st);
}

namespace {

using KernelFn = void (*)(dsr_region_desc, const uint8_t *, uint8_t *, dsr_team_status *,
                          uint8_t *, uint64_t, uint32_t, uint64_t);

template <class P>
KernelFn pick(uint32_t threads) {
  if (threads <= 128) return plain_kernel<P, 128, 16>;
  if (threads <= 256) return plain_kernel<P, 256, 8>;
  if (threads <= 512) return plain_kernel<P, 512, 4>;
  return plain_kernel<P, 1024, 2>;
}

KernelFn plain_kernel_for(uint32_t program, uint32_t threads) {
  switch (program) {
    case DSR_PROG_PAPER_SCALARS: return pick<ProgPaperScalars>(threads);
    case DSR_PROG_PAPER_ARRAYS: return pick<ProgPaperArrays>(threads);
    case DSR_PROG_SCALARS: return pick<ProgScalars>(threads);
    case DSR_PROG_NESTED: return pick<ProgNested>(threads);
    case DSR_PROG_SWEEP: return pick<ProgSweep>(threads);
    case DSR_PROG_HETERO: return pick<ProgHetero>(threads);
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

extern "C" const char *dsr_last_error_string(const dsr_ctx *ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> g(g_err_mu);
  thread_local std::string copy;
  copy = g_last_err;
  return copy.c_str();
}

// ---------------------------------------------------------------------------
// Descriptor checks (host only)
// ---------------------------------------------------------------------------
static uint64_t pad16(uint64_t n) { return (n + 15u) & ~static_cast<uint64_t>(15u); }

static uint32_t desc_width(const dsr_region_desc &d) {
  const uint32_t w = d.threads > 32u ? d.threads - 32u : 1u;
  return d.width ? d.width : w;
}

int32_t dsr_check_shape(const dsr_region_desc *d, const char **why) {
  *why = "";
  if (!d) return (*why = "null descriptor"), DSR_ERR_INVALID;
  if (d->teams == 0 || d->teams > 0x7fffffffu) return (*why = "teams out of range"), DSR_ERR_INVALID;
  if (d->threads < 32 || d->threads > DSR_MAX_THREADS || d->threads % 32)
    return (*why = "threads must be a multiple of 32 in [32, 1024]"), DSR_ERR_INVALID;
  if (d->depth == 0 || d->depth > DSR_MAX_DEPTH) return (*why = "depth out of range"), DSR_ERR_INVALID;
  const uint32_t wmax = d->threads > 32u ? d->threads - 32u : 1u;
  if (d->width > wmax) return (*why = "width exceeds the team's workers"), DSR_ERR_INVALID;
  for (uint32_t k = 0; k < d->depth; ++k)
    if (d->frame_bytes[k] == 0 || d->frame_bytes[k] % 4)
      return (*why = "frame sizes must be positive multiples of 4"), DSR_ERR_INVALID;
  if (d->image_offset % 16 || d->out_offset % 16)
    return (*why = "image/out offsets must be 16-byte aligned"), DSR_ERR_INVALID;
  const uint32_t w = desc_width(*d);
  switch (d->program) {
    case DSR_PROG_PAPER_SCALARS:
      if (d->depth != 1 || d->param == 0 || d->param > 4096 ||
          d->frame_bytes[0] != ((4u * d->param + 7u) & ~7u) + 8u)
        return (*why = "paper-scalars frame must hold param ints and a pointer"), DSR_ERR_INVALID;
      break;
    case DSR_PROG_PAPER_ARRAYS:
      if (d->depth != 1 || d->param == 0 || d->param > 4096 ||
          d->frame_bytes[0] != 4u * d->param * w)
        return (*why = "paper-arrays frame must hold param int[width] arrays"), DSR_ERR_INVALID;
      break;
    case DSR_PROG_SCALARS:
      if (d->depth != 1 || d->frame_bytes[0] != 16 || d->param == 0)
        return (*why = "scalars needs depth 1, a 16-byte frame, param >= 1"), DSR_ERR_INVALID;
      break;
    case DSR_PROG_NESTED:
      for (uint32_t k = 0; k < d->depth; ++k)
        if (d->frame_bytes[k] != 1088)
          return (*why = "nested frames are 1088 bytes"), DSR_ERR_INVALID;
      if (d->param == 0 || static_cast<uint64_t>(d->teams) * d->param > 0xffffffffull)
        return (*why = "nested needs 1 <= teams*param < 2^32"), DSR_ERR_INVALID;
      break;
    case DSR_PROG_SWEEP:
      if (d->depth != 1) return (*why = "sweep has one frame"), DSR_ERR_INVALID;
      break;
    case DSR_PROG_HETERO:
      break;
    default:
      return (*why = "unknown program"), DSR_ERR_INVALID;
  }
  return DSR_OK;
}

extern "C" int32_t dsr_region_extent(const dsr_region_desc *d, uint64_t *image_bytes,
                                     uint64_t *out_bytes, uint64_t *n_status) {
  const char *why;
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(nullptr, DSR_ERR_INVALID, "%s", why);
  const uint64_t T = d->teams, w = desc_width(*d);
  uint64_t ib = 0, ob = 0;
  switch (d->program) {
    case DSR_PROG_PAPER_SCALARS:
    case DSR_PROG_PAPER_ARRAYS: ob = 4 * T * w; break;
    case DSR_PROG_SCALARS: ib = 16ull * d->param; ob = 4ull * d->param * T * w; break;
    case DSR_PROG_NESTED: ib = T * d->depth * 1088ull; ob = 4 * T * d->param; break;
    case DSR_PROG_SWEEP: ib = T * d->frame_bytes[0]; ob = 4 * T * w; break;
    case DSR_PROG_HETERO:
      for (uint32_t k = 0; k < d->depth; ++k) ib += pad16(d->frame_bytes[k]);
      ob = 4 * T * w;
      break;
  }
  if (image_bytes) *image_bytes = ib;
  if (out_bytes) *out_bytes = ob;
  if (n_status) *n_status = T;
  return DSR_OK;
}

extern "C" int32_t dsr_validate_region(const dsr_region_desc *d, uint64_t image_bytes,
                                       uint64_t out_bytes, uint64_t n_status) {
  uint64_t ib, ob, ns;
  int32_t rc = dsr_region_extent(d, &ib, &ob, &ns);
  if (rc != DSR_OK) return rc;
  if (ib && d->image_offset + ib > image_bytes)
    return dsr_fail(nullptr, DSR_ERR_INVALID, "images end at %llu > %llu bytes",
                    (unsigned long long)(d->image_offset + ib), (unsigned long long)image_bytes);
  if (d->out_offset + ob > out_bytes)
    return dsr_fail(nullptr, DSR_ERR_INVALID, "outputs end at %llu > %llu bytes",
                    (unsigned long long)(d->out_offset + ob), (unsigned long long)out_bytes);
  if (static_cast<uint64_t>(d->status_index) + ns > n_status)
    return dsr_fail(nullptr, DSR_ERR_INVALID, "statuses end at %llu > %llu entries",
                    (unsigned long long)(d->status_index + ns), (unsigned long long)n_status);
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
  uint64_t sp = 0, spill = 0;
  for (uint32_t k = 0; k < d->depth; ++k) {
    const uint64_t fp = pad16(d->frame_bytes[k]);
    if (sp + fp <= slab_bytes)
      sp += fp;
    else
      spill += fp;
  }
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

static int32_t set_smem_attr(dsr_ctx *ctx, uint32_t smem) {
  static const uint32_t kThreads[] = {128, 256, 512, 1024};
  for (uint32_t p = DSR_PROG_PAPER_SCALARS; p <= DSR_PROG_HETERO; ++p)
    for (uint32_t t : kThreads) {
      cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(plain_kernel_for(p, t)),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
      if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "cudaFuncSetAttribute");
    }
  return DSR_OK;
}

extern "C" int32_t dsr_stack_init(dsr_ctx *ctx, uint32_t smem_slab_bytes,
                                  uint64_t overflow_bytes_per_team, uint32_t max_teams,
                                  void *overflow_pool_dev, uint64_t pool_bytes) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
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
  int32_t rc = set_smem_attr(ctx, kCtrlBytes + smem_slab_bytes);
  if (rc != DSR_OK) return rc;
  rc = dsr_ctx_stack_changed(ctx, kCtrlBytes + smem_slab_bytes);
  if (rc != DSR_OK) return rc;
  ctx->slab_bytes = smem_slab_bytes;
  ctx->ovf_per_team = overflow_bytes_per_team;
  ctx->max_teams = overflow_bytes_per_team ? max_teams : 0xffffffffu;
  ctx->pool = static_cast<uint8_t *>(overflow_pool_dev);
  ctx->pool_bytes = pool_bytes;
  ctx->stack_ready = true;
  return DSR_OK;
}

// ---------------------------------------------------------------------------
// Plain launch
// ---------------------------------------------------------------------------
int32_t dsr_launch_plain(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                         void *out_dev, dsr_team_status *status_dev, cudaStream_t s) {
  KernelFn k = plain_kernel_for(d->program, d->threads);
  k<<<d->teams, d->threads, kCtrlBytes + ctx->slab_bytes, s>>>(
      *d, static_cast<const uint8_t *>(images_dev), static_cast<uint8_t *>(out_dev), status_dev,
      ctx->pool, ctx->ovf_per_team, ctx->slab_bytes, ctx->timeout_ns);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "plain launch");
  return DSR_OK;
}

static int32_t check_launch(dsr_ctx *ctx, const dsr_region_desc *d, const void *out_dev,
                            const void *status_dev) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!ctx->stack_ready) return dsr_fail(ctx, DSR_ERR_INVALID, "dsr_stack_init not called");
  const char *why;
  if (dsr_check_shape(d, &why) != DSR_OK) return dsr_fail(ctx, DSR_ERR_INVALID, "%s", why);
  if (!out_dev || !status_dev) return dsr_fail(ctx, DSR_ERR_INVALID, "null output or status");
  if (ctx->ovf_per_team && d->teams > ctx->max_teams)
    return dsr_fail(ctx, DSR_ERR_BUDGET, "%u teams exceed the %u overflow slabs", d->teams,
                    ctx->max_teams);
  return DSR_OK;
}

extern "C" int32_t dsr_launch_region(dsr_ctx *ctx, const dsr_region_desc *d,
                                     const void *images_dev, uint64_t image_bytes,
                                     void *out_dev, uint64_t out_bytes,
                                     dsr_team_status *status_dev, uint64_t n_status,
                                     void *stream) {
  int32_t rc = check_launch(ctx, d, out_dev, status_dev);
  if (rc != DSR_OK) return rc;
  if ((rc = dsr_validate_region(d, image_bytes, out_bytes, n_status)) != DSR_OK)
    return dsr_fail(ctx, rc, "%s", dsr_last_error_string(nullptr));
  uint64_t ib = 0;
  dsr_region_extent(d, &ib, nullptr, nullptr);
  if (ib && !images_dev) return dsr_fail(ctx, DSR_ERR_INVALID, "null images");
  return dsr_launch_plain(ctx, d, images_dev, out_dev, status_dev,
                          static_cast<cudaStream_t>(stream));
}

extern "C" int32_t dsr_run_region_host(dsr_ctx *ctx, const dsr_region_desc *d,
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
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return dsr_cuda_fail(ctx, e, "sync");
  return DSR_OK;
}
