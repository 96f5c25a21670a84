// dsr_ctx.h -- the context object behind the C ABI's opaque dsr_ctx
// (internal to the library).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "dsr.h"

struct dsr_batch_state;
struct dsr_serve_state;

struct dsr_ctx {
  int device = 0;
  int sm_count = 0;
  int max_smem_optin = 0;
  uint64_t timeout_ns = 1000000000ull;
  // stacks (dsr_stack_init)
  bool stack_ready = false;
  uint32_t slab_bytes = 0;  // with slab_auto: the cap (what a CTA can hold)
  bool slab_auto = false;   // each plain launch sizes its slab to its region
  uint64_t ovf_per_team = 0;
  uint32_t max_teams = 0;
  uint8_t *pool = nullptr;
  uint64_t pool_bytes = 0;
  uint64_t stack_gen = 0;   // dsr_stack_init calls that succeeded (launch graphs keep theirs)
  // launch forms
  dsr_batch_state *batch = nullptr;
  dsr_serve_state *serve = nullptr;
  std::string err;
};

// Record an error on ctx (and process-wide); returns `code`.
int32_t dsr_fail(dsr_ctx *ctx, int32_t code, const char *fmt, ...);
int32_t dsr_cuda_fail(dsr_ctx *ctx, cudaError_t e, const char *what);
// DSR_OK when the calling thread's current device is the ctx's; otherwise
// DSR_ERR_INVALID (a launch would run on another GPU than the ctx's pool).
int32_t dsr_check_device(dsr_ctx *ctx);
// Descriptor shape checks shared by every launch form.
int32_t dsr_check_shape(const dsr_region_desc *d, const char **why);
// Slab of a plain launch of *d: the configured slab, or with DSR_SLAB_AUTO
// the region's footprint slab capped at what a CTA can hold.
uint32_t dsr_plain_slab(const dsr_ctx *ctx, const dsr_region_desc *d);
// The checks dsr_launch_region makes before it launches.
int32_t dsr_check_region_launch(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                                uint64_t image_bytes, const void *out_dev, uint64_t out_bytes,
                                const void *status_dev, uint64_t n_status);
// Dynamic shared memory of the plain launch of *d (slab, control block and
// the balanced-residency padding); fills the host-side caches the launch reads.
uint32_t dsr_plain_launch_smem(dsr_ctx *ctx, const dsr_region_desc *d);
// The plain launch itself (arguments already checked).
int32_t dsr_launch_plain(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                         void *out_dev, dsr_team_status *status_dev, cudaStream_t s);
// Hooks of the batched / served forms into the context's lifecycle.
void dsr_ctx_release(dsr_ctx *ctx);
void dsr_serve_release(dsr_ctx *ctx);
int32_t dsr_ctx_stack_changed(dsr_ctx *ctx, uint32_t smem_per_team);
