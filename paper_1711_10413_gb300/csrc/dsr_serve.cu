// dsr_serve.cu -- served launch form (device-resident request loop).
#include <cuda_runtime.h>

#include "dsr.h"
#include "dsr_ctx.h"

struct dsr_serve_state {};

void dsr_serve_release(dsr_ctx *ctx) {
  delete ctx->serve;
  ctx->serve = nullptr;
}
