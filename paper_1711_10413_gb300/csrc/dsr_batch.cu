// dsr_batch.cu -- batched launch form (persistent kernel over many region
// instances) and the context hooks it needs.
#include <cuda_runtime.h>

#include "dsr.h"
#include "dsr_ctx.h"

struct dsr_batch_state {};

void dsr_ctx_release(dsr_ctx *ctx) {
  delete ctx->batch;
  ctx->batch = nullptr;
}

int32_t dsr_ctx_stack_changed(dsr_ctx *, uint32_t) { return DSR_OK; }
