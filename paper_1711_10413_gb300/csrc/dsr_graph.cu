// dsr_graph.cu -- launch graphs: a sequence of plain region launches
// captured once into a CUDA graph and replayed with one host call.
//
// The paper's runtime launches one kernel per target region (Sec. 4); a
// program that runs the same regions again and again (the same shapes on
// the same buffers, or on buffers it rotates through) pays the host's launch
// call each time. Captured, the launches keep their programmatic stream
// serialisation as graph edges, so each still waits for the one before it
// before it touches global memory, and the GPU takes the kernel nodes
// without a host call each.
#include <cuda_runtime.h>

#include <cstdint>

#include "dsr.h"
#include "dsr_ctx.h"

struct dsr_graph {
  cudaGraphExec_t exec = nullptr;
  const dsr_ctx *ctx = nullptr;
  int device = 0;
  uint64_t stack_gen = 0;  // the ctx's stack configuration at the capture
  uint32_t launches = 0;
};

extern "C" int32_t dsr_graph_capture_regions(dsr_ctx *ctx, const dsr_region_desc *descs,
                                             const dsr_region_buffers *bufs, uint32_t n,
                                             dsr_graph **out) {
  if (!ctx) return dsr_fail(nullptr, DSR_ERR_INVALID, "null ctx");
  if (!descs || !bufs || !out || n == 0)
    return dsr_fail(ctx, DSR_ERR_INVALID, "null argument or no launches");
  *out = nullptr;
  // every launch checked, and its shared-memory size resolved, before the
  // capture starts (nothing but launches is issued while capturing)
  for (uint32_t i = 0; i < n; ++i) {
    const dsr_region_buffers &b = bufs[i];
    const int32_t rc = dsr_check_region_launch(ctx, descs + i, b.images_dev, b.image_bytes,
                                               b.out_dev, b.out_bytes, b.status_dev, b.n_status);
    if (rc != DSR_OK)
      return dsr_fail(ctx, rc, "launch %u: %s", i, dsr_last_error_string(ctx));
    dsr_plain_launch_smem(ctx, descs + i);
  }
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "capture stream");
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  int32_t rc = DSR_OK;
  if (e == cudaSuccess) {
    for (uint32_t i = 0; i < n && rc == DSR_OK; ++i) {
      const dsr_region_buffers &b = bufs[i];
      rc = dsr_launch_plain(ctx, descs + i, b.images_dev, b.out_dev, b.status_dev, s);
    }
    // the capture ends whatever happened inside it
    const cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (rc == DSR_OK && e2 != cudaSuccess) e = e2;
  }
  cudaGraphExec_t exec = nullptr;
  if (rc == DSR_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s);
  if (rc != DSR_OK) return rc;
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "graph capture");
  dsr_graph *g = new dsr_graph();
  g->exec = exec;
  g->ctx = ctx;
  g->device = ctx->device;
  g->stack_gen = ctx->stack_gen;
  g->launches = n;
  *out = g;
  return DSR_OK;
}

extern "C" int32_t dsr_graph_launch(dsr_ctx *ctx, dsr_graph *g, void *stream) {
  if (!ctx || !g) return dsr_fail(ctx, DSR_ERR_INVALID, "null argument");
  if (g->ctx != ctx || g->device != ctx->device)
    return dsr_fail(ctx, DSR_ERR_INVALID, "the graph was captured for another ctx");
  if (g->stack_gen != ctx->stack_gen)
    return dsr_fail(ctx, DSR_ERR_INVALID,
                    "the stack configuration changed since the capture (dsr_stack_init)");
  if (int32_t rc = dsr_check_device(ctx)) return rc;
  const cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return dsr_cuda_fail(ctx, e, "graph launch");
  return DSR_OK;
}

extern "C" int32_t dsr_graph_destroy(dsr_graph *g) {
  if (!g) return DSR_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  delete g;
  return DSR_OK;
}
