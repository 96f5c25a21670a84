/*
 * dsr_device.cuh -- device API of the data-sharing runtime, for region
 * programs written by the user (compile with nvcc for sm_103a, -I include,
 * and link against libdsr).
 *
 * The paper's runtime interface (Sec. 4, Fig. "codegen-master" and
 * "codegen-worker"; Sec. 5.1-5.3) is what compiled OpenMP code calls in
 * generic mode: the team's master thread runs the target region's
 * sequential code, pushes the locals that a nested parallel region shares
 * onto a per-team stack in shared memory (global memory when they do not
 * fit), hands the workers references to them (prepare_parallel / the list
 * of shared-variable references), releases the workers at one barrier and
 * waits for them at another, and pops the locals when they go out of
 * scope. This header exposes those steps to hand-written programs:
 *
 *   master side (the team's sequential code)      worker side (a region)
 *   dsr_push(team, nbytes)   -> frame address     dsr_frame(level)
 *   dsr_fill(team, frame, src, nbytes)            dsr_frame_bytes(level)
 *   dsr_parallel(team, body, nthreads, arg)       dsr_thread_num(thr)
 *   dsr_fork(...) ... dsr_join(team)              dsr_num_threads(thr)
 *   dsr_pop(team, frame)                          dsr_team_num(thr)
 *   dsr_set_check(team, k, value)                 dsr_body(thr), dsr_arg(thr)
 *
 * A program is a struct:
 *
 *   struct MyProgram {
 *     static constexpr uint32_t kProgram = DSR_PROG_USER + 0;  // descriptor id
 *     // bytes of images and of output the region's descriptor indexes
 *     __host__ __device__ static void extent(const dsr_region_desc &d,
 *                                            uint64_t *image_bytes,
 *                                            uint64_t *out_bytes);
 *     __device__ static void master(dsr_team &team);     // sequential code
 *     __device__ static void body(const dsr_thread &thr);  // one thread of a
 *   };                                                      // parallel region
 *
 * Optionally, a plain launch's inputs can be pulled into L2 before the
 * kernel waits for the work queued ahead of it in the stream (programmatic
 * dependent launch lets its CTAs start while that work finishes):
 *
 *     __device__ static void prefetch(const dsr_region_desc &d,
 *                                     const uint8_t *images, uint32_t team);
 *
 * runs on one lane of each team's master warp before that wait and may only
 * call dsr_prefetch_l2 (hints that change no value a load returns): it must
 * not read or write global memory, since what the earlier work writes is
 * not visible yet.
 *
 * and is launched with dsr_launch_user_region<MyProgram> (one CTA per team,
 * one launch per region, Sec. 4), dsr_launch_user_batch<MyProgram> (many
 * region instances in one persistent launch) or served with
 * dsr_serve_user_start<MyProgram> (a device-resident server fed by
 * dsr_serve_submit), which instantiate the same kernels the built-in
 * programs run.
 *
 * Execution model.
 *  - master() runs on the 32 lanes of the team's master warp together (a
 *    warp set aside for the master thread as in Sec. 4, the CTA's last
 *    warp). Its
 *    control flow must be the same in all 32 lanes, and every dsr_* call on
 *    the master side is made by all 32 lanes at once. A statement that the
 *    paper's single master thread runs goes inside `if (dsr_is_master())`,
 *    followed by dsr_master_sync() before other lanes read what it wrote;
 *    order-free work over a frame may be split over the lanes (dsr_lane()).
 *  - body() runs once per thread tid < nthreads of each parallel region, on
 *    the team's worker threads; a region wider than the workers runs its
 *    threads round robin on them. Bodies must not synchronise with one
 *    another (no barrier inside a region); any order of a region's threads
 *    must give the same result.
 *  - A frame's address is the same in the master and the workers (a generic
 *    pointer to shared or global memory). Writes the master made before
 *    dsr_parallel / dsr_fork are visible to the workers of that region, and
 *    the workers' writes are visible to the master after dsr_parallel /
 *    dsr_join returns.
 *  - Errors never trap: a push that fits neither the shared-memory slab nor
 *    the team's overflow slab returns nullptr and sets DSR_ERR_OVERFLOW (the
 *    program must stop pushing and return); a pop of a frame that is not
 *    the top one sets DSR_ERR_LIFO. When master() returns, the frames it
 *    left are popped and the team's dsr_team_status record is written
 *    (status, depth left, peak stack bytes, peak overflow bytes, check
 *    words).
 */
#ifndef DSR_DEVICE_CUH_
#define DSR_DEVICE_CUH_

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "dsr.h"
#include "dsr_kernels.cuh"
#include "dsr_serve_kernel.cuh"

/* The master's handle on its team (master side only). */
struct dsr_team {
  const dsr::Env *e;
  dsr::Stack *s;
};

/* One thread of a parallel region (worker side). */
struct dsr_thread {
  const dsr::Env *e;
  uint32_t tid;       /* thread number in the region, 0 .. nthreads-1 */
  uint32_t nthreads;  /* threads of the region */
  uint32_t body;      /* the body id the master passed */
  uint32_t arg;       /* the argument the master passed */
};

/* ---- master side --------------------------------------------------------- */

/* Lane number in the master warp (0 = the master thread). */
__device__ __forceinline__ uint32_t dsr_lane() { return dsr::lane_id(); }

/* True in the master thread: lane 0 of the master warp (Sec. 4). */
__device__ __forceinline__ bool dsr_is_master() { return dsr::lane_id() == 0; }

/* Hint: pull [src, src + nbytes) of global memory into L2 (one bulk
 * prefetch per 64 KiB; src 16-byte aligned and nbytes a multiple of 16, else
 * nothing is done). No completion, no effect on any value a load returns. */
__device__ __forceinline__ void dsr_prefetch_l2(const void *src, uint32_t nbytes) {
  dsr::prefetch_l2(src, nbytes);
}

/* Orders the master warp's lanes: writes a lane made before it are visible
 * to the others after it. */
__device__ __forceinline__ void dsr_master_sync() { __syncwarp(); }

/* Push a frame of nbytes for the team's shared locals (Sec. 5.3: the shared
 * stack; Sec. 5.2: global memory when it does not fit). Reserved in 16-byte
 * units in the team's shared-memory slab if it fits there, else in its
 * global overflow slab; 16-byte aligned. Returns the frame's address (the
 * same in every lane), or nullptr with DSR_ERR_OVERFLOW when neither slab
 * has room or DSR_MAX_FRAMES frames are live. Contents are undefined until
 * the program writes them. */
__device__ __forceinline__ void *dsr_push(dsr_team &t, uint32_t nbytes) {
  return dsr::push(*t.s, nbytes);
}

/* Pop the top frame (Sec. 5.2: shared locals are released when their scope
 * ends, last in first out). `frame` must be the address the last live push
 * returned; otherwise nothing is popped and DSR_ERR_LIFO is set and
 * returned. */
__device__ __forceinline__ int32_t dsr_pop(dsr_team &t, void *frame) {
  const uint32_t depth = t.s->depth();
  if (depth == 0) {
    dsr::set_status(*t.s, DSR_ERR_LIFO);
    return DSR_ERR_LIFO;
  }
  __syncwarp();  // lane 0 wrote the frame table entry at the push
  const uint32_t bytes = dsr::ctrl()->frames[depth - 1].bytes;
  return dsr::pop(*t.s, static_cast<const uint8_t *>(frame), bytes);
}

/* Copy nbytes (a multiple of 4) from global memory at src into a frame the
 * team pushed: one bulk copy for a frame in the shared-memory slab (src
 * 16-byte aligned, nbytes a multiple of 16, at least 64), a copy split over
 * the workers for a large frame elsewhere (between two barriers, as a
 * runtime-owned step), else a copy by the master warp's lanes. A bulk copy
 * that does not complete within the ctx's wait timeout sets DSR_ERR_TIMEOUT.
 * Returns when the frame holds the data. */
__device__ __forceinline__ void dsr_fill(dsr_team &t, void *frame, const void *src,
                                         uint32_t nbytes) {
  uint8_t *f = static_cast<uint8_t *>(frame);
  dsr::fill<true>(*t.s, f, __isShared(f) != 0, static_cast<const uint8_t *>(src), nbytes, 0u);
}

/* Start parallel region `body` with nthreads threads (Sec. 4: the master
 * publishes the work and releases the workers at a named barrier; Fig.
 * "codegen-master"). `arg` reaches every thread (dsr_arg). The master may
 * do work of its own that touches no frame the region uses before
 * dsr_join. */
__device__ __forceinline__ void dsr_fork(dsr_team &t, uint32_t body, uint32_t nthreads,
                                         uint32_t arg) {
  dsr::fork<void>(*t.e, body, nthreads < 1u ? 1u : nthreads, arg);
}

/* Wait for the region started by dsr_fork (the join barrier). */
__device__ __forceinline__ void dsr_join(dsr_team &) { dsr::join(); }

/* dsr_fork then dsr_join: run a parallel region to completion. */
__device__ __forceinline__ void dsr_parallel(dsr_team &t, uint32_t body, uint32_t nthreads,
                                             uint32_t arg) {
  dsr_fork(t, body, nthreads, arg);
  dsr_join(t);
}

/* Record check word k < DSR_MAX_DEPTH (the same value in every lane) in the
 * team's status record. */
__device__ __forceinline__ void dsr_set_check(dsr_team &t, uint32_t k, uint32_t v) {
  dsr::set_chk(*t.s, k, v);
}

/* The team's status so far (DSR_OK until a push or pop fails). */
__device__ __forceinline__ int32_t dsr_get_status(const dsr_team &t) { return t.s->status(); }

/* Frames live on the team's stack. */
__device__ __forceinline__ uint32_t dsr_depth(const dsr_team &t) { return t.s->depth(); }

__device__ __forceinline__ const dsr_region_desc &dsr_desc(const dsr_team &t) { return *t.e->d; }
__device__ __forceinline__ uint32_t dsr_team_num(const dsr_team &t) { return t.e->team; }
__device__ __forceinline__ const uint8_t *dsr_images(const dsr_team &t) { return t.e->images; }
__device__ __forceinline__ uint8_t *dsr_out(const dsr_team &t) { return t.e->out; }

/* Threads of a region by default: the descriptor's width, or all workers
 * (threads - 32), or 1 for a team without workers (a team of one). */
__device__ __forceinline__ uint32_t dsr_region_width(const dsr_team &t) {
  return dsr::region_width(*t.e->d);
}

/* ---- both sides ---------------------------------------------------------- */

/* Address and size of live frame `level` (0 = the first pushed): the list of
 * references the master hands the workers (Sec. 5.1-5.2). */
__device__ __forceinline__ void *dsr_frame(uint32_t level) {
  return dsr::ctrl()->frames[level].ptr;
}
__device__ __forceinline__ uint32_t dsr_frame_bytes(uint32_t level) {
  return dsr::ctrl()->frames[level].bytes;
}

/* ---- worker side --------------------------------------------------------- */

__device__ __forceinline__ uint32_t dsr_thread_num(const dsr_thread &w) { return w.tid; }
__device__ __forceinline__ uint32_t dsr_num_threads(const dsr_thread &w) { return w.nthreads; }
__device__ __forceinline__ uint32_t dsr_team_num(const dsr_thread &w) { return w.e->team; }
__device__ __forceinline__ uint32_t dsr_body(const dsr_thread &w) { return w.body; }
__device__ __forceinline__ uint32_t dsr_arg(const dsr_thread &w) { return w.arg; }
__device__ __forceinline__ const dsr_region_desc &dsr_desc(const dsr_thread &w) { return *w.e->d; }
__device__ __forceinline__ const uint8_t *dsr_images(const dsr_thread &w) { return w.e->images; }
__device__ __forceinline__ uint8_t *dsr_out(const dsr_thread &w) { return w.e->out; }

/* ---- launching a user-written program ------------------------------------ */

namespace dsr {

// The program's optional prefetch, under the name the plain kernel looks for.
template <class U, class = void>
struct UserPrefetch {};
template <class U>
struct UserPrefetch<U, std::void_t<decltype(&U::prefetch)>> {
  __device__ static void prefetch_inputs(const Env &e) { U::prefetch(*e.d, e.images, e.team); }
};

// A user program seen through the interface the kernels call.
template <class U>
struct UserProgram : UserPrefetch<U> {
  static constexpr uint32_t kProgram = U::kProgram;
  static constexpr bool kDense = false;
  static constexpr bool kUser = true;
  DSR_HD static void extent(const dsr_region_desc &d, uint64_t *ib, uint64_t *ob) {
    U::extent(d, ib, ob);
  }
  __device__ static void master(const Env &e, Stack &s) {
    dsr_team t{&e, &s};
    U::master(t);
  }
  __device__ static void run(const Env &e, uint32_t work, uint32_t first, uint32_t W,
                             uint32_t n, uint32_t arg) {
    dsr_thread w{&e, first, n, work, arg};
    for (uint32_t v = first; v < n; v += W) {
      w.tid = v;
      U::body(w);
    }
  }
};

// The dynamic shared-memory limit of kernel k on `device`, raised to at
// least `smem` once (kept per kernel and device for the process).
inline cudaError_t ensure_smem_limit(const void *k, int device, uint32_t smem) {
  struct Entry {
    const void *k;
    int device;
    uint32_t smem;
  };
  static std::mutex mu;
  static std::vector<Entry> set;
  std::lock_guard<std::mutex> g(mu);
  for (Entry &x : set)
    if (x.k == k && x.device == device) {
      if (x.smem >= smem) return cudaSuccess;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem));
      if (e == cudaSuccess) x.smem = smem;
      return e;
    }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) set.push_back({k, device, smem});
  return e;
}

}  // namespace dsr

/* Launch one region instance of user program U (the plain form: d->teams
 * CTAs of d->threads threads on `stream`, one per team; Sec. 4). Arguments
 * and checks as dsr_launch_region, with the buffer extents U::extent
 * states; d->program must be U::kProgram (>= DSR_PROG_USER). Asynchronous;
 * the launch allows programmatic stream serialisation like the built-in
 * programs' (no thread touches global memory before the kernel ahead of it
 * in the stream has completed). Returns a dsr_status;
 * dsr_last_error_string(ctx) says why a launch was refused. */
template <class U>
int32_t dsr_launch_user_region(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                               uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                               dsr_team_status *status_dev, uint64_t n_status, void *stream) {
  static_assert(U::kProgram >= DSR_PROG_USER, "user programs take ids >= DSR_PROG_USER");
  using P = dsr::UserProgram<U>;
  uint64_t ib = 0, ob = 0;
  if (d && d->program == U::kProgram && dsr::shape_error(*d) == 0) U::extent(*d, &ib, &ob);
  if (d && d->program != U::kProgram)
    return dsr_report_error(ctx, DSR_ERR_INVALID, "descriptor names another program");
  dsr_plain_config cfg;
  int32_t rc = dsr_user_plain_config(ctx, d, ib, ob, image_bytes, out_bytes, n_status, out_dev,
                                     status_dev, &cfg);
  if (rc != DSR_OK) return rc;
  if (ib && !images_dev) return dsr_report_error(ctx, DSR_ERR_INVALID, "null images");
  const uint32_t block = d->threads > 32u ? d->threads : 64u;
  const dsr::PlainFn k = dsr::pick_plain<P>(block);
  cudaError_t e = dsr::ensure_smem_limit(reinterpret_cast<const void *>(k), cfg.device,
                                         cfg.ctrl_bytes + cfg.slab_bytes);
  if (e != cudaSuccess) return dsr_report_error(ctx, DSR_ERR_CUDA, cudaGetErrorString(e));
  // at most ceil(teams / SMs) CTAs per SM, as the library's plain launch
  const uint32_t smem = dsr::balanced_smem(reinterpret_cast<const void *>(k), block,
                                           cfg.ctrl_bytes + cfg.slab_bytes, d->teams, cfg.device,
                                           cfg.max_smem);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(d->teams);
  lc.blockDim = dim3(block);
  lc.dynamicSmemBytes = smem;
  lc.stream = static_cast<cudaStream_t>(stream);
  lc.attrs = attr;
  lc.numAttrs = 1;
  e = cudaLaunchKernelEx(&lc, k, *d, static_cast<const uint8_t *>(images_dev),
                         static_cast<uint8_t *>(out_dev), status_dev,
                         static_cast<uint8_t *>(cfg.pool_dev), cfg.ovf_per_team, cfg.slab_bytes,
                         cfg.timeout_ns);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_report_error(ctx, DSR_ERR_CUDA, cudaGetErrorString(e));
  return DSR_OK;
}

/* Run n region instances of user program U in one persistent launch (the
 * batched form): arguments, checks and workspace as dsr_launch_batch
 * (tuning NULL: 256 threads, 16 KiB slab), every descriptor checked on the
 * device against U::extent before its teams run. No graph is captured
 * here; the call only enqueues work on `stream`, so a caller may capture it
 * itself. Asynchronous. Returns a dsr_status. */
template <class U>
int32_t dsr_launch_user_batch(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                              uint64_t total_teams, const void *images_dev, uint64_t image_bytes,
                              void *out_dev, uint64_t out_bytes, dsr_team_status *status_dev,
                              uint64_t n_status, void *workspace_dev, uint64_t workspace_bytes,
                              const dsr_batch_tuning *tuning, void *stream) {
  static_assert(U::kProgram >= DSR_PROG_USER, "user programs take ids >= DSR_PROG_USER");
  using P = dsr::UserProgram<U>;
  dsr_batch_tuning t = {256, 16384, 0, 0};
  if (tuning) t = *tuning;
  // resident CTAs of this program's kernel in the tuning's shape (0 when
  // the shape is out of range: dsr_batch_prepare then says why)
  uint32_t per_sm = 0;
  const dsr::BatchFn k = dsr::pick_batch<P>(t.threads);
  const uint32_t smem = dsr::batch_smem(t.slab_bytes);
  int device = 0;
  if (t.threads >= 64 && t.threads <= DSR_MAX_THREADS && t.threads % 32 == 0 &&
      t.slab_bytes % 16 == 0 && cudaGetDevice(&device) == cudaSuccess &&
      dsr::ensure_smem_limit(reinterpret_cast<const void *>(k), device, smem) == cudaSuccess) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<const void *>(k),
                                                      static_cast<int>(t.threads),
                                                      smem) == cudaSuccess && occ > 0)
      per_sm = t.ctas_per_sm && t.ctas_per_sm < static_cast<uint32_t>(occ)
                   ? t.ctas_per_sm
                   : static_cast<uint32_t>(occ);
  }
  cudaGetLastError();  // a refused attribute is reported through the plan below
  dsr_batch_plan plan;
  int32_t rc = dsr_batch_prepare(ctx, descs_dev, n, U::kProgram, total_teams, images_dev,
                                 image_bytes, out_dev, out_bytes, status_dev, n_status,
                                 workspace_dev, workspace_bytes, t.threads, t.slab_bytes, per_sm,
                                 stream, &plan);
  if (rc != DSR_OK) return rc;
  k<<<plan.grid, plan.threads, dsr::batch_smem(plan.slab_bytes),
      static_cast<cudaStream_t>(stream)>>>(plan);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return dsr_report_error(ctx, DSR_ERR_CUDA, cudaGetErrorString(e));
  return DSR_OK;
}

namespace dsr {

// The hooks through which the library's served form runs user program U:
// the descriptor check, the kernel's attributes and occupancy, and the
// server launch, all in the user's translation unit.
template <class U>
struct UserServer {
  using P = UserProgram<U>;
  static int32_t validate(const dsr_region_desc *d, uint64_t image_bytes, uint64_t out_bytes,
                          uint64_t n_status) {
    return d && program_fits<P>(*d, image_bytes, out_bytes, n_status) ? DSR_OK : DSR_ERR_INVALID;
  }
  static int32_t prepare(uint32_t threads, uint32_t smem_bytes, int32_t *ctas_per_sm) {
    *ctas_per_sm = 0;
    const void *k = reinterpret_cast<const void *>(pick_serve<P>(threads));
    int device = 0, occ = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        ensure_smem_limit(k, device, smem_bytes) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, static_cast<int>(threads),
                                                      smem_bytes) != cudaSuccess)
      return DSR_ERR_CUDA;
    *ctas_per_sm = occ;
    return DSR_OK;
  }
  static int32_t launch(const void *args, uint32_t grid, uint32_t threads, uint32_t smem_bytes,
                        void *stream) {
    pick_serve<P>(threads)<<<grid, threads, smem_bytes, static_cast<cudaStream_t>(stream)>>>(
        *static_cast<const ServeArgs *>(args));
    // the library reads (and clears) the error itself
    return cudaPeekAtLastError() == cudaSuccess ? DSR_OK : DSR_ERR_CUDA;
  }
};

}  // namespace dsr

/* Serve user program U: dsr_serve_start_user with U's hooks (its descriptor
 * check by U::extent, its server kernel instantiated here; the table is
 * dsr_serve_user_program<U>(), static, valid for the process). cfg->program
 * must be U::kProgram. Requests then go through dsr_serve_submit /
 * dsr_serve_poll / dsr_serve_stop like a built-in program's. */
template <class U>
const dsr_serve_program *dsr_serve_user_program() {
  static_assert(U::kProgram >= DSR_PROG_USER, "user programs take ids >= DSR_PROG_USER");
  static const dsr_serve_program prog = {U::kProgram, 0u, &dsr::UserServer<U>::validate,
                                         &dsr::UserServer<U>::prepare,
                                         &dsr::UserServer<U>::launch};
  return &prog;
}

template <class U>
int32_t dsr_serve_user_start(dsr_ctx *ctx, const dsr_serve_cfg *cfg, void *workspace_dev,
                             uint64_t workspace_bytes) {
  return dsr_serve_start_user(ctx, cfg, workspace_dev, workspace_bytes,
                              dsr_serve_user_program<U>());
}

#endif /* DSR_DEVICE_CUH_ */
