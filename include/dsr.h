/*
 * dsr.h -- C ABI of the GB300 data-sharing runtime for OpenMP-style
 * generic-mode target regions.
 *
 * The method (Bercea et al., "Implementing implicit OpenMP data sharing on
 * GPUs", LLVM-HPC'17): in generic mode one master thread per team runs the
 * sequential code of a target region while the worker threads wait
 * (Sec. 4, Fig. "codegen-master" / "codegen-worker"); locals declared in
 * that code and referenced by a nested parallel region are implicitly
 * shared (Sec. 3.2). They live on a per-team stack in shared memory
 * (Sec. 5.3, "Shared memory stack"), the master passes the workers
 * references to them (Sec. 5.1-5.2), and a global-memory fallback catches
 * what does not fit (Sec. 5.2, last paragraph; Sec. 7).
 *
 * This library implements that runtime on sm_103a: a per-team frame stack
 * in a shared-memory slab spilling to per-team global overflow slabs, a
 * master/worker state machine with named-barrier handoff, frame-address
 * publication and a region-body executor. It runs built-in region programs
 * (DSR_PROG_*), each a fixed master code + parallel bodies.
 *
 * Conventions for every entry point:
 *  - Return value: a dsr_status (DSR_OK = 0). Failures never abort the
 *    process; dsr_last_error_string() describes the last failure of a ctx.
 *  - Pointers named *_dev are device pointers (e.g. a torch tensor's
 *    data_ptr) owned by the caller; the library never frees them. Pointers
 *    named *_host are host pointers owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (0 = legacy default stream);
 *    launches are asynchronous on it unless stated otherwise.
 *  - Device-side errors (stack overflow, LIFO misuse) are written to the
 *    per-team dsr_team_status records; the host reads them after a sync.
 *    No kernel traps.
 *  - A dsr_ctx is not thread-safe: calls on one ctx must not overlap (use
 *    one ctx per host thread). The host-side checks that take no ctx
 *    (dsr_validate_region, dsr_region_extent, dsr_region_footprint,
 *    dsr_footprint_model, dsr_batch_workspace_bytes) may be called from
 *    any thread.
 */
#ifndef DSR_H_
#define DSR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSR_MAX_DEPTH 4      /* frame sizes one region descriptor carries */
#define DSR_MAX_FRAMES 8     /* frame-table entries per team stack */
#define DSR_MAX_THREADS 1024 /* threads per team, master warp included */
#define DSR_PENDING (-1)     /* dsr_serve_poll: the request has not completed */
#define DSR_SLAB_AUTO 0xFFFFFFFFu /* dsr_stack_init: size each plain launch's slab */

typedef enum dsr_status {
  DSR_OK = 0,
  DSR_ERR_INVALID = 1,  /* malformed argument or descriptor */
  DSR_ERR_OVERFLOW = 2, /* a push did not fit in slab + overflow slab */
  DSR_ERR_LIFO = 3,     /* a pop named a frame that is not the top one */
  DSR_ERR_BUDGET = 4,   /* not enough pool / queue space for the request */
  DSR_ERR_TIMEOUT = 5,  /* a bounded wait ran out (on the device, or a server's drain) */
  DSR_ERR_CUDA = 6      /* a CUDA runtime call failed */
} dsr_status;

/* Built-in region programs (the master code and parallel bodies each one
 * runs are stated beside each id). W = threads - 32 workers; a region runs
 * `width` threads (0 = all W; a team with W == 0 runs each region with one
 * thread, a team of one). */
enum {
  /* Sec. 6.1, Fig. "Implicitly sharing 8 variables": shares param ints and
   * the array reference; a[team*width + tid] += sum of the ints (c_i = i). */
  DSR_PROG_PAPER_SCALARS = 1,
  /* Sec. 6.1, Fig. "Implicitly sharing an array": shares param int[width]
   * arrays filled with 10; a[team*width + tid] += sum_m d_m[tid]. */
  DSR_PROG_PAPER_ARRAYS = 2,
  /* param sequential regions per team, each pushing int32 s[4] from the
   * image; out[(r*teams + team)*width + tid] =
   *   (s0*tid + s1) ^ ((s2 >> (tid & 7)) + s3). */
  DSR_PROG_SCALARS = 3,
  /* depth nested master-side calls, each pushing {int32 s[16]; int32
   * arr[256]} (1088 B) from a per-(team, level) image; the innermost level
   * writes param int32 per team; chk[k] = the word the master summed after
   * level k's join. */
  DSR_PROG_NESTED = 4,
  /* one frame of float[frame_bytes/4] from a per-team image; out[team*width
   * + tid] = fp32 sum, in index order, of the elements tid, tid+width, ... */
  DSR_PROG_SWEEP = 5,
  /* heterogeneous instances: depth levels of int32[frame_bytes[k]/4] from
   * per-instance images; innermost out[team*width + tid] = hash-sum of the
   * worker's strided elements of every live frame. */
  DSR_PROG_HETERO = 6,
  /* sharing at worker level (Sec. 7, future work: the all-to-all pattern
   * and a runtime-managed global stack): depth 2, frame_bytes = {16, S},
   * threads >= 64. The master pushes int32 s[4] from the team's image; in
   * the parallel region every worker t < width pushes its own frame G_t =
   * int32[S/4] (image words ^ mix32(s0 + t)) on a stack of its warp, and
   * runs a nested parallel region on its warp's 32 lanes, which get the
   * frame's address by shuffle: G_t[w] = mix32(G_t[w] + s1 + w); then
   * out[team*width + t] = (sum G_t) ^ s2. The warp stacks share out what
   * the team's slab and overflow slab have left, evenly over the W/32
   * worker warps; a worker frame that fits neither share gives OVERFLOW.
   * chk[0] = sum of the team's outputs. param 0: the nested teams get their
   * workers' keys and frame offsets by warp shuffles; param 1: from a
   * per-warp table in shared memory (the same results; the two ways of
   * sharing within a warp, side by side). Plain launch only. */
  DSR_PROG_WORKERS = 7,
  /* First id of user-written programs: a program written against the device
   * API of dsr_device.cuh and launched through its launch templates carries
   * an id >= DSR_PROG_USER in its descriptors. The library checks such a
   * descriptor's shape (teams, threads, depth, frame sizes, alignment) and
   * the buffer extents the program states; the frames and bodies are the
   * program's own. */
  DSR_PROG_USER = 256
};

/* One region instance: a target region with `teams` teams (one CTA each in
 * the plain launch), Sec. 4 and Sec. 6.1. 64 bytes, little-endian. */
typedef struct dsr_region_desc {
  uint32_t program;                    /* DSR_PROG_* */
  uint32_t teams;                      /* >= 1 */
  uint32_t threads;                    /* per team, multiple of 32 in [32, 1024] */
  uint32_t depth;                      /* frames pushed per team, 1..DSR_MAX_DEPTH */
  uint32_t frame_bytes[DSR_MAX_DEPTH]; /* size of frame k, multiple of 4 */
  uint32_t width;                      /* threads per parallel region, 0 = all */
  uint32_t param;                      /* program parameter (see DSR_PROG_*) */
  uint32_t salt;                       /* per-instance salt (DSR_PROG_HETERO) */
  uint32_t status_index;               /* team 0's entry in the status array */
  uint64_t image_offset;               /* byte offset of the images, 16-aligned */
  uint64_t out_offset;                 /* byte offset of the output, 16-aligned */
} dsr_region_desc;

/* What each team reports when it ends (32 bytes). */
typedef struct dsr_team_status {
  int32_t status;              /* DSR_OK, DSR_ERR_OVERFLOW or DSR_ERR_LIFO */
  uint32_t depth_final;        /* live frames at team exit: 0 when balanced */
  uint32_t hwm_bytes;          /* peak reserved stack bytes, slab + overflow */
  uint32_t spill_bytes;        /* peak reserved overflow-slab bytes */
  uint32_t chk[DSR_MAX_DEPTH]; /* program check words (worker->master writes) */
} dsr_team_status;

typedef struct dsr_config {
  int32_t device;           /* CUDA device ordinal */
  uint32_t flags;           /* reserved, 0 */
  uint64_t wait_timeout_ns; /* bound on every device-side wait; 0 = 1 s */
} dsr_config;

/* Shared-memory and occupancy figures of a team shape on this GPU, the
 * GB300 counterpart of the paper's per-team footprint (Sec. 6.2.1: stack +
 * reference list + thread-private state) and teams-per-SM arithmetic
 * (Sec. 6.2.2). */
typedef struct dsr_footprint {
  uint32_t smem_per_team;   /* dynamic smem: control block + frame slab */
  uint32_t ctrl_bytes;      /* control block: frame table, work, counters */
  uint32_t slab_bytes;      /* frame slab */
  uint32_t teams_per_sm;    /* resident teams per SM (model) */
  uint32_t limit;           /* 1 = threads, 2 = smem, 3 = registers, 4 = blocks */
  uint32_t spill_bytes;     /* bytes per team that go to the overflow slab */
} dsr_footprint;

typedef struct dsr_ctx dsr_ctx;

/* ---- lifecycle ---------------------------------------------------------- */

/* Create a context on cfg->device (NULL cfg: device 0, defaults). Allocates
 * only host metadata. *out receives the handle, owned by the caller and
 * released with dsr_destroy. Errors: DSR_ERR_INVALID (out == NULL),
 * DSR_ERR_CUDA (device not usable). */
int32_t dsr_create(dsr_ctx **out, const dsr_config *cfg);

/* Release a context and the CUDA graphs it captured. Caller-owned buffers
 * are untouched. NULL is accepted. */
int32_t dsr_destroy(dsr_ctx *ctx);

/* Text of the ctx's last failure ("" if none). Owned by the ctx; valid until
 * the next call on it. Accepts NULL (returns the process-wide last error). */
const char *dsr_last_error_string(const dsr_ctx *ctx);

/* Record a failure on ctx (its dsr_last_error_string becomes msg) and
 * return code. For code built on this library -- the launch templates of
 * dsr_device.cuh -- to report its own failures the way the library does.
 * ctx may be NULL (only the process-wide last error is set). */
int32_t dsr_report_error(dsr_ctx *ctx, int32_t code, const char *msg);

/* ---- stacks (Sec. 5.3 shared stack, Sec. 5.2 global fallback) ---------- */

/* Configure every team's stack: a shared-memory slab of smem_slab_bytes
 * (multiple of 16, at most what one CTA can hold next to the control
 * block; or DSR_SLAB_AUTO: every plain launch sizes its slab to the
 * region's dsr_region_footprint, capped at what a CTA can hold -- the
 * shared memory is then allocated per region from an estimate of its need
 * rather than preallocated, the paper's proposal of Sec. 7) and a global
 * overflow slab of overflow_bytes_per_team, carved for
 * team t at overflow_pool_dev + t * overflow_bytes_per_team. The pool is a
 * caller-owned device buffer of pool_bytes (16-byte aligned) that the ctx
 * borrows; max_teams * overflow_bytes_per_team must fit in it. A push that
 * fits in neither slab fails with DSR_ERR_OVERFLOW in the team's status.
 * Errors: DSR_ERR_INVALID (sizes, alignment), DSR_ERR_BUDGET (pool too
 * small). */
int32_t dsr_stack_init(dsr_ctx *ctx, uint32_t smem_slab_bytes, uint64_t overflow_bytes_per_team,
                       uint32_t max_teams, void *overflow_pool_dev, uint64_t pool_bytes);

/* ---- host-side checks (no GPU needed) ---------------------------------- */

/* Check a descriptor: shape limits, the frame sizes its program requires,
 * 16-byte alignment of offsets, and that its images, outputs and statuses
 * fit in image_bytes, out_bytes and n_status. DSR_OK or DSR_ERR_INVALID. */
int32_t dsr_validate_region(const dsr_region_desc *d, uint64_t image_bytes, uint64_t out_bytes,
                            uint64_t n_status);

/* Bytes of input image, output and status entries a descriptor needs
 * (any pointer may be NULL). DSR_ERR_INVALID for a malformed descriptor. */
int32_t dsr_region_extent(const dsr_region_desc *d, uint64_t *image_bytes, uint64_t *out_bytes,
                          uint64_t *n_status);

/* Stack footprint of a region's teams, from its descriptor alone: the
 * bytes its stack holds at its deepest point (*stack_bytes, the hwm_bytes a
 * team reports when nothing spills) and the shared-memory slab that keeps
 * every frame out of the overflow slab under the runtime's placement
 * (*slab_bytes; for DSR_PROG_WORKERS the warp stacks' even shares make it
 * larger than the stack bytes when the region width is not a multiple of
 * 32). The estimate the paper proposes for sizing shared memory (Sec. 7).
 * Either pointer may be NULL. DSR_ERR_INVALID for a malformed descriptor. */
int32_t dsr_region_footprint(const dsr_region_desc *d, uint64_t *stack_bytes,
                             uint64_t *slab_bytes);

/* Footprint and occupancy model of a team shape (threads, frame sizes of
 * one descriptor, slab size) on a GB300-class SM: 228 KB shared memory per
 * SM with 1 KB reserved per CTA, 64 warps, 32 CTAs, 65536 registers; regs is
 * the kernel's registers per thread (0 = 64). No GPU is touched. */
int32_t dsr_footprint_model(const dsr_region_desc *d, uint32_t slab_bytes, uint32_t regs,
                            dsr_footprint *out);

/* What the plain launch of a descriptor gets on this GPU, measured from the
 * compiled kernel rather than modelled: the GB300 counterpart of the
 * paper's register counts and teams-per-SM columns (Sec. 6.2.2, Tables 2,
 * 2b, 5, 6), which the paper reads off the compiled kernel. */
typedef struct dsr_occupancy {
  uint32_t threads;         /* CTA threads of the launch (one extra warp when threads == 32) */
  uint32_t regs_per_thread; /* registers of the kernel the launch runs */
  uint32_t smem_per_team;   /* shared memory a team uses: control block + slab */
  uint32_t ctas_per_sm;     /* resident teams per SM as launched (the CUDA occupancy
                               calculator at the launch's dynamic shared memory, which
                               balanced residency may pad: see dsr_launch_region) */
  uint32_t sm_count;        /* SMs of the device */
  uint32_t spill_bytes;     /* bytes per team its frames put in the overflow slab */
} dsr_occupancy;

/* Occupancy of the plain launch of *d with the ctx's stack configuration
 * (dsr_stack_init). Queries the runtime only; launches nothing. Errors:
 * DSR_ERR_INVALID (bad descriptor, no stack configured), DSR_ERR_CUDA. */
int32_t dsr_region_occupancy(dsr_ctx *ctx, const dsr_region_desc *d, dsr_occupancy *out);

/* ---- plain launch: one CTA per team, one launch per region -------------- */

/* Launch one region instance (Sec. 4: the target region is one kernel
 * launch): d->teams CTAs of d->threads threads on `stream`, each with the
 * ctx's slab. images_dev (image_bytes long) and out_dev (out_bytes long)
 * are the buffers the descriptor's offsets index; status_dev holds n_status
 * records, of which teams d->status_index .. + d->teams - 1 are written.
 * The descriptor is checked against these sizes before anything launches.
 * Requires dsr_stack_init; d->teams <= the max_teams given there when an
 * overflow slab is configured. Asynchronous. The launch allows
 * programmatic stream serialisation: its CTAs may be placed while the kernel
 * before it in the stream drains, but none of its threads touches global
 * memory before that kernel has completed, so stream order holds for every
 * buffer. Balanced residency: when d->teams exceeds the SM count and
 * ceil(teams / SMs) CTAs per SM is below the kernel's occupancy, the launch
 * asks for enough dynamic shared memory (beyond the control block and slab
 * it uses) that no SM holds more than ceil(teams / SMs) of its teams, so
 * that no SM ends the launch later for holding more than its share.
 * Errors: DSR_ERR_INVALID, DSR_ERR_BUDGET, DSR_ERR_CUDA (launch failure). */
int32_t dsr_launch_region(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_dev,
                          uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                          dsr_team_status *status_dev, uint64_t n_status, void *stream);

/* The same region from host memory: copies image_bytes from images_host to
 * images_dev, launches, copies out_bytes of out_dev back to out_host and
 * the statuses to status_host, then synchronises `stream`. Host buffers
 * should be pinned for asynchronous copies. out_dev is first written from
 * out_host when the program updates its output in place (PAPER_*). */
int32_t dsr_run_region_host(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_host,
                            uint64_t image_bytes, void *out_host, uint64_t out_bytes,
                            dsr_team_status *status_host, void *images_dev, void *out_dev,
                            dsr_team_status *status_dev, void *stream);

/* dsr_run_region_host without the final synchronisation: the upload, the
 * launch and the downloads are enqueued on `stream` and the call returns.
 * The host buffers must be pinned (so the copies are asynchronous) and must
 * not be touched until the stream has passed the downloads. Steps enqueued
 * on two streams, each with its own device and host buffers, overlap one
 * step's download with the next step's upload and kernel. Same arguments
 * and errors as dsr_run_region_host, except that a failure of the copies
 * or the kernel surfaces at the caller's synchronisation. */
int32_t dsr_enqueue_region_host(dsr_ctx *ctx, const dsr_region_desc *d, const void *images_host,
                                uint64_t image_bytes, void *out_host, uint64_t out_bytes,
                                dsr_team_status *status_host, void *images_dev, void *out_dev,
                                dsr_team_status *status_dev, void *stream);

/* ---- launch graphs: repeated plain launches without a host call each ---- */

/* The buffers one region's descriptor offsets index (device memory,
 * caller-owned), as dsr_launch_region takes them. */
typedef struct dsr_region_buffers {
  const void *images_dev;
  uint64_t image_bytes;
  void *out_dev;
  uint64_t out_bytes;
  dsr_team_status *status_dev;
  uint64_t n_status;
} dsr_region_buffers;

/* An instantiated CUDA graph of plain region launches. */
typedef struct dsr_graph dsr_graph;

/* Capture n plain launches into a CUDA graph: launch i runs descs[i] on
 * bufs[i], checked as dsr_launch_region checks it, with the same
 * programmatic stream serialisation, so each launch of the graph depends on
 * the one before it as consecutive launches on a stream do (its CTAs may be
 * placed while that one drains; none touches global memory before it has
 * completed). Nothing runs until dsr_graph_launch. *out receives the graph
 * (caller-owned, dsr_graph_destroy). The graph keeps the ctx's stack
 * configuration of the capture (slab, overflow pool): a later dsr_stack_init
 * on ctx makes its replays refuse. Errors: those of dsr_launch_region for a
 * launch it would refuse (with the launch's index in the message; nothing
 * is kept), DSR_ERR_INVALID (null argument, n == 0), DSR_ERR_CUDA. */
int32_t dsr_graph_capture_regions(dsr_ctx *ctx, const dsr_region_desc *descs,
                                  const dsr_region_buffers *bufs, uint32_t n, dsr_graph **out);

/* Replay the graph's launches, in order, on `stream` (one host call for all
 * of them). Asynchronous. Errors: DSR_ERR_INVALID (null argument, another
 * ctx's or device's graph, or the stack configuration changed since the
 * capture), DSR_ERR_CUDA. */
int32_t dsr_graph_launch(dsr_ctx *ctx, dsr_graph *g, void *stream);

/* Free the graph; its replays must have completed. NULL is accepted. */
int32_t dsr_graph_destroy(dsr_graph *g);

/* ---- batched launch: many instances, one persistent kernel -------------- */

/* CTA shape of the persistent kernel. Teams of any width run on it: a region
 * wider than the CTA's workers runs its threads round robin on them. */
typedef struct dsr_batch_tuning {
  uint32_t threads;     /* CTA threads, multiple of 32 in [64, 1024] (32 are the master warp) */
  uint32_t slab_bytes;  /* shared-memory slab per CTA, multiple of 16 */
  uint32_t ctas_per_sm; /* resident CTAs per SM; 0 = as many as fit */
  uint32_t reserved;    /* 0 */
} dsr_batch_tuning;

/* Device workspace a batch of n instances with total_teams teams needs:
 * task cursors, cost-class counters and the (instance, team) task list.
 * Caller-owned, 16-byte aligned, reusable across launches of the batch. */
uint64_t dsr_batch_workspace_bytes(uint32_t n, uint64_t total_teams);

/* Host-side check of n host descriptors against the buffer sizes, and the
 * sum of their teams. DSR_ERR_INVALID names the first bad descriptor. */
int32_t dsr_batch_count(const dsr_region_desc *descs_host, uint32_t n, uint64_t image_bytes,
                        uint64_t out_bytes, uint64_t n_status, uint64_t *total_teams);

/* Run n region instances of one program (descs_dev: n descriptors in device
 * memory, 16-byte aligned) in one persistent launch on `stream`: a grid of
 * CTAs of tuning->threads threads with a slab of tuning->slab_bytes each
 * (NULL tuning: 256 threads, 16 KB), pulling (instance, team) tasks from a
 * cursor. This is the paper's fork/join runtime (Sec. 4, 5) run for many
 * target regions at once instead of one kernel launch per region. Every
 * descriptor is checked on the device before its teams run; a bad one (or
 * one of another program) gets DSR_ERR_INVALID in its statuses where those
 * are addressable, and is counted (dsr_batch_errors). total_teams must be
 * the instances' team sum; the workspace must hold
 * dsr_batch_workspace_bytes(n, total_teams). Overflow slabs come from the
 * ctx's pool, one per CTA (the grid is capped at the pool's max_teams).
 * use_graph != 0 captures the launch in a CUDA graph kept by the ctx
 * (keyed by all arguments) and replays it. Asynchronous. Errors:
 * DSR_ERR_INVALID, DSR_ERR_BUDGET (workspace too small), DSR_ERR_CUDA. */
int32_t dsr_launch_batch(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                         uint32_t program, uint64_t total_teams, const void *images_dev,
                         uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                         dsr_team_status *status_dev, uint64_t n_status, void *workspace_dev,
                         uint64_t workspace_bytes, const dsr_batch_tuning *tuning, void *stream,
                         int use_graph);

/* After a batch completed: tasks rejected on the device and tasks counted
 * by its scan (synchronises `stream`). */
int32_t dsr_batch_errors(dsr_ctx *ctx, const void *workspace_dev, uint32_t *errors,
                         uint64_t *tasks_counted, void *stream);

/* Ask the batch running on workspace_dev (NULL: the static workspace of
 * dsr_launch_batch_static on the ctx's device) to stop early: each of its
 * CTAs takes no further task after its next grab (a few tasks at most), so
 * a batch with a pathological instance can be drained without waiting out
 * every task. The flag is written by a host-to-device copy on a stream of
 * the ctx (a copy engine, since the persistent kernel holds every SM); the
 * call does not wait. It stops a batch that is running: a launch clears the
 * flag when its scan starts, so call it after the launch has begun (a batch
 * still queued behind other work may miss it). Teams that never ran keep
 * whatever their status words held; dsr_batch_progress says how many tasks
 * were taken. Errors: DSR_ERR_INVALID, DSR_ERR_CUDA. */
int32_t dsr_batch_abort(dsr_ctx *ctx, void *workspace_dev);

/* After a batch completed (synchronises `stream`): tasks its CTAs took (ran,
 * or rejected as invalid) and tasks its scan counted; fewer taken than
 * counted means the batch was stopped by dsr_batch_abort. workspace_dev
 * NULL: the static workspace. */
int32_t dsr_batch_progress(dsr_ctx *ctx, const void *workspace_dev, uint64_t *tasks_taken,
                           uint64_t *tasks_counted, void *stream);

/* Autotuner: runs the batch once per candidate CTA shape (64..512
 * threads) and slab size (2..32 KB), each at the most resident CTAs per SM
 * that fit, and returns the fastest in *best (and its time in *best_ms).
 * The outputs hold a correct result afterwards. Synchronises `stream`. The
 * paper sizes its shared stack statically (Sec. 5.3, Sec. 7); this picks
 * the slab from measured throughput instead. */
int32_t dsr_autotune(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                     uint32_t program, uint64_t total_teams, const void *images_dev,
                     uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                     dsr_team_status *status_dev, uint64_t n_status, void *workspace_dev,
                     uint64_t workspace_bytes, void *stream, dsr_batch_tuning *best,
                     float *best_ms);

/* One plain launch per region for n host descriptors: the per-region launch
 * baseline of the batched form. Same checks and errors as
 * dsr_launch_region. */
int32_t dsr_launch_regions(dsr_ctx *ctx, const dsr_region_desc *descs_host, uint32_t n,
                           const void *images_dev, uint64_t image_bytes, void *out_dev,
                           uint64_t out_bytes, dsr_team_status *status_dev, uint64_t n_status,
                           void *stream);

/* Batched launch that allocates nothing. The paper has no counterpart: it
 * is here for callers that cannot allocate device memory -- code on a path
 * where cudaMalloc/cudaFree are not allowed (they can synchronise the
 * whole device), or a plug-in whose host application owns all device
 * memory through its own allocator. The same run as dsr_launch_batch
 * (same arguments but no workspace and no graph flag), with its workspace
 * in a file-scope device array of dsr_batch_static_capacity() bytes (8 MiB:
 * about one million teams) that every GPU loading this library keeps until
 * the process exits. A batch whose workspace would be larger is refused
 * with DSR_ERR_BUDGET. The ctx's device must be the calling thread's
 * current device (else DSR_ERR_INVALID, nothing runs). The first call on a
 * device finds the array's device address (cudaGetSymbolAddress) and keeps
 * it for the process, and the first call on a ctx sets the kernels'
 * shared-memory limit; make the first call before any stream capture, and
 * do not use this entry point across a cudaDeviceReset. All calls share the
 * one array and leave its contents behind (each call re-initialises what it
 * reads), so calls whose launches overlap on the GPU -- on different
 * streams without ordering, or from different threads -- race and must not
 * be issued. Device-side rejections (including teams that total_teams left
 * no task slot for) are read with dsr_batch_static_errors. Overflow slabs
 * still come from the ctx's pool when dsr_stack_init configured one. */
int32_t dsr_launch_batch_static(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                                uint32_t program, uint64_t total_teams, const void *images_dev,
                                uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                                dsr_team_status *status_dev, uint64_t n_status,
                                const dsr_batch_tuning *tuning, void *stream);

/* Size in bytes of the fixed workspace dsr_launch_batch_static uses. */
uint64_t dsr_batch_static_capacity(void);

/* dsr_batch_errors for the last dsr_launch_batch_static on the ctx's device:
 * reads the fixed workspace's header (tasks rejected on the device, among
 * them teams that total_teams left no task slot for, and tasks counted by
 * its scan). Synchronises `stream`; the batch must have been enqueued on it
 * (or completed). Errors: DSR_ERR_INVALID (no static batch ran on this
 * device yet), DSR_ERR_CUDA. */
int32_t dsr_batch_static_errors(dsr_ctx *ctx, uint32_t *errors, uint64_t *tasks_counted,
                                void *stream);

/* ---- launches of user-written programs (dsr_device.cuh) ----------------- */

/* What a plain launch of a user-written program needs from the ctx: the
 * stack configuration of dsr_stack_init resolved for one region. Filled by
 * dsr_user_plain_config; the launch template of dsr_device.cuh passes it to
 * the plain kernel compiled in the user's translation unit. */
typedef struct dsr_plain_config {
  void *pool_dev;        /* overflow pool (team t's slab at + t * ovf_per_team) */
  uint64_t ovf_per_team; /* overflow-slab bytes per team, 0 = none */
  uint64_t timeout_ns;   /* bound of every device-side wait */
  uint32_t slab_bytes;   /* shared-memory slab of this launch */
  uint32_t ctrl_bytes;   /* control block in front of the slab */
  int32_t device;        /* the ctx's device */
  uint32_t max_smem;     /* dynamic shared memory a CTA may opt in to */
} dsr_plain_config;

/* Check a plain launch of a user-written program (d->program >=
 * DSR_PROG_USER) and resolve its stack configuration: the descriptor's
 * shape, image_need bytes of images from d->image_offset within image_bytes
 * and out_need bytes of output from d->out_offset within out_bytes (the
 * extents the program states), d->teams statuses from d->status_index within
 * n_status, non-null outputs, the ctx's device current on the calling thread
 * and d->teams within the overflow slabs of dsr_stack_init. The slab is the
 * ctx's (with DSR_SLAB_AUTO: the sum of the descriptor's 16-byte-rounded
 * frame sizes, capped). Launches nothing. Errors: DSR_ERR_INVALID,
 * DSR_ERR_BUDGET. */
int32_t dsr_user_plain_config(dsr_ctx *ctx, const dsr_region_desc *d, uint64_t image_need,
                              uint64_t out_need, uint64_t image_bytes, uint64_t out_bytes,
                              uint64_t n_status, const void *out_dev, const void *status_dev,
                              dsr_plain_config *cfg);

/* Arguments of the persistent batched kernel: filled by dsr_batch_prepare
 * and passed by value to the kernel (device pointers as void*). */
typedef struct dsr_batch_plan {
  const void *descs;    /* n descriptors (device) */
  const void *tasks;    /* (instance, team) task list in the workspace */
  void *hdr;            /* workspace header: cursors, counts, errors */
  const void *images;
  void *out;
  void *status;         /* dsr_team_status[n_status] */
  void *pool;           /* overflow pool, one slab per CTA */
  uint64_t capacity;    /* task slots (= total_teams) */
  uint64_t image_bytes;
  uint64_t out_bytes;
  uint64_t n_status;
  uint64_t ovf_per_cta;
  uint64_t timeout_ns;
  uint32_t n;           /* instances */
  uint32_t slab_bytes;  /* shared-memory slab per CTA */
  uint32_t grid;        /* CTAs of the persistent launch */
  uint32_t threads;     /* threads per CTA */
} dsr_batch_plan;

/* First half of a batched launch of program `program` (a built-in id or a
 * user-written one): checks the arguments as dsr_launch_batch does (with
 * the CTA shape `threads` x `slab_bytes`, and `ctas_per_sm` resident CTAs
 * per SM, which the caller computed for the kernel it will launch), then
 * enqueues on `stream` the scan of the instances' team counts and the
 * expansion of the (instance, team) task list into the workspace, and fills
 * *plan with the persistent kernel's grid and arguments. The caller then
 * launches the kernel on the same stream with dynamic shared memory
 * plan->slab_bytes plus the control block and the accumulator area
 * (dsr::batch_smem; the launch template of dsr_device.cuh does both).
 * Errors: as dsr_launch_batch. */
int32_t dsr_batch_prepare(dsr_ctx *ctx, const dsr_region_desc *descs_dev, uint32_t n,
                          uint32_t program, uint64_t total_teams, const void *images_dev,
                          uint64_t image_bytes, void *out_dev, uint64_t out_bytes,
                          dsr_team_status *status_dev, uint64_t n_status, void *workspace_dev,
                          uint64_t workspace_bytes, uint32_t threads, uint32_t slab_bytes,
                          uint32_t ctas_per_sm, void *stream, dsr_batch_plan *plan);

/* ---- served form: a device-resident request loop ------------------------ */

/* A server: one persistent kernel that keeps every CTA's stack live and runs
 * submitted region instances team by team as CTAs free up (continuous
 * batching). All requests share the buffers named here; each request's
 * descriptor offsets index them. */
typedef struct dsr_serve_cfg {
  uint32_t program;          /* DSR_PROG_SCALARS, _NESTED or _HETERO (a user id: dsr_serve_start_user) */
  uint32_t threads;          /* server CTA threads, multiple of 32 in [64, 1024] */
  uint32_t slab_bytes;       /* shared-memory slab per CTA, multiple of 16 */
  uint32_t ctas_per_sm;      /* 0 = as many as fit */
  uint32_t capacity;         /* requests in flight at most (ring slots), <= 2^24 */
  uint32_t reserved;         /* 0 */
  uint64_t idle_timeout_ns;  /* a CTA with no work for this long leaves; 0 = 2 s */
  const void *images_dev;
  uint64_t image_bytes;
  void *out_dev;
  uint64_t out_bytes;
  dsr_team_status *status_dev;
  uint64_t n_status;
} dsr_serve_cfg;

/* Device workspace of a server with `capacity` request slots. */
uint64_t dsr_serve_workspace_bytes(uint32_t capacity);

/* Start serving: allocates the pinned request and completion rings (host
 * memory mapped into the device, owned by the ctx) and launches the server
 * kernel on a ctx-owned stream. Overflow slabs come from the ctx's pool, one
 * per server CTA. Every device-side wait of the server is bounded; a server
 * idle for idle_timeout_ns exits and is started again by the next submit or
 * poll. Errors: DSR_ERR_INVALID, DSR_ERR_BUDGET (workspace), DSR_ERR_CUDA. */
int32_t dsr_serve_start(dsr_ctx *ctx, const dsr_serve_cfg *cfg, void *workspace_dev,
                        uint64_t workspace_bytes);

/* A user-written program's server (include/dsr_device.cuh,
 * dsr_serve_user_start, fills this in): the library runs the host side of
 * the served form and calls these hooks, which live in the user's
 * translation unit with the program's server kernel. */
typedef struct dsr_serve_program {
  uint32_t program;  /* the program's descriptor id, >= DSR_PROG_USER */
  uint32_t reserved; /* 0 */
  /* Host-side check of one request against the server's buffers: DSR_OK,
   * or DSR_ERR_INVALID when the descriptor is malformed or indexes past
   * image_bytes / out_bytes / n_status. */
  int32_t (*validate)(const dsr_region_desc *d, uint64_t image_bytes, uint64_t out_bytes,
                      uint64_t n_status);
  /* Set the server kernel's shared-memory limit for CTAs of `threads`
   * threads and `smem_bytes` of dynamic shared memory on the current
   * device, and give its resident CTAs per SM (0: the shape does not fit).
   * DSR_OK or DSR_ERR_CUDA. */
  int32_t (*prepare)(uint32_t threads, uint32_t smem_bytes, int32_t *ctas_per_sm);
  /* Launch the server kernel: `grid` CTAs of `threads` threads with
   * `smem_bytes` of dynamic shared memory on `stream`, its one argument the
   * block at `args` (the library's server arguments, the ServeArgs layout of
   * include/dsr_serve_kernel.cuh). DSR_OK or DSR_ERR_CUDA. */
  int32_t (*launch)(const void *args, uint32_t grid, uint32_t threads, uint32_t smem_bytes,
                    void *stream);
} dsr_serve_program;

/* dsr_serve_start for a user-written program: cfg->program must equal
 * prog->program (>= DSR_PROG_USER) and every hook must be set; the
 * program's own validate hook checks each submitted descriptor. Admission
 * counts a request's spill from its descriptor's depth and frame_bytes as
 * for the built-in programs. Everything else (rings, workspace, submit,
 * poll, stop, stats, bench) as dsr_serve_start. The hooks must stay valid
 * until the server is stopped and released (dsr_destroy). Errors as
 * dsr_serve_start. */
int32_t dsr_serve_start_user(dsr_ctx *ctx, const dsr_serve_cfg *cfg, void *workspace_dev,
                             uint64_t workspace_bytes, const dsr_serve_program *prog);

/* Submit one region instance (non-blocking). The descriptor is checked on
 * the host. Admission: the request needs a free ring slot and, for its
 * teams' frames that do not fit the server's slab, overflow bytes
 * (spill per team x min(teams, server CTAs)) within the pool; otherwise
 * DSR_ERR_BUDGET (try again after completions). A team that could never fit
 * slab + its CTA's overflow slab is refused with DSR_ERR_OVERFLOW.
 * *ticket receives the request's number. */
int32_t dsr_serve_submit(dsr_ctx *ctx, const dsr_region_desc *d, uint64_t *ticket);

/* Completion of a ticket: *status = DSR_PENDING, or the worst status of the
 * request's teams once it completed (reported once per ticket). */
int32_t dsr_serve_poll(dsr_ctx *ctx, uint64_t ticket, int32_t *status);

/* Drain and stop: the server finishes every submitted request and exits;
 * blocks until it has, for at most twice the idle timeout plus 30 s, after
 * which it returns DSR_ERR_TIMEOUT with the server still on the GPU. The
 * rings stay for a later dsr_serve_start. */
int32_t dsr_serve_stop(dsr_ctx *ctx);

/* Counters: requests submitted and completed, server CTAs that left on the
 * idle timeout, teams rejected on the device. */
int32_t dsr_serve_stats(dsr_ctx *ctx, uint64_t *submitted, uint64_t *completed,
                        uint32_t *idle_exits, uint32_t *errors);

/* Open-loop latency run on a started server: request i is submitted at
 * arrival_ns[i] (nanoseconds from a start 1 ms after the call; a full ring
 * delays submission), and latency_ns[i] = the time its completion was seen
 * minus arrival_ns[i] (negative: -2 - status for a failed request).
 * *elapsed_ns = start to last completion. Runs on the calling thread. */
int32_t dsr_serve_bench(dsr_ctx *ctx, const dsr_region_desc *descs, uint32_t n,
                        const int64_t *arrival_ns, int64_t *latency_ns, int64_t *elapsed_ns);

/* The same arrivals served by one plain launch per request on `stream`
 * (completion seen through an event per request): the per-region launch
 * baseline of the served form. The server must not be running. */
int32_t dsr_launch_bench(dsr_ctx *ctx, const dsr_region_desc *descs, uint32_t n,
                         const int64_t *arrival_ns, int64_t *latency_ns, int64_t *elapsed_ns,
                         const void *images_dev, uint64_t image_bytes, void *out_dev,
                         uint64_t out_bytes, dsr_team_status *status_dev, uint64_t n_status,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DSR_H_ */
