/* dsr_diag.h -- self-checks of the device runtime's failure handling.
 *
 * The paper's only failure path is the global-memory fallback of the shared
 * stack (Sec. 5.2). The runtime adds one more rule of its own: every wait on
 * the device (fills completing on an mbarrier, the streamed fill's chunks,
 * the server's polling) gives up after the context's timeout and reports
 * DSR_ERR_TIMEOUT instead of spinning on. The checks below exercise that
 * rule on a wait that nothing completes, and the stack's error statuses on
 * pushes and pops misused on purpose, without faulting, trapping or hanging
 * the GPU.
 */
#ifndef DSR_DIAG_H
#define DSR_DIAG_H

#include <stdint.h>

#include "dsr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Launch one CTA whose first thread arms a shared-memory mbarrier for 16
 * bytes that no copy will deliver and waits on it with the runtime's own
 * bounded wait, limited to timeout_ns of %globaltimer. result_dev (device
 * memory, two uint64_t, caller-owned) receives { status, elapsed ns }: the
 * status is DSR_ERR_TIMEOUT when the wait gave up, as it must, and DSR_OK if
 * it completed. No copy is in flight when the kernel exits. timeout_ns must
 * be at most 10 s. Asynchronous on `stream`. Errors: DSR_ERR_INVALID (no
 * ctx, null result, timeout too long), DSR_ERR_CUDA (launch failure). */
int32_t dsr_check_bounded_wait(dsr_ctx *ctx, uint64_t timeout_ns, uint64_t *result_dev,
                               void *stream);

/* The team stack's push and pop (Sec. 5.2: frames allocated on the shared
 * stack, the global-memory fallback, release in LIFO order), misused on
 * purpose by one master warp with a 96-byte slab and a 64-byte overflow
 * slab (scratch_dev, caller-owned device memory of at least 64 bytes,
 * 16-byte aligned). result_dev (device memory, n_result >= 25 uint64_t)
 * receives, in order:
 *   team 1: pushes of 48, 40 and 64 bytes -> [0] first in the slab, [1]
 *     second in the slab, [2] third in the overflow slab, [3] slab bytes
 *     reserved (96), [4] overflow bytes reserved (64); a pop of the second
 *     frame, not the top -> [5] its status (DSR_ERR_LIFO), [6] depth (3),
 *     [7] slab bytes, [8] overflow bytes (nothing popped); the three pops in
 *     order -> [9..11] their statuses (DSR_OK), [12] depth (0), [13] slab
 *     bytes (0), [14] overflow bytes (0), [15] the team's status (the first
 *     error, DSR_ERR_LIFO), [16] peak bytes (160), [17] peak overflow bytes
 *     (64);
 *   team 2: pushes of 48, 48, 64 and 16 bytes -> [18] status
 *     (DSR_ERR_OVERFLOW), [19] the fourth push gave no frame (1), [20] depth
 *     (3); a pop of the top frame with a wrong size -> [21] DSR_ERR_LIFO;
 *   team 3: DSR_MAX_FRAMES + 1 pushes of 16 bytes -> [22] frames pushed
 *     (DSR_MAX_FRAMES), [23] status (DSR_ERR_OVERFLOW: the frame table is
 *     full), [24] depth (DSR_MAX_FRAMES).
 * Asynchronous on `stream`. Errors: DSR_ERR_INVALID (no ctx, short result or
 * scratch), DSR_ERR_CUDA (launch failure). */
int32_t dsr_check_stack(dsr_ctx *ctx, uint64_t *result_dev, uint32_t n_result,
                        void *scratch_dev, uint64_t scratch_bytes, void *stream);

/* Measured shared-memory bandwidth of this GPU: the roofline the runtime's
 * stack traffic (frames written and read in the shared-memory slab, Sec.
 * 5.3) is reported against. Every SM runs CTAs of 1024 threads (as many as
 * fit) that stream conflict-free 16-byte loads (ld.shared.v4, a warp
 * reading 512 consecutive bytes) from a 32 KiB buffer, `reps` rounds of 8
 * loads per thread; one warm-up launch, then one launch timed with CUDA
 * events on `stream`. scratch_dev: caller-owned device memory of 4
 * uint64_t. Synchronises `stream`. out receives the bytes loaded, the
 * event time, the bandwidth, and the SM clock during the timed launch (the
 * %clock64 cycles over the %globaltimer nanoseconds of its slowest CTA),
 * from which the bytes per SM per clock follow. Errors: DSR_ERR_INVALID
 * (null argument, reps 0 or above 2^20), DSR_ERR_CUDA. */
typedef struct dsr_smem_probe {
  uint64_t bytes;           /* shared-memory bytes loaded by the timed launch */
  double ms;                /* its duration between CUDA events */
  double gbs;               /* bytes / ms, all SMs */
  double sm_mhz;            /* SM clock during it */
  double bytes_per_clk_sm;  /* gbs / (SMs x SM clock) */
  uint32_t ctas;            /* CTAs of the launch */
  uint32_t threads;         /* threads per CTA */
} dsr_smem_probe;

int32_t dsr_probe_smem_bandwidth(dsr_ctx *ctx, uint32_t reps, uint64_t *scratch_dev,
                                 void *stream, dsr_smem_probe *out);

#ifdef __cplusplus
}
#endif

#endif /* DSR_DIAG_H */
