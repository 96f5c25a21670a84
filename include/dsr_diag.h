/* dsr_diag.h -- self-checks of the device runtime's failure handling.
 *
 * The paper's only failure path is the global-memory fallback of the shared
 * stack (Sec. 5.2). The runtime adds one more rule of its own: every wait on
 * the device (fills completing on an mbarrier, the streamed fill's chunks,
 * the server's polling) gives up after the context's timeout and reports
 * DSR_ERR_TIMEOUT instead of spinning on. The check below exercises that
 * rule on a wait that nothing completes, without faulting, trapping or
 * hanging the GPU.
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

#ifdef __cplusplus
}
#endif

#endif /* DSR_DIAG_H */
