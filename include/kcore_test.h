/*
 * kcore_test.h -- test hooks of libkcore (not for production use).
 *
 * Failure injection on the host, so that the library's error paths can be
 * exercised without faulting a GPU: the library makes every device
 * allocation through its per-device stream-ordered pool, and its page-locked
 * host buffers through one helper or the batch engine's staging pool; a hook
 * here makes one chosen allocation request fail as if memory had run out.
 * (The paper has no counterpart; failure handling is the library's own.)
 */
#ifndef KCORE_TEST_H
#define KCORE_TEST_H

#include <stdint.h>

#include "kcore.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Arm the injector: the k-th allocation request the library makes after this
 * call (device pool, page-locked host block or staging pool; counted across
 * all threads and devices, starting at 1) fails with out-of-memory, as the
 * CUDA call would; later requests succeed again.  k = 0 disarms.  Also resets
 * the counter read by kcore_test_alloc_count.  The entry point that made the
 * request returns KCORE_ERR_OOM and releases what it had taken; the batch
 * engine fails the admission batch that needed the memory and keeps running.
 * A failed staging-pool request is not an error: the engine then uses
 * pageable memory.
 */
void kcore_test_fail_alloc(int64_t k);

/* Allocation requests counted since the last kcore_test_fail_alloc call. */
int64_t kcore_test_alloc_count(void);

/*
 * Waits for all work on the current device (cudaDeviceSynchronize) and reads
 * the library pool's bytes in use and bytes reserved there
 * (cudaMemPoolAttrUsedMemCurrent / cudaMemPoolAttrReservedMemCurrent);
 * 0 and 0 before the pool's first use.  Errors: ERR_CUDA.
 */
kcore_status kcore_test_pool_usage(int64_t* used, int64_t* reserved);

#ifdef __cplusplus
}
#endif

#endif /* KCORE_TEST_H */
