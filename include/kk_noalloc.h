/*
 * kk_noalloc.h - symbolic phase that allocates nothing (include kk_spgemm.h
 * first).
 *
 * The paper has no counterpart of this entry point.  It exists for callers
 * that cannot call cudaMalloc: a host application that owns all device memory
 * through its own pool allocator and forbids allocations behind its back, a
 * plug-in that runs inside such a framework, or a latency-critical loop in
 * which an allocation (and the device-wide synchronisation cudaMalloc and
 * cudaFree may bring) is not allowed.  The regular kk_spgemm_symbolic needs a
 * handle, and creating a handle and growing its scratch allocate device
 * memory.
 *
 * kk_spgemm_symbolic_noalloc computes the same row pointers and nnz(C) as
 * kk_spgemm_symbolic for C = A*B (same conventions: int32 A / B structure on
 * the device, int64 c_rowptr[m+1] caller-allocated on the device, nnz(C) to
 * the host) but keeps every temporary in fixed-size device memory that the
 * library reserves when it is loaded:
 *   - at most KK_NOALLOC_MAX_ROWS rows of A; larger A returns KK_ERR_CAPACITY
 *     and does nothing;
 *   - the reserved scratch (KK_NOALLOC_MAX_ROWS counts + block sums, about
 *     4.1 MB) stays allocated on every GPU that loads the library until the
 *     process exits;
 *   - the first call on a device looks up that scratch's device address (a
 *     host-side symbol lookup, no allocation) and caches it; make that first
 *     call before capturing any stream into a CUDA graph;
 *   - every call on a device shares the same scratch, which keeps the last
 *     call's contents: calls whose work overlaps on the GPU (different
 *     streams, or different host threads without ordering) race and give wrong
 *     results.  Issue them one after another.
 * The call is enqueued on cuda_stream (NULL = legacy default stream) and
 * blocks until nnz(C) is on the host.  Errors: KK_ERR_INVALID_ARG (NULL or
 * inconsistent arguments), KK_ERR_CAPACITY (too many rows), KK_ERR_BAD_INDEX
 * (A.rowptr[0] != 0, a row of A whose bounds are decreasing or outside A's
 * entries, a column of A outside B's rows, a referenced row of B whose bounds
 * are decreasing or outside B's entries, or a column of B outside [0, B.n)):
 * every row is checked before any of its indices is used to read memory, and a
 * bad row counts 0 -- c_rowptr is still written, but nnz_c is not set),
 * KK_ERR_CUDA.  It uses a slower counting scheme (one CTA per row, a bit vector
 * swept over the row's non-empty 32768-column windows) than the binned kernels
 * of kk_spgemm_symbolic.
 */
#ifndef KK_NOALLOC_H_
#define KK_NOALLOC_H_

#include "kk_spgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define KK_NOALLOC_MAX_ROWS (1 << 20)

kk_status kk_spgemm_symbolic_noalloc(const kk_csr* A, const kk_csr* B, int64_t* c_rowptr,
                                     int64_t* nnz_c, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KK_NOALLOC_H_ */
