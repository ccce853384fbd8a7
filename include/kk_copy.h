/*
 * kk_copy.h - C ABI of the result download helper (include kk_spgemm.h first).
 *
 * Not part of the paper's method: a serving utility for the end-to-end path.
 * kk_copy_to_host streams `bytes` bytes from device memory into page-locked
 * host memory with a kernel (the host buffer is written through its device
 * mapping, which unified addressing provides for memory from cudaHostAlloc or
 * cudaHostRegister).  The copy engines stay free for other transfers.  (The
 * library's own small read-backs, nnz(C) of a symbolic phase among them, are
 * written by a kernel through the same kind of mapping, so they do not queue
 * behind a large download on a copy engine either: a serving loop may download
 * C with cudaMemcpyAsync instead, which on a GB300 measured faster, 8.2 against
 * 10.6 ms per 27-point 100^3 step, the kernel competing with the product for
 * the SMs.)
 *
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream); the copy is
 * enqueued there and the call does not block.  dst_host: page-locked host
 * memory (else KK_ERR_INVALID_ARG); src_device: device memory.  Both 16-byte
 * aligned with bytes a multiple of 16 take the vectorised kernel; other
 * alignments are copied with cudaMemcpyAsync on the same stream.
 */
#ifndef KK_COPY_H_
#define KK_COPY_H_

#include "kk_spgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

kk_status kk_copy_to_host(void* cuda_stream, void* dst_host, const void* src_device, size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* KK_COPY_H_ */
