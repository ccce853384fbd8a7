/*
 * kk_batched.h - C ABI of the batched form: many independent products
 * C_k = A_k * B_k (k = 0 .. count-1) in one call per phase (include
 * kk_spgemm.h first).
 *
 * The Kokkos Kernels paper runs many small dense problems inside one parallel
 * launch (Sec. "Dense Linear Algebra", batched BLAS: one launch over a batch,
 * team-level routines per problem).  The batched form applies that to the
 * two-phase SpGEMM of Sec. "Standard SpGEMM Kernel": the rows of all products
 * form one global row space R = sum_k A_k.m (pair k owns global rows
 * [R_k, R_k + A_k.m)); rows are binned by their flop bound (symbolic) and
 * nnz (numeric) across the whole batch, and one persistent kernel per phase
 * drains a work queue of (bin, row tile) items, each row using the accumulator
 * its bin calls for (warp hash set / map, or CTA hash set / map).
 *
 * Output layout: one row-pointer array for the whole batch, int64[R + 1],
 * holding absolute positions into one column array and one value array of
 * total_nnz entries.  Row pointers of C_k are c_rowptr[R_k .. R_k + A_k.m];
 * c_rowptr[R_k] is the batch base of C_k.
 *
 * Two execution modes (options.batched_mode):
 *   1 - persistent: the work-queue kernels above.  With options.batched_graph
 *       = 1 and a non-default stream, each phase is captured into a CUDA graph
 *       on its first call and replayed by later calls with the same pairs
 *       (same pointers and sizes).  A batch with a row beyond the batched
 *       accumulators (a flop bound or an nnz(C(i,:)) above the largest
 *       persistent bin) is handed whole to the packed form below, inside the
 *       same symbolic call (its numeric calls follow); such a batch is then
 *       not captured.
 *   2 - packed (and 0, the default): the batch becomes one block-diagonal
 *       product diag(A_k) * diag(B_k) in handle scratch (A's columns shifted to
 *       the packed rows of B_k, B's columns kept local, so C's rows come out in
 *       pair order with local columns) and runs through the plain two-phase
 *       kernels, rows of all pairs binned together across every tier (thread,
 *       window with kept structure, warp hash, wide); no capacity limits, no
 *       graph capture (the symbolic phase reads its bin sizes on the host).
 *       Needs the sums of A_k.nnz, B_k.nnz and B_k.m below 2^31.
 */
#ifndef KK_BATCHED_H_
#define KK_BATCHED_H_

#include "kk_spgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Batched symbolic phase.  A and B are HOST arrays of `count` device CSR
 * descriptors; A[k].n must equal B[k].m.  c_rowptr is a caller-allocated
 * device int64[R + 1].  c_offsets (host int64[count + 1], may be NULL)
 * receives the base of every C_k and the total; *total_nnz (host) the total.
 * Blocks until the total is on the host. */
kk_status kk_spgemm_batched_symbolic(kk_spgemm_handle h, int32_t count, const kk_csr* A,
                                     const kk_csr* B, int64_t* c_rowptr, int64_t* c_offsets,
                                     int64_t* total_nnz);

/* Batched numeric phase for the pairs of the last batched symbolic call
 * (values may differ, patterns may not).  c_colind (int32[total]) and c_vals
 * (float64[total]) are caller-allocated device arrays.  Asynchronous. */
kk_status kk_spgemm_batched_numeric(kk_spgemm_handle h, int32_t count, const kk_csr* A,
                                    const kk_csr* B, const int64_t* c_rowptr, int32_t* c_colind,
                                    double* c_vals);

#ifdef __cplusplus
}
#endif

#endif /* KK_BATCHED_H_ */
