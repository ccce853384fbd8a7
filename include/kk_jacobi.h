/*
 * kk_jacobi.h - C ABI of the Jacobi-fused numeric phase (include kk_spgemm.h first).
 *
 * Operation (Kokkos Kernels paper, Sec. "Jacobi-Fused SpGEMM Kernel"):
 *     C = (I - omega D^-1 A) B,
 * A square m-by-m with every diagonal entry stored and nonzero, D = diag(A)
 * (D(i) = the sum of row i's stored (i,i) entries: repeats add, as everywhere),
 * B m-by-k, omega a scalar.  Row i is
 *     C(i,:) = B(i,:) + s_i * (A(i,:) B),   s_i = -omega / D(i),
 * computed without forming A*B or D^-1 A*B: s_i is computed once per row, folded
 * into the values of A's row (and 1 into its first diagonal entry) by one pass
 * over A's values, and the plain numeric kernels then produce C directly.
 * Because A(i,i) is stored, B(i,:) lies inside (A B)(i,:), so C has the
 * structure of A*B and the symbolic phase is the plain one (kk_spgemm_symbolic
 * on the same handle, A and B); structure reuse across calls works as for
 * kk_spgemm_numeric (new values of A or B, same patterns, any omega).
 *
 * Arguments: as kk_spgemm_numeric, plus omega (finite).  A->vals and B->vals
 * are read; c_colind / c_vals are caller-allocated device arrays of nnz(C).
 * Asynchronous like kk_spgemm_numeric; the handle keeps one float64 scratch
 * array of nnz(A) entries.
 *
 * Errors: KK_ERR_INVALID_ARG (returned) when A is not square, omega is not
 * finite or the arguments are null; a row of A without a stored diagonal entry
 * or whose diagonal sums to 0 sets KK_ERR_INVALID_ARG on the device, reported
 * at the next kk_spgemm_sync or blocking call (C's values are then undefined);
 * otherwise as kk_spgemm_numeric.
 *
 * Accuracy: each value within 1e-12 * (|s_i| sum_j |a_ij||b_jc| + |b_ic|) of
 * the exact result (the plain product's bound with A's values scaled by s_i).
 */
#ifndef KK_JACOBI_H_
#define KK_JACOBI_H_

#include "kk_spgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

kk_status kk_spgemm_jacobi_numeric(kk_spgemm_handle h, double omega, const kk_csr* A,
                                   const kk_csr* B, const int64_t* c_rowptr, int32_t* c_colind,
                                   double* c_vals);

#ifdef __cplusplus
}
#endif

#endif /* KK_JACOBI_H_ */
