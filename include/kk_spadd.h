/*
 * kk_spadd.h - C ABI of sparse matrix addition (include kk_spgemm.h first).
 *
 * Operation (Kokkos Kernels paper, Sec. "SpAdd"): C = alpha A + beta B, A, B
 * and C m-by-n in CSR (A, B: int32 row pointers and columns, float64 values;
 * C: int64 row pointers, int32 columns, float64 values).  Row i of C holds the
 * union of the columns of A(i,:) and B(i,:) in ascending order; entries of the
 * same row and column merge additively, also repeated columns within A or B;
 * the structure is structural (a sum that cancels keeps an explicit 0.0).
 * Input rows may be unsorted and may repeat columns.
 *
 * Two phases, as in the paper: the symbolic phase counts the entries of every
 * row of C and keeps, in the handle, the slot in C's row of every entry of A
 * and of B; the numeric phase scatters alpha a and beta b to those slots, for
 * any values of A and B on the same index arrays (symbolic reuse).
 *
 * kk_spadd_symbolic: A, B (values not read), c_rowptr device int64[m + 1]
 *   caller-allocated; *nnz_c (host) receives nnz(C).  Blocks until nnz(C) is on
 *   the host.  Errors: KK_ERR_INVALID_ARG (null arguments, shapes differ),
 *   KK_ERR_BAD_INDEX (a column outside [0, n)), KK_ERR_CAPACITY (a row of more
 *   than 8192 combined entries of A and B).
 * kk_spadd_numeric: the A and B index arrays of the last kk_spadd_symbolic
 *   call on this handle (else KK_ERR_STRUCTURE_MISMATCH; before any:
 *   KK_ERR_NOT_SYMBOLIC), their values, alpha and beta; c_colind int32[nnz(C)]
 *   and c_vals float64[nnz(C)] caller-allocated.  Asynchronous.  An entry of C
 *   with at most one contributing entry of A and one of B is exactly
 *   alpha a + beta b (each product rounded once, one rounded sum); repeated
 *   columns within A or B are added in no fixed order, within
 *   1e-12 * (sum |alpha a| + sum |beta b|).
 * The handle keeps int32 slots for nnz(A) + nnz(B) entries and int32 per row.
 */
#ifndef KK_SPADD_H_
#define KK_SPADD_H_

#include "kk_spgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

kk_status kk_spadd_symbolic(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B, int64_t* c_rowptr,
                            int64_t* nnz_c);
kk_status kk_spadd_numeric(kk_spgemm_handle h, double alpha, const kk_csr* A, double beta,
                           const kk_csr* B, const int64_t* c_rowptr, int32_t* c_colind, double* c_vals);

#ifdef __cplusplus
}
#endif

#endif /* KK_SPADD_H_ */
