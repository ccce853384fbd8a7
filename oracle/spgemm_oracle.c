/*
 * CPU oracle for two-phase SpGEMM, C = A*B on CSR.  TEST INFRASTRUCTURE ONLY:
 * nothing on the product path may call, link or load this file; only tests/,
 * the smoke check in __graft_entry__.py and the cpu_baseline leg of bench.py do.
 *
 * What it computes (Kokkos Kernels paper, Sec. "Standard SpGEMM Kernel", Eq. 1):
 *     C(i,:) = sum_{j in A(i,:)} A(i,j) * B(j,:)
 * written out as plain, single-threaded Gustavson (row by row over A), split into
 * the two phases the same section describes:
 *   - symbolic: the number of nonzeros of every row of C (structural count);
 *   - numeric:  the column indices and values of those nonzeros.
 * A dense marker array of length k plays the role of the dense accumulator the
 * section describes (a bit vector for symbolic, a scalar array for numeric).
 *
 * Readings of points the paper leaves open (each repeated in the design notes):
 *   - structure is structural: an entry whose contributions cancel to 0.0 stays;
 *   - each row of C is emitted with its columns in ascending order;
 *   - duplicated or unsorted columns in A or B are allowed and merge additively;
 *   - summation order: contributions to C(i,c) are taken in the stored order of
 *     A(i,:), then of B(j,:); the first is v = a*b, every later one v = fma(a,b,v).
 *     Build with -ffp-contract=off so the compiler cannot fuse the first product.
 *
 * Indices are 0-based.  Row pointers of A and B are int32, of C int64.
 * Every entry point works on a row range [r0, r1) of A/C so that large products
 * can be checked block by block.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/* Symbolic phase for rows [r0, r1): counts[i - r0] = nnz(C(i,:)).
 * Returns 0 on success, -1 if scratch allocation fails. */
int oracle_symbolic_rows(int32_t r0, int32_t r1, int32_t k,
                         const int32_t* a_rowptr, const int32_t* a_colind,
                         const int32_t* b_rowptr, const int32_t* b_colind,
                         int64_t* counts) {
  int64_t* marker = (int64_t*)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
  if (!marker) return -1;
  for (int32_t c = 0; c < k; ++c) marker[c] = -1;
  for (int32_t i = r0; i < r1; ++i) {
    int64_t cnt = 0;
    for (int32_t p = a_rowptr[i]; p < a_rowptr[i + 1]; ++p) {
      int32_t j = a_colind[p];
      for (int32_t q = b_rowptr[j]; q < b_rowptr[j + 1]; ++q) {
        int32_t c = b_colind[q];
        if (marker[c] != i) { marker[c] = i; ++cnt; }
      }
    }
    counts[i - r0] = cnt;
  }
  free(marker);
  return 0;
}

/* Numeric phase for rows [r0, r1).  offsets[i - r0] .. offsets[i - r0 + 1] is the
 * slice of colind/vals that receives row i (offsets relative to the block, as
 * produced by an exclusive scan of the symbolic counts).  Returns 0 on success,
 * -1 on allocation failure, -2 if a row's count disagrees with its slice. */
int oracle_numeric_rows(int32_t r0, int32_t r1, int32_t k,
                        const int32_t* a_rowptr, const int32_t* a_colind, const double* a_vals,
                        const int32_t* b_rowptr, const int32_t* b_colind, const double* b_vals,
                        const int64_t* offsets, int32_t* colind, double* vals) {
  size_t kk = (size_t)(k > 0 ? k : 1);
  int64_t* marker = (int64_t*)malloc(sizeof(int64_t) * kk);
  double* acc = (double*)malloc(sizeof(double) * kk);
  if (!marker || !acc) { free(marker); free(acc); return -1; }
  for (int32_t c = 0; c < k; ++c) marker[c] = -1;
  for (int32_t i = r0; i < r1; ++i) {
    int64_t base = offsets[i - r0], end = offsets[i - r0 + 1], len = 0;
    for (int32_t p = a_rowptr[i]; p < a_rowptr[i + 1]; ++p) {
      int32_t j = a_colind[p];
      double a = a_vals[p];
      for (int32_t q = b_rowptr[j]; q < b_rowptr[j + 1]; ++q) {
        int32_t c = b_colind[q];
        if (marker[c] != i) {
          marker[c] = i;
          acc[c] = a * b_vals[q];
          if (base + len >= end) { free(marker); free(acc); return -2; }
          colind[base + len] = c;
          ++len;
        } else {
          acc[c] = fma(a, b_vals[q], acc[c]);
        }
      }
    }
    if (base + len != end) { free(marker); free(acc); return -2; }
    qsort(colind + base, (size_t)len, sizeof(int32_t), cmp_i32);
    for (int64_t t = 0; t < len; ++t) vals[base + t] = acc[colind[base + t]];
  }
  free(marker);
  free(acc);
  return 0;
}

/* Per-row flop upper bound used by row binning:
 * flop[i - r0] = sum_{j in A(i,:)} nnz(B(j,:)) (the number of multiply-adds row i
 * of C needs).  Plain definition from Eq. 1; no scratch. */
void oracle_row_flops(int32_t r0, int32_t r1,
                      const int32_t* a_rowptr, const int32_t* a_colind,
                      const int32_t* b_rowptr, int64_t* flop) {
  for (int32_t i = r0; i < r1; ++i) {
    int64_t f = 0;
    for (int32_t p = a_rowptr[i]; p < a_rowptr[i + 1]; ++p) {
      int32_t j = a_colind[p];
      f += (int64_t)(b_rowptr[j + 1] - b_rowptr[j]);
    }
    flop[i - r0] = f;
  }
}
