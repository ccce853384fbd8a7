/*
 * kk_spgemm.h - C ABI of the GB300 two-phase sparse matrix-matrix multiply.
 *
 * Operation (Kokkos Kernels paper, Sec. "SpGEMM: Sparse Matrix Matrix Multiply",
 * first paragraph, and Sec. "Standard SpGEMM Kernel", Eq. 1):
 *     C = A * B,  A m-by-n, B n-by-k, C m-by-k, all sparse in CSR,
 *     C(i,:) = sum_{j in A(i,:)} A(i,j) * B(j,:).
 * Split into the two phases of the same section: a symbolic phase that computes
 * the number of nonzeros of every row of C (and so C's row pointers, the last of
 * which is nnz(C)), and a numeric phase that computes C's column indices and
 * values.  The symbolic result is kept in the handle, so the numeric phase can be
 * re-run for new values on the same sparsity patterns (Sec. 2: the symbolic /
 * numeric interface split "for better performance").
 *
 * Conventions for every entry point
 *   - Index base 0.  A and B: int32 row pointers and column indices, float64
 *     values.  C: int64 row pointers (nnz(C) may exceed 2^31-1), int32 column
 *     indices, float64 values.
 *   - All matrix arrays are DEVICE pointers owned by the caller.  The library
 *     never frees or retains them beyond the call (the handle keeps only its own
 *     scratch and the symbolic result).
 *   - Output rows of C have strictly ascending column indices.  Structure is
 *     structural: an entry whose contributions cancel keeps an explicit 0.0.
 *   - Input rows may be unsorted and may repeat a column; repeats merge
 *     additively.
 *   - Work is enqueued on the handle's stream.  kk_spgemm_symbolic blocks until
 *     nnz(C) is known on the host (the one host synchronisation the method needs:
 *     C's arrays are allocated from it).  kk_spgemm_numeric does not block;
 *     errors the device detects in it surface at the next kk_spgemm_sync or
 *     blocking call on the same handle.
 *   - Every function returns a kk_status and never aborts the process.
 *     kk_spgemm_last_error gives a one-line detail of the last failure.
 */
#ifndef KK_SPGEMM_H_
#define KK_SPGEMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KK_OK = 0,
  KK_ERR_INVALID_ARG = 1,         /* null pointer, negative size, A.n != B.m, ... */
  KK_ERR_CUDA = 2,                /* a CUDA runtime call failed (detail in last_error) */
  KK_ERR_OOM = 3,                 /* device scratch allocation failed */
  KK_ERR_STRUCTURE_MISMATCH = 4,  /* numeric called with other dims / nnz / structure than symbolic */
  KK_ERR_CAPACITY = 5,            /* an accumulator or output buffer was too small */
  KK_ERR_TIMEOUT = 6,             /* a bounded device wait ran out */
  KK_ERR_NOT_SYMBOLIC = 7,        /* numeric before any symbolic on this handle */
  KK_ERR_BAD_INDEX = 8            /* a column index of A or B lies outside its range */
} kk_status;

/* A CSR matrix in device memory (caller-owned).  vals may be NULL where only the
 * structure is read (symbolic phase). */
typedef struct {
  int32_t m;               /* rows */
  int32_t n;               /* columns */
  int32_t nnz;             /* == rowptr[m] */
  const int32_t* rowptr;   /* int32[m+1] */
  const int32_t* colind;   /* int32[nnz] */
  const double* vals;      /* float64[nnz] or NULL */
} kk_csr;

/* Arithmetic of the numeric phase's accumulator. */
typedef enum {
  KK_ARITH_AUTO = 0,  /* DF32 where every value's exponent fits its safe range and the row's
                         error bound holds, FP64 otherwise; the window tier's rows of at most 256
                         columns run in FP64 (measured faster there on GB300) */
  KK_ARITH_FP64 = 1,  /* native float64 fused multiply-add in storage order */
  KK_ARITH_DF32 = 2   /* float64 emulated as an unevaluated pair of float32 on the FP32 pipe */
} kk_arith;

/* Options; kk_spgemm_options_default fills the defaults.  A NULL options
 * pointer means the defaults. */
typedef struct {
  int32_t arith;          /* kk_arith */
  int32_t debug_checks;   /* 1: extra device-side consistency checks in numeric */
  int32_t timing;         /* 1: record CUDA events around every kernel (see kk_spgemm_kernel_times)
                             and count the per-tier statistics (kk_spgemm_stats) */
  int32_t force_tier;     /* testing: -1 = automatic; 0 = team hash, 1 = CTA hash, 2 = dense chunks,
                             3 = window wherever a row qualifies (team hash elsewhere) */
  int32_t team_vec_min_len; /* mean B-row length from which a team walks B rows lane-parallel (else flattened) */
  int32_t sym_team_max_flop;  /* rows up to this flop bound use a team hash in the symbolic phase */
  int32_t sym_cta_max_flop;   /* rows up to this flop bound use a CTA hash; above it dense chunks */
  int32_t num_team_max_nnz;   /* rows up to this nnz(C(i,:)) use a team hash in the numeric phase */
  int32_t num_cta_max_nnz;    /* rows up to this nnz use a CTA hash; above it dense chunks */
  int32_t use_window;         /* 1: rows whose column span fits a shared-memory window use the
                                 dense window accumulator (needs B rows sorted) */
  int32_t batched_graph;      /* 1: batched phases are captured into CUDA graphs and replayed
                                 (needs a non-default stream) */
  int32_t sym_load_pct;       /* hash tables of the symbolic phase are sized so the flop bound
                                 fills at most this percentage (10..100, default 75) */
  int32_t num_load_pct;       /* numeric maps are sized so nnz(C(i,:)) fills at most this
                                 percentage (10..50, default 50; the sort buffer holds half) */
  int32_t structure_cache;    /* 1: the symbolic phase keeps the structure of every window row
                                 (its non-empty 32-column words, at most 64 per row, 6 bytes
                                 each) so that the numeric phase of the same A and B arrays
                                 writes C's columns without re-deriving them (default 1) */
  int32_t wide_cache_mb;      /* budget for the wide tier's kept bit vectors (rows whose values
                                 go to C by atomics keep their k-bit column vector from the
                                 symbolic phase): MiB, 0 = one eighth of the device memory,
                                 -1 = none; only with structure_cache = 1 */
  int32_t batched_mode;       /* batched form (kk_batched.h): 1 = persistent work-queue kernels
                                 (graph-capturable), 2 = the batch as one block-diagonal product
                                 through the plain two-phase kernels, 0 = automatic (2) */
  int32_t batched_learned;    /* 1: the block-diagonal batched form runs the learned form
                                 (kk_learned.h: speculative one-pass sized by the predictor
                                 attached with kk_spgemm_set_predictor, or by the flop bound
                                 without one) instead of the plain two phases (default 0).
                                 The first numeric call after such a symbolic call returns
                                 the values the speculative pass computed from the values the
                                 symbolic call saw; later numeric calls recompute from the
                                 current values */
  int32_t stage_long_rows;    /* 1: in the wide tier's symbolic phase, pieces of long B rows
                                 (>= 512 entries) are copied into shared memory by bulk copies
                                 (cp.async.bulk, two buffers of 256 columns per warp, mbarrier
                                 completion) instead of per-lane loads (default 0: on GB300 the
                                 per-lane loads measured faster, R-MAT scale 20 47 ms against 62) */
  int32_t small_max_rows;     /* products with A of at most this many rows (0..8192, default 4096)
                                 and rows of A averaging at most 32 products run each phase as one
                                 launch of one CTA (C rows of at most 16 columns, counted and
                                 accumulated in registers; float64 in A-row storage order); a row
                                 with more columns sends the call to the tiered path.  Only with
                                 force_tier = -1; 0 = never */
} kk_spgemm_options;

typedef struct kk_spgemm_handle_s* kk_spgemm_handle;

/* Fill *opt with the defaults. */
kk_status kk_spgemm_options_default(kk_spgemm_options* opt);

/* Create a handle bound to the current CUDA device and to cuda_stream (a
 * cudaStream_t; NULL = the legacy default stream).  opt may be NULL.
 * The handle owns its scratch; kk_spgemm_destroy frees it. */
kk_status kk_spgemm_handle_create(kk_spgemm_handle* h, const kk_spgemm_options* opt,
                                  void* cuda_stream);

/* Rebind the handle to another stream (same device). */
kk_status kk_spgemm_set_stream(kk_spgemm_handle h, void* cuda_stream);

/* Symbolic phase (Sec. "Standard SpGEMM Kernel": symbolic computes the number of
 * nonzeros of each row of C; the last row pointer is nnz(C)).
 *   A, B      structure read (vals ignored); A->n must equal B->m.
 *   c_rowptr  device int64[A->m + 1], caller-allocated; receives the exclusive
 *             scan of the row counts, c_rowptr[0] = 0, c_rowptr[m] = nnz(C).
 *   nnz_c     host int64 out.
 * Blocks until nnz(C) is on the host.  Keeps the row binning and counts in the
 * handle for the numeric phase. */
kk_status kk_spgemm_symbolic(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                             int64_t* c_rowptr, int64_t* nnz_c);

/* Numeric phase (same section: column indices and values of C).
 * A and B must have the dims, nnz and sparsity patterns of the last symbolic
 * call on this handle; their values may differ (symbolic reuse).  c_rowptr is
 * the array the symbolic phase filled; c_colind (int32[nnz(C)]) and c_vals
 * (float64[nnz(C)]) are caller-allocated device arrays.  Asynchronous. */
kk_status kk_spgemm_numeric(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                            const int64_t* c_rowptr, int32_t* c_colind, double* c_vals);

/* Wait for the handle's stream and report any device-side error recorded since
 * the last check. */
kk_status kk_spgemm_sync(kk_spgemm_handle h);

/* Destroy the handle and free its scratch (synchronises its stream first). */
kk_status kk_spgemm_destroy(kk_spgemm_handle h);

/* Static string naming a status code. */
const char* kk_status_string(kk_status s);

/* Detail of the last failure on this handle (valid until the next call on it). */
const char* kk_spgemm_last_error(kk_spgemm_handle h);

/* Arithmetic the last numeric call used (kk_arith value, never AUTO). */
int32_t kk_spgemm_last_arith(kk_spgemm_handle h);

/* Per-kernel timing, when options.timing == 1.  Synchronises the stream, then
 * writes up to max_kernels entries: names (static strings), total milliseconds
 * and launch counts accumulated since the last reset, and returns the number of
 * distinct kernels in *count.  reset != 0 clears the accumulators afterwards. */
kk_status kk_spgemm_kernel_times(kk_spgemm_handle h, int32_t max_kernels, const char** names,
                                 double* total_ms, int64_t* launches, int32_t* count,
                                 int32_t reset);

/* Statistics: rows per tier in each phase of the last symbolic call
 * (stats[0..2] symbolic team/CTA/dense, stats[3..5] numeric team/CTA/dense),
 * stats[6] = total flops (multiply-adds), stats[7] = 1 if B's rows were
 * strictly ascending, stats[8] / stats[9] = kernels launched by the last
 * symbolic / numeric call, stats[10] / stats[11] = rows in the window tier of
 * the symbolic / numeric phase; after a learned symbolic call (kk_learned.h)
 * stats[12] = rows sent to the speculative one-pass, stats[13] = of those, rows
 * that overflowed and were re-run, stats[14] = rows predicted heavy (plain
 * path), stats[15] = staging entries; after a plain symbolic call on a handle
 * with options.timing = 1 (else 0): stats[16..19] = C entries and
 * stats[20..23] = A entries of the rows in each numeric tier (team, CTA,
 * dense, window), for per-kernel byte accounting;
 * stats[24] = window rows whose structure the last symbolic call kept for the
 * numeric phase (options.structure_cache), stats[25] = (word, mask) pairs of
 * the compressed B it built (compare with nnz(B)); with options.timing = 1,
 * after a plain symbolic call stats[26..29] = multiply-adds of the rows in each
 * numeric tier (team, CTA, dense, window), for the FP64-pipe bound; stats[30] = rows of A when the
 * last symbolic call took the small-product path (options.small_max_rows; the
 * other entries are then 0 but stats[6], stats[8], stats[9]), else 0;
 * stats[31] = 0. */
kk_status kk_spgemm_stats(kk_spgemm_handle h, int64_t stats[32]);

#ifdef __cplusplus
}
#endif

#endif /* KK_SPGEMM_H_ */
