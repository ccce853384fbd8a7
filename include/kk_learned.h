/*
 * kk_learned.h - C ABI of the learned row-capacity predictor and of the
 * speculative one-pass form of the two-phase SpGEMM (include kk_spgemm.h first).
 *
 * The Kokkos Kernels paper has no learned component; its two-phase method
 * (Sec. "Standard SpGEMM Kernel") runs a symbolic sweep over every row before
 * the numeric one.  The learned form predicts each row's nnz(C(i,:)) class from
 * cheap row features with a small MLP and runs one speculative pass that
 * computes structure and values together into a staging area sized by the
 * predictions; rows whose prediction was too small overflow and are re-run
 * through the plain symbolic + numeric path, so the result is the same CSR
 * (structure bit-identical, values within the same bound).  The overflow /
 * re-run pattern mirrors the paper's speculative graph colouring (Sec.
 * "Distance-1 Graph Coloring": colour speculatively, detect conflicts, redo).
 *
 * Network: F = 8 features -> 32 -> 32 -> 16 classes, ReLU, softmax cross-entropy.
 * Parameters are one float32 vector of KK_MLP_NUM_PARAMS entries in the order
 * W1 (8 x 32, row-major), b1 (32), W2 (32 x 32), b2 (32), W3 (32 x 16), b3 (16).
 *
 * Features of row i of C = A*B, in this order, each log2(1 + value):
 *   nnz(A(i,:)); flop = sum_{j in A(i,:)} nnz(B(j,:)); max and mean (flop / nnz)
 *   of the referenced B-row lengths; their spread (max - min); the column span
 *   (max column - min column + 1 over the referenced non-empty B rows, 0 if
 *   none); min(flop, span); min(flop, span, k) with k the columns of B.
 * Class of a count c: 0 if c <= 16, else ceil(log2(c / 16)), capped at 15;
 * capacity of class t: 16 * 2^t.
 *
 * All arrays are device arrays unless marked host; every call is enqueued on
 * the given stream (or the handle's) and returns a kk_status.
 */
#ifndef KK_LEARNED_H_
#define KK_LEARNED_H_

#include "kk_spgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define KK_MLP_FEATURES 8
#define KK_MLP_HIDDEN 32
#define KK_MLP_CLASSES 16
#define KK_MLP_NUM_PARAMS 1872

/* Features of every row of C = A*B into features (float32[m * 8], row-major). */
kk_status kk_spgemm_row_features(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                                 float* features);

/* Capacity class of every row from C's row pointers (int64[m+1]) into cls
 * (int32[m]): the training labels the symbolic phase generates. */
kk_status kk_capacity_classes(void* cuda_stream, int32_t m, const int64_t* c_rowptr, int32_t* cls);

/* Seeded initialisation of params (float32[KK_MLP_NUM_PARAMS]): weights uniform
 * in +-sqrt(6 / fan_in) from a SplitMix64 stream, biases 0. */
kk_status kk_mlp_init(void* cuda_stream, float* params, uint64_t seed);

/* Mean softmax cross-entropy of the n samples X (float32[n*8]) with labels y
 * (int32[n]) and its gradient with respect to params: grad (float32[1872]) and
 * loss (float32[1]) are overwritten. */
kk_status kk_mlp_loss_grad(void* cuda_stream, int32_t n, const float* X, const int32_t* y,
                           const float* params, float* grad, float* loss);

/* One Adam step (Kingma & Ba) on params with moment buffers m1, m2
 * (float32[1872] each, zero at step 1); step counts from 1. */
kk_status kk_mlp_adam(void* cuda_stream, const float* grad, float* params, float* m1, float* m2,
                      int32_t step, float lr, float beta1, float beta2, float eps);

/* Mini-batch Adam training on the GPU: `epochs` passes over the n samples in a
 * seeded order, batches of `batch` samples.  params is updated in place;
 * *final_loss (host) receives the mean loss over the last epoch. */
kk_status kk_mlp_train(void* cuda_stream, int32_t n, const float* X, const int32_t* y,
                       float* params, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                       float* final_loss);

/* Predicted class of each sample: the smallest class whose cumulative softmax
 * probability reaches `quantile` (quantile <= 0: argmax). */
kk_status kk_mlp_predict(void* cuda_stream, int32_t n, const float* X, const float* params,
                         float quantile, int32_t* cls);

/* Attach predictor parameters (host float32[KK_MLP_NUM_PARAMS], copied) and the
 * capacity quantile to a handle; NULL detaches (the learned form then sizes
 * rows by their flop bound). */
kk_status kk_spgemm_set_predictor(kk_spgemm_handle h, const float* params_host, float quantile);

/* Learned symbolic phase: row features and MLP inference fused into one row
 * pass, then one speculative pass computing structure and values of every
 * row predicted to fit a warp accumulator into a staging area, a plain
 * symbolic pass for the rows predicted heavy and for the rows that overflowed,
 * and the scan of all counts into c_rowptr (int64[m+1]).  A and B need values.
 * The one-pass needs B's rows strictly ascending; otherwise every row takes
 * the plain path (same result, no speculation).  Blocks until nnz(C) is on the
 * host. */
kk_status kk_spgemm_learned_symbolic(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                                     int64_t* c_rowptr, int64_t* nnz_c);

/* Learned numeric phase: moves the staged rows into C and runs the plain
 * numeric pass on the heavy and overflowed rows.  A and B must be the
 * matrices (values included) of the last learned symbolic call; for new values
 * on the same patterns call kk_spgemm_numeric instead.  Asynchronous. */
kk_status kk_spgemm_learned_numeric(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                                    const int64_t* c_rowptr, int32_t* c_colind, double* c_vals);

#ifdef __cplusplus
}
#endif

#endif /* KK_LEARNED_H_ */
