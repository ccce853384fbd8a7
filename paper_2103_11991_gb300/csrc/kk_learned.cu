// Device kernels of the learned form (kk_learned.h): the fused row analysis
// (features + MLP inference -> predicted capacity class per row), the
// selection of rows that need the plain two-phase path, and the copy of staged
// rows into C.
#include "kk_internal.h"
#include "kk_learned.h"
#include "kk_mlp.cuh"

namespace kk {
namespace {

constexpr int kLearnedBlock = 256;

// The learned form's row classification, one thread per row, from the row
// analysis (flop bound, span, longest and shortest referenced B row): the
// features, the MLP inference (or, without a predictor, the guaranteed bound
// min(flop, span, k)) and the row's learned bin: [0, kOnepassClasses) = warp hash one-pass of that capacity class,
// [kOnepassClasses, kLearnedHeavy) = window one-pass of that window class,
// kLearnedHeavy = heavy (plain path), 0xFF = no products.
__global__ void __launch_bounds__(kLearnedBlock)
k_learned_classify(CsrView A, int32_t bn, const int32_t* __restrict__ b_sorted, int32_t use_window,
                   int32_t window_onepass,
                   const float* __restrict__ params, float quantile, int32_t use_pred,
                   const long long* __restrict__ flop, const int32_t* __restrict__ row_span,
                   const int2* __restrict__ stat, uint8_t* __restrict__ lbin, int32_t* __restrict__ cap) {
  __shared__ float P[kMlpParams];
  if (use_pred)
    for (int t = threadIdx.x; t < kMlpParams; t += blockDim.x) P[t] = params[t];
  __syncthreads();
  const int sorted = *b_sorted;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < A.m;
       r += (long long)gridDim.x * blockDim.x) {
    const long long f = flop[r];
    if (f == 0) {
      lbin[r] = 0xFF;
      cap[r] = 0;
      continue;
    }
    const long long span = row_span[r];
    int c;
    if (use_pred) {
      const int nza = A.rowptr[r + 1] - A.rowptr[r];
      const int2 st = stat[r];
      const double mean = nza ? (double)f / nza : 0.0;
      const double v[kMlpF] = {(double)nza, (double)f, (double)st.x, mean, (double)(st.x - st.y),
                               (double)span, fmin((double)f, (double)span),
                               fmin(fmin((double)f, (double)span), (double)bn)};
      float x[kMlpF];
#pragma unroll
      for (int q = 0; q < kMlpF; ++q) x[q] = log2f(1.0f + (float)v[q]);
      float h1[kMlpH], h2[kMlpH], z[kMlpC];
      mlp_forward(P, x, h1, h2, z);
      c = mlp_class(z, quantile);
    } else {
      long long bound = f < span ? f : span;
      if (bound > bn) bound = bn;
      c = capacity_class_of(bound);
    }
    uint8_t lb = (uint8_t)kLearnedHeavy;
    if (sorted && c < kOnepassClasses) {
      lb = (uint8_t)c;  // warp hash one-pass
      for (int w = 0; use_window && w < kNumWindowClasses; ++w) {  // needs B_C
        if (span <= window_bits(w) && (long long)window_bits(w) <= (long long)kWindowFlopRatio * f) {
          // window one-pass; with the structure cache on, the plain path
          // instead (its numeric phase is then the value pass alone, which
          // the one-pass measured slower than)
          lb = (uint8_t)(window_onepass ? kOnepassClasses + w : kLearnedHeavy);
          break;
        }
      }
    }
    lbin[r] = lb;
    cap[r] = lb < kLearnedHeavy ? (16 << c) : 0;
  }
}

// Rows that take the plain path (heavy, or overflowed in the one-pass): their
// symbolic bin from the flop bound; every other row is skipped.  Also records
// the plain-path flag used by the learned numeric phase.
__global__ void k_learned_leftover(int32_t m, const uint8_t* __restrict__ lbin,
                                   const int32_t* __restrict__ cnt, uint8_t* __restrict__ plain,
                                   const uint8_t* __restrict__ sbin_all, uint8_t* __restrict__ sbin) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t b = lbin[i];
    const bool p = (b == (uint8_t)kLearnedHeavy) || (b != 0xFF && cnt[i] < 0);
    plain[i] = p ? 1 : 0;
    sbin[i] = p ? sbin_all[i] : (uint8_t)0xFF;
  }
}

__global__ void k_mask_bins(int32_t m, const uint8_t* __restrict__ plain, const uint8_t* __restrict__ nbin,
                            uint8_t* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = plain[i] ? nbin[i] : (uint8_t)0xFF;
}

// Warp per row: copy a staged row (columns and values) into C.
__global__ void k_copy_staged(int32_t m, const uint8_t* __restrict__ lbin, const uint8_t* __restrict__ plain,
                              const int64_t* __restrict__ soff, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ scol, const double* __restrict__ sval,
                              int32_t* __restrict__ ccol, double* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = w0; i < m; i += nw) {
    const uint8_t b = lbin[i];
    if (b == 0xFF || b >= (uint8_t)kLearnedHeavy || plain[i]) continue;
    const int64_t src = soff[i], dst = rowptr[i];
    const int n = (int)(rowptr[i + 1] - dst);
    for (int e = lane; e < n; e += 32) {
      ccol[dst + e] = scol[src + e];
      cval[dst + e] = sval[src + e];
    }
  }
}

int grid1(long long n, int block, int cap) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

cudaError_t launch_learned_classify(const LaunchCtx& ctx, const CsrView& A, int32_t bn,
                                    const int32_t* b_sorted, int32_t use_window, int32_t window_onepass,
                                    const float* params,
                                    float quantile, int32_t use_pred, const long long* flop,
                                    const int32_t* row_span, const int2* stat, uint8_t* lbin, int32_t* cap) {
  if (A.m <= 0) return cudaSuccess;
  k_learned_classify<<<grid1(A.m, kLearnedBlock, ctx.num_sms * 8), kLearnedBlock, 0, ctx.stream>>>(
      A, bn, b_sorted, use_window, window_onepass, params, quantile, use_pred, flop, row_span, stat, lbin, cap);
  return cudaGetLastError();
}

cudaError_t launch_learned_leftover(const LaunchCtx& ctx, int32_t m, const uint8_t* lbin,
                                    const int32_t* cnt, uint8_t* plain, const uint8_t* sbin_all,
                                    uint8_t* sbin) {
  if (m <= 0) return cudaSuccess;
  k_learned_leftover<<<grid1(m, 256, ctx.num_sms * 8), 256, 0, ctx.stream>>>(m, lbin, cnt, plain,
                                                                             sbin_all, sbin);
  return cudaGetLastError();
}

cudaError_t launch_mask_bins(const LaunchCtx& ctx, int32_t m, const uint8_t* plain,
                             const uint8_t* nbin, uint8_t* out) {
  if (m <= 0) return cudaSuccess;
  k_mask_bins<<<grid1(m, 256, ctx.num_sms * 8), 256, 0, ctx.stream>>>(m, plain, nbin, out);
  return cudaGetLastError();
}

cudaError_t launch_copy_staged(const LaunchCtx& ctx, int32_t m, const uint8_t* lbin,
                               const uint8_t* plain, const int64_t* soff, const int64_t* rowptr,
                               const int32_t* scol, const double* sval, int32_t* ccol,
                               double* cval) {
  if (m <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "copy_staged");
  k_copy_staged<<<grid1((long long)m * 32, 256, ctx.num_sms * 16), 256, 0, ctx.stream>>>(
      m, lbin, plain, soff, rowptr, scol, sval, ccol, cval);
  timer_end(ctx.timer, ctx.stream);
  return cudaGetLastError();
}

}  // namespace kk
