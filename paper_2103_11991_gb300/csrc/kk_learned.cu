// Device kernels of the learned form (kk_learned.h): the fused row analysis
// (features + MLP inference -> predicted capacity class per row), the
// selection of rows that need the plain two-phase path, and the copy of staged
// rows into C.
#include "kk_internal.h"
#include "kk_learned.h"
#include "kk_mlp.cuh"

namespace kk {
namespace {

constexpr int kLearnedBlock = 128;

// One thread per row: flop bound, span, features, MLP inference, and the
// row's learned bin: [0, kOnepassClasses) = warp hash one-pass of that
// capacity class, [kOnepassClasses, kLearnedHeavy) = window one-pass of that
// window class, kLearnedHeavy = heavy (plain path), 0xFF = no products.
__global__ void __launch_bounds__(kLearnedBlock)
k_learned_analyze(CsrView A, CsrView B, const int32_t* __restrict__ b_sorted, int32_t use_window,
                  const float* __restrict__ params, float quantile, int32_t use_pred,
                  long long* __restrict__ flop, int32_t* __restrict__ row_lo,
                  int32_t* __restrict__ row_span, uint8_t* __restrict__ lbin,
                  int32_t* __restrict__ cap, unsigned long long* total_flop, int* status) {
  __shared__ float P[kMlpParams];
  unsigned long long acc = 0;
  if (use_pred)
    for (int t = threadIdx.x; t < kMlpParams; t += blockDim.x) P[t] = params[t];
  __syncthreads();
  const int sorted = *b_sorted;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  // each warp takes 32 consecutive rows: the lanes gather every row's
  // statistics together (coalesced), then lane t runs the MLP for row base + t
  for (long long base = warp0 * 32; base < A.m; base += nwarps * 32) {
    long long my_f = 0;
    int my_nza = 0, my_mx = 0, my_mn = 0, my_lo = 0x7fffffff, my_hi = -1;
    const int nrow = (int)min((long long)32, A.m - base);
    for (int t = 0; t < nrow; ++t) {
      const long long r = base + t;
      int pa = A.rowptr[r], pe = A.rowptr[r + 1];
      if (pa < 0 || pe < pa || pe > A.nnz || (r == 0 && pa != 0)) {
        if (lane == 0) set_status(status, KK_ERR_BAD_INDEX);
        pe = pa;
      }
      long long f = 0;
      int mx = 0, mn = 0x7fffffff, lo = 0x7fffffff, hi = -1;
      for (int p = pa + lane; p < pe; p += 32) {
        const int j = A.colind[p];
        if ((unsigned)j >= (unsigned)B.m) {
          set_status(status, KK_ERR_BAD_INDEX);
          continue;
        }
        const int bs = B.rowptr[j], be = B.rowptr[j + 1];
        const int len = be - bs;
        f += len;
        mx = max(mx, len);
        mn = min(mn, len);
        if (len > 0) {
          lo = min(lo, B.colind[bs]);
          hi = max(hi, B.colind[be - 1]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == t) {
        my_f = f;
        my_nza = pe - pa;
        my_mx = mx;
        my_mn = my_nza ? mn : 0;
        my_lo = lo;
        my_hi = hi;
      }
    }
    if (lane >= nrow) continue;
    const long long r = base + lane;
    const long long f = my_f;
    const long long span = my_hi >= my_lo ? (long long)my_hi - my_lo + 1 : 0;
    flop[r] = f;
    acc += (unsigned long long)f;
    row_lo[r] = my_hi >= my_lo ? my_lo : 0;
    row_span[r] = span > 0x7fffffff ? 0x7fffffff : (int)span;
    if (f == 0) {
      lbin[r] = 0xFF;
      cap[r] = 0;
      continue;
    }
    int c;
    if (use_pred) {
      const double mean = my_nza ? (double)f / my_nza : 0.0;
      const double v[kMlpF] = {(double)my_nza, (double)f, (double)my_mx, mean, (double)(my_mx - my_mn),
                               (double)span, fmin((double)f, (double)span),
                               fmin(fmin((double)f, (double)span), (double)B.n)};
      float x[kMlpF];
#pragma unroll
      for (int t = 0; t < kMlpF; ++t) x[t] = log2f(1.0f + (float)v[t]);
      float h1[kMlpH], h2[kMlpH], z[kMlpC];
      mlp_forward(P, x, h1, h2, z);
      c = mlp_class(z, quantile);
    } else {
      // no predictor: size by the guaranteed bound min(flop, span, k)
      long long bound = f < span ? f : span;
      if (bound > B.n) bound = B.n;
      c = capacity_class_of(bound);
    }
    uint8_t lb = (uint8_t)kLearnedHeavy;
    if (sorted && c < kOnepassClasses) {
      lb = (uint8_t)c;  // warp hash one-pass
      for (int w = 0; use_window && w < kNumWindowClasses; ++w) {  // needs B_C
        if (span <= window_bits(w) && (long long)window_bits(w) <= (long long)kWindowFlopRatio * f) {
          lb = (uint8_t)(kOnepassClasses + w);  // window one-pass
          break;
        }
      }
    }
    lbin[r] = lb;
    cap[r] = lb < kLearnedHeavy ? (16 << c) : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && acc) atomicAdd(total_flop, acc);
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

cudaError_t launch_learned_analyze(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                   const int32_t* b_sorted, int32_t use_window,
                                   const float* params, float quantile,
                                   int32_t use_pred, long long* flop, int32_t* row_lo,
                                   int32_t* row_span, uint8_t* lbin, int32_t* cap,
                                   unsigned long long* total_flop) {
  if (A.m <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "learned_analyze");
  k_learned_analyze<<<grid1(A.m, kLearnedBlock, ctx.num_sms * 16), kLearnedBlock, 0, ctx.stream>>>(
      A, B, b_sorted, use_window, params, quantile, use_pred, flop, row_lo, row_span, lbin, cap,
      total_flop,
      ctx.status);
  timer_end(ctx.timer, ctx.stream);
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
