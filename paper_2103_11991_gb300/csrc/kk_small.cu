// Small products: each phase in one launch (a latency path).
//
// For A with at most options.small_max_rows rows, the paper's two phases (Sec.
// "Standard SpGEMM Kernel") run without the analysis, binning, scan and
// per-tier launches of the general path, whose launch latencies dominate a
// product of this size (the 64^2 5-point product has 10^5 multiply-adds): the
// symbolic kernel counts every row's distinct columns in registers (one
// thread per row, as the thread tier does) and checks the indices as the
// analysis passes do; the last CTA to finish (a ticket taken after each CTA's
// counts are visible; nothing waits) scans the counts into C's row pointers.
// The numeric kernel accumulates every row in registers in A-row storage
// order (first contribution a*b, later ones fma(a, b, v): the oracle's order,
// so results are bit-exact) and writes it sorted.  A row with more than
// kSmallN distinct columns stops the attempt (the caller then runs the
// general path); indices outside their ranges are reported as in the general
// path.
#include "kk_internal.h"
#include "kk_device.cuh"

namespace kk {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Exclusive scan over the CTA's threads (blockDim.x a multiple of 32, at most
// 1024); *total receives the sum.  Ends with a barrier.
__device__ __forceinline__ long long small_exscan(long long v, long long* tmp, long long* total) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long n = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const long long x = lane < nw ? tmp[lane] : 0;
    long long xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long n = __shfl_up_sync(kFull, xi, o);
      if (lane >= o) xi += n;
    }
    tmp[lane] = xi - x;
    if (lane == 31) tmp[32] = xi;
  }
  __syncthreads();
  const long long r = tmp[warp] + incl - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

// flags[0]: a row had more than kSmallN columns; flags[1]: an index outside
// its range; flags[2]: the CTAs' ticket counter (zero before the launch).
// cnt: scratch of A.m counts.  out[0] = nnz(C), out[1] = multiply-adds.
__global__ void __launch_bounds__(kSmallThreads)
k_small_symbolic(CsrView A, CsrView B, int64_t* __restrict__ c_rowptr, int32_t* __restrict__ cnt,
                 int32_t* flags, long long* out) {
  __shared__ long long tmp[33];
  __shared__ int s_last;
  const int m = A.m;
  int bad = 0, over = 0;
  long long flop = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (A.rowptr[0] != 0 || B.rowptr[0] != 0)) bad = 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    if (pa < 0 || pe < pa || pe > A.nnz) {
      bad = 1;
      pe = pa;
    }
    int key[kSmallN];
    int n = 0;
    for (int p = pa; p < pe && !over; ++p) {
      const int j = A.colind[p];
      if ((unsigned)j >= (unsigned)B.m) {
        bad = 1;
        continue;
      }
      const int bs = B.rowptr[j], be = B.rowptr[j + 1];
      if (bs < 0 || be < bs || be > B.nnz) {
        bad = 1;
        continue;
      }
      flop += be - bs;
      for (int q = bs; q < be; ++q) {
        const int c = B.colind[q];
        if ((unsigned)c >= (unsigned)B.n) {
          bad = 1;
          continue;
        }
        bool found = false;
#pragma unroll
        for (int k = 0; k < kSmallN; ++k) found |= (k < n && key[k] == c);
        if (!found) {
          if (n < kSmallN) {
#pragma unroll
            for (int k = 0; k < kSmallN; ++k)
              if (k == n) key[k] = c;
            ++n;
          } else {
            over = 1;
            break;
          }
        }
      }
    }
    cnt[i] = n;
  }
  bad = __any_sync(kFull, bad);
  over = __any_sync(kFull, over);
  for (int o = 16; o > 0; o >>= 1) flop += __shfl_xor_sync(kFull, flop, o);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(&flags[1], 1);
    if (over) atomicOr(&flags[0], 1);
    if (flop) atomicAdd(reinterpret_cast<unsigned long long*>(&out[1]), (unsigned long long)flop);
  }
  // the last CTA to finish scans all counts
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&flags[2], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (__ldcg(&flags[0]) != 0) return;  // a row beyond the path: the tiered path takes over
  const int R = (m + blockDim.x - 1) / blockDim.x;
  const int r0 = threadIdx.x * R;
  long long mine = 0;
  for (int k = 0; k < R; ++k)
    if (r0 + k < m) mine += __ldcg(&cnt[r0 + k]);
  long long total;
  long long run = small_exscan(mine, tmp, &total);
  for (int k = 0; k < R; ++k) {
    if (r0 + k < m) {
      c_rowptr[r0 + k] = run;
      run += __ldcg(&cnt[r0 + k]);
    }
  }
  if (threadIdx.x == 0) {
    c_rowptr[m] = total;
    out[0] = total;
  }
}

// JAC: the Jacobi-fused product, A(i,:) taken as s_i A(i,:) plus 1 at the
// row's first diagonal entry, s_i = -omega / D(i) (D(i) the sum of the row's
// stored diagonal entries), formed from the row itself as the thread tier does.
template <bool JAC>
__global__ void __launch_bounds__(kSmallNumThreads)
k_small_numeric(CsrView A, CsrView B, const int64_t* __restrict__ c_rowptr, int32_t* __restrict__ c_colind,
                double* __restrict__ c_vals, int* status) {
  int over = 0, mismatch = 0, bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.m; i += gridDim.x * blockDim.x) {
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    const int64_t off = c_rowptr[i];
    const int cnt = (int)(c_rowptr[i + 1] - off);
    double s = 1.0;
    int dpos = -1;
    if (JAC) {
      double d = 0.0;
      for (int p = pa; p < pe; ++p) {
        if (A.colind[p] == i) {
          d = dpos < 0 ? A.vals[p] : d + A.vals[p];
          dpos = dpos < 0 ? p : dpos;
        }
      }
      if (dpos < 0 || (__double_as_longlong(d) << 1) == 0) {
        bad = 1;
        s = 0.0;
      } else {
        s = -A.jac_omega * jacobi_recip(d);
      }
    }
    int key[kSmallN];
    double val[kSmallN];
    int n = 0;
    for (int p = pa; p < pe; ++p) {
      const int j = A.colind[p];
      const double a = JAC ? (p == dpos ? fma(s, A.vals[p], 1.0) : s * A.vals[p]) : A.vals[p];
      const int be = B.rowptr[j + 1];
      for (int q = B.rowptr[j]; q < be; ++q) {
        const int c = B.colind[q];
        const double b = B.vals[q];
        int hit = -1;
#pragma unroll
        for (int k = 0; k < kSmallN; ++k) hit = (k < n && key[k] == c) ? k : hit;
        if (hit >= 0) {
          double cur = 0.0;
#pragma unroll
          for (int k = 0; k < kSmallN; ++k) cur = k == hit ? val[k] : cur;
          const double t = fma(a, b, cur);
#pragma unroll
          for (int k = 0; k < kSmallN; ++k) val[k] = k == hit ? t : val[k];
        } else if (n < kSmallN) {
          // insertion keeps the columns ascending
          int pos = 0;
#pragma unroll
          for (int k = 0; k < kSmallN; ++k) pos += (k < n && key[k] < c) ? 1 : 0;
#pragma unroll
          for (int k = kSmallN - 1; k > 0; --k) {
            if (k <= n && k > pos) {
              key[k] = key[k - 1];
              val[k] = val[k - 1];
            }
          }
          const double prod = a * b;
#pragma unroll
          for (int k = 0; k < kSmallN; ++k) {
            if (k == pos) {
              key[k] = c;
              val[k] = prod;
            }
          }
          ++n;
        } else {
          over = 1;
        }
      }
    }
    if (n != cnt) mismatch = 1;
#pragma unroll
    for (int k = 0; k < kSmallN; ++k) {
      if (k < n && k < cnt) {
        c_colind[off + k] = key[k];
        c_vals[off + k] = val[k];
      }
    }
  }
  if (over) set_status(status, KK_ERR_CAPACITY);
  if (mismatch) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  if (JAC && bad) set_status(status, KK_ERR_INVALID_ARG);
}

}  // namespace

cudaError_t launch_small_symbolic(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, int64_t* c_rowptr,
                                  int32_t* cnt, int32_t* flags, long long* out) {
  const int grid = (A.m + kSmallThreads - 1) / kSmallThreads;
  k_small_symbolic<<<grid, kSmallThreads, 0, ctx.stream>>>(A, B, c_rowptr, cnt, flags, out);
  return cudaGetLastError();
}

cudaError_t launch_small_numeric(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                 const int64_t* c_rowptr, int32_t* c_colind, double* c_vals) {
  const int grid = (A.m + kSmallNumThreads - 1) / kSmallNumThreads;
  if (A.jac_s != nullptr)
    k_small_numeric<true><<<grid, kSmallNumThreads, 0, ctx.stream>>>(A, B, c_rowptr, c_colind, c_vals, ctx.status);
  else
    k_small_numeric<false><<<grid, kSmallNumThreads, 0, ctx.stream>>>(A, B, c_rowptr, c_colind, c_vals, ctx.status);
  return cudaGetLastError();
}

}  // namespace kk
