// Thread tier: rows with very few products (the smallest bins), one thread
// per row, the row's accumulator in registers.
//
// The paper's method A (Sec. "Standard SpGEMM Kernel": one row per thread,
// B rows walked sequentially) for rows whose product count is so small that
// any shared-memory table, its clearing and its sort cost more than the
// products: the symbolic phase keeps the distinct columns seen so far in a
// register array (at most kThreadSymMax), the numeric phase keeps up to
// kThreadNumMax (column, value) pairs sorted by insertion.  Values are float64
// in storage order (first contribution a*b, later ones fma(a, b, v)), the
// oracle's order, so the thread tier is bit-exact.  Thirty-two rows per warp
// keep many independent load chains in flight.
#include "kk_internal.h"
#include "kk_device.cuh"

namespace kk {
namespace {

constexpr int kThreadBlock = 256;

template <int N>
__global__ void __launch_bounds__(kThreadBlock)
k_sym_thread(CsrView A, CsrView B, const int32_t* __restrict__ rows, int32_t nrows,
             int32_t* __restrict__ cnt, int* status) {
  int over = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    const int i = rows[r];
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    int key[N];
    int n = 0;
    for (int p = pa; p < pe; ++p) {
      const int j = A.colind[p];
      const int be = B.rowptr[j + 1];
      for (int q = B.rowptr[j]; q < be; ++q) {
        const int c = B.colind[q];
        bool found = false;
#pragma unroll
        for (int k = 0; k < N; ++k) found |= (k < n && key[k] == c);
        if (!found) {
          if (n < N) {
#pragma unroll
            for (int k = 0; k < N; ++k)
              if (k == n) key[k] = c;
            ++n;
          } else {
            over = 1;
          }
        }
      }
    }
    cnt[i] = n;
  }
  if (over) set_status(status, KK_ERR_CAPACITY);
}

template <int N, bool JAC>
__global__ void __launch_bounds__(kThreadBlock)
k_num_thread(CsrView A, CsrView B, const int64_t* __restrict__ c_rowptr,
             const int32_t* __restrict__ rows, int32_t nrows, int32_t* __restrict__ c_colind,
             double* __restrict__ c_vals, int* status) {
  int over = 0, mismatch = 0, bad = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x) {
    const int i = rows[r];
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    const int64_t off = c_rowptr[i];
    const int cnt = (int)(c_rowptr[i + 1] - off);
    int key[N];
    double val[N];
    int n = 0;
    // JAC (a template switch: the plain kernel keeps its registers): the
    // Jacobi-fused product, A(i,:) taken as s_i A(i,:) plus 1 at the row's first
    // diagonal entry, s_i = -omega / D(i) with D(i) the sum of the row's stored
    // diagonal entries in storage order.  The row is short, so a first pass over
    // it finds D(i); the second pass below reads it again from L1.
    ARowScale ars{1.0, -1, JAC};
    if (JAC) {
      double d = 0.0;
      int first = -1;
      for (int p = pa; p < pe; ++p) {
        if (A.colind[p] == i) {
          d = first < 0 ? A.vals[p] : d + A.vals[p];
          first = first < 0 ? p : first;
        }
      }
      if (first < 0 || (__double_as_longlong(d) << 1) == 0) {
        bad = 1;
        ars.s = 0.0;
      } else {
        ars.s = -A.jac_omega * jacobi_recip(d);
      }
      ars.p = first;
    }
    for (int p = pa; p < pe; ++p) {
      const int j = A.colind[p];
      const double a = JAC ? a_scaled(ars, p, A.vals[p]) : A.vals[p];
      const int be = B.rowptr[j + 1];
      for (int q = B.rowptr[j]; q < be; ++q) {
        const int c = B.colind[q];
        const double b = B.vals[q];
        // the slot holding c, if any (keys are distinct); the float64 update is
        // then done once on a value picked by selects, not once per slot under a
        // predicate (the FP64 pipe is the scarce one on this part)
        int hit = -1;
#pragma unroll
        for (int k = 0; k < N; ++k) hit = (k < n && key[k] == c) ? k : hit;
        if (hit >= 0) {
          double cur = 0.0;
#pragma unroll
          for (int k = 0; k < N; ++k) cur = k == hit ? val[k] : cur;
          const double t = fma(a, b, cur);
#pragma unroll
          for (int k = 0; k < N; ++k) val[k] = k == hit ? t : val[k];
        } else {
          if (n < N) {
            // insertion keeps the columns ascending
            int pos = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) pos += (k < n && key[k] < c) ? 1 : 0;
#pragma unroll
            for (int k = N - 1; k > 0; --k) {
              if (k <= n && k > pos) {
                key[k] = key[k - 1];
                val[k] = val[k - 1];
              }
            }
            const double prod = a * b;
#pragma unroll
            for (int k = 0; k < N; ++k) {
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
    }
    if (n != cnt) mismatch = 1;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k < n && k < cnt) {
        c_colind[off + k] = key[k];
        c_vals[off + k] = val[k];
      }
    }
  }
  if (over) set_status(status, KK_ERR_CAPACITY);
  if (mismatch) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  // a row without a stored diagonal, or whose diagonal sums to 0
  if (JAC && bad) set_status(status, KK_ERR_INVALID_ARG);
}

int thread_grid(const LaunchCtx& ctx, int nrows) {
  long long g = ((long long)nrows + kThreadBlock - 1) / kThreadBlock;
  const long long cap = (long long)ctx.num_sms * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_symbolic_thread(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                   const int32_t* rows, int32_t nrows, int32_t* cnt) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "sym_thread");
  k_sym_thread<kThreadSymMax><<<thread_grid(ctx, nrows), kThreadBlock, 0, ctx.stream>>>(
      A, B, rows, nrows, cnt, ctx.status);
  timer_end(ctx.timer, ctx.stream);
  return cudaGetLastError();
}

cudaError_t launch_numeric_thread(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                  const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                  int32_t* c_colind, double* c_vals) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "num_thread");
  auto kern = A.jac_s != nullptr ? k_num_thread<kThreadNumMax, true>
                                 : k_num_thread<kThreadNumMax, false>;
  kern<<<thread_grid(ctx, nrows), kThreadBlock, 0, ctx.stream>>>(
      A, B, c_rowptr, rows, nrows, c_colind, c_vals, ctx.status);
  timer_end(ctx.timer, ctx.stream);
  return cudaGetLastError();
}

}  // namespace kk
