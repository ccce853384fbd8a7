// Sparse matrix addition C = alpha A + beta B (Kokkos Kernels paper, Sec.
// "SpAdd"), symbolic and numeric phases.
//
// Symbolic, per row: the row's entries of A and B become 64-bit keys
// (column << 32 | source bit (B) << 31 | index within the source row) in
// shared memory and are sorted by a bitonic network; equal columns are then
// adjacent, so a scan of "first of its column" flags gives nnz(C(i,:)) and, for
// every entry of A and of B, its slot in the row of C (the paper's Apos and
// Bpos).  Rows that are both strictly ascending take their slots by binary
// search of each entry in the other row (no sort).  When both rows are sorted
// (repeats allowed) the keys are laid out as A ascending, then
// padding, then B descending: a bitonic sequence, so only the final merge
// stage runs (the paper's sorted-input method); otherwise the full sort runs
// (its unsorted-input method).  Rows of up to kAddWarpMax combined entries take
// one warp, rows of up to kAddCtaMax one CTA of 1024 threads; longer rows are
// reported as KK_ERR_CAPACITY.
//
// Numeric: C's values are zeroed, then every entry of A and of B adds its
// scaled value at its slot (float64 atomics: an entry of C with at most one
// entry of A and one of B is the same sum in either order; repeated columns
// within A or B are added in no fixed order) and writes its column.
#include "kk_internal.h"
#include "kk_device.cuh"

namespace kk {
namespace {

using u64 = unsigned long long;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kAddWarpMax = 256;
constexpr int kAddCtaMax = 8192;
constexpr int kAddWarps = 4;     // warps per CTA of the warp kernel
constexpr int kAddCtaThreads = 1024;
constexpr u64 kAddPad = ~0ull;

__device__ __forceinline__ int next_pow2(int x) {
  int n = 32;
  while (n < x) n <<= 1;
  return n;
}

// Exclusive scan of v over the CTA (blockDim.x a multiple of 32, at most 1024);
// *total receives the sum.  scratch: 33 ints of shared memory.
__device__ __forceinline__ int add_block_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int incl = team_inclusive_scan<32>(v, lane, kFull);
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < nw ? scratch[lane] : 0;
    const int wi = team_inclusive_scan<32>(w, lane, kFull);
    if (lane < nw) scratch[lane] = wi - w;
    if (lane == 31) scratch[32] = wi;
  }
  __syncthreads();
  const int r = scratch[warp] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

// Bitonic sort (merge_only: the final merge of an already bitonic sequence) of
// key[0, n), n a power of two, by NT cooperating threads (32: one warp, else the
// whole CTA).
template <int NT>
__device__ __forceinline__ void add_sort(u64* key, int n, int tid, bool merge_only) {
  for (int k = merge_only ? n : 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = tid; t < n; t += NT) {
        const int l = t ^ j;
        if (l > t) {
          const u64 a = key[t], b = key[l];
          const bool up = (t & k) == 0;
          if ((a > b) == up) {
            key[t] = b;
            key[l] = a;
          }
        }
      }
      if (NT == 32) __syncwarp();
      else __syncthreads();
    }
  }
}

// Keys of row r into key[0, n): A at [0, la), padding, B reversed at [n - lb, n).
// Returns (by reference) whether both rows are non-decreasing and whether a
// column lies outside [0, ncols).
template <int NT>
__device__ __forceinline__ void add_load(const CsrView& A, const CsrView& B, int pa, int la, int pb,
                                         int lb, int n, u64* key, int tid, int& unsorted, int& bad) {
  for (int t = tid; t < n; t += NT) key[t] = kAddPad;
  if (NT == 32) __syncwarp();
  else __syncthreads();
  for (int t = tid; t < la; t += NT) {
    const int c = A.colind[pa + t];
    if ((unsigned)c >= (unsigned)A.n) bad = 1;
    if (t > 0 && A.colind[pa + t - 1] > c) unsorted = 1;
    key[t] = ((u64)(uint32_t)c << 32) | (u64)t;
  }
  for (int t = tid; t < lb; t += NT) {
    const int c = B.colind[pb + t];
    if ((unsigned)c >= (unsigned)B.n) bad = 1;
    if (t > 0 && B.colind[pb + t - 1] > c) unsorted = 1;
    key[n - 1 - t] = ((u64)(uint32_t)c << 32) | (1ull << 31) | (u64)t;
  }
}

// First index in the sorted row x[0, len) whose column is >= c.
__device__ __forceinline__ int add_lower_bound(const int32_t* __restrict__ x, int len, int c) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (x[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Slots of one strictly ascending row against another (merge by binary
// search, no sort): entry k of x at column c lands at
//   k + #{y < c} - #{columns of x before k that are also in y},
// the last term an exclusive scan of "found in y" flags.  Returns the number
// of columns x shares with y.
__device__ __forceinline__ int add_slots_sorted(const int32_t* __restrict__ x, int lx,
                                                const int32_t* __restrict__ y, int ly,
                                                int32_t* __restrict__ pos, int lane) {
  int common = 0;
  for (int t0 = 0; t0 < lx; t0 += 32) {
    const int t = t0 + lane;
    int lb = 0, found = 0;
    if (t < lx) {
      const int c = x[t];
      lb = add_lower_bound(y, ly, c);
      found = (lb < ly && y[lb] == c) ? 1 : 0;
    }
    const int incl = team_inclusive_scan<32>(found, lane, kFull);
    if (t < lx) pos[t] = t + lb - (common + incl - found);
    common += __shfl_sync(kFull, incl, 31);
  }
  return common;
}

// One warp per row; rows longer than kAddWarpMax go to the long-row list.
__global__ void __launch_bounds__(kAddWarps * 32)
k_spadd_sym_warp(CsrView A, CsrView B, int32_t* __restrict__ cnt, int32_t* __restrict__ apos,
                 int32_t* __restrict__ bpos, int32_t* __restrict__ long_rows,
                 int32_t* __restrict__ long_count, int* status) {
  __shared__ u64 keys[kAddWarps][kAddWarpMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  u64* key = keys[warp];
  const long long nw = (long long)gridDim.x * kAddWarps;
  int bad = 0;
  for (long long r = (long long)blockIdx.x * kAddWarps + warp; r < A.m; r += nw) {
    const int pa = A.rowptr[r], la = A.rowptr[r + 1] - pa;
    const int pb = B.rowptr[r], lb = B.rowptr[r + 1] - pb;
    const int L = la + lb;
    if (L > kAddWarpMax) {
      if (lane == 0) long_rows[atomicAdd(long_count, 1)] = (int32_t)r;
      continue;
    }
    if (L == 0) {
      if (lane == 0) cnt[r] = 0;
      continue;
    }
    // both rows strictly ascending (no repeated column): slots by binary search
    int strict_bad = 0;
    for (int t = lane; t < la; t += 32) {
      const int c = A.colind[pa + t];
      if ((unsigned)c >= (unsigned)A.n) bad = 1;
      if (t > 0 && A.colind[pa + t - 1] >= c) strict_bad = 1;
    }
    for (int t = lane; t < lb; t += 32) {
      const int c = B.colind[pb + t];
      if ((unsigned)c >= (unsigned)B.n) bad = 1;
      if (t > 0 && B.colind[pb + t - 1] >= c) strict_bad = 1;
    }
    if (!__any_sync(kFull, strict_bad)) {
      const int common = add_slots_sorted(A.colind + pa, la, B.colind + pb, lb, apos + pa, lane);
      add_slots_sorted(B.colind + pb, lb, A.colind + pa, la, bpos + pb, lane);
      if (lane == 0) cnt[r] = la + lb - common;
      continue;
    }
    const int n = next_pow2(L);
    int unsorted = 0;
    add_load<32>(A, B, pa, la, pb, lb, n, key, lane, unsorted, bad);
    unsorted = __any_sync(kFull, unsorted);
    __syncwarp();
    add_sort<32>(key, n, lane, !unsorted);
    // slots: scan of "first of its column" flags over the L sorted keys
    int run = 0;
    for (int t0 = 0; t0 < L; t0 += 32) {
      const int t = t0 + lane;
      u64 k = 0;
      int first = 0;
      if (t < L) {
        k = key[t];
        first = (t == 0 || (key[t - 1] >> 32) != (k >> 32)) ? 1 : 0;
      }
      const int incl = team_inclusive_scan<32>(first, lane, kFull);
      if (t < L) {
        const int slot = run + incl - 1;
        const int idx = (int)(k & 0x7fffffffull);
        if (k & (1ull << 31)) bpos[pb + idx] = slot;
        else apos[pa + idx] = slot;
      }
      run += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) cnt[r] = run;
    __syncwarp();
  }
  if (bad) set_status(status, KK_ERR_BAD_INDEX);
}

// One CTA of kAddCtaThreads per long row (dynamic shared memory kAddCtaMax keys).
__global__ void __launch_bounds__(kAddCtaThreads)
k_spadd_sym_cta(CsrView A, CsrView B, int32_t* __restrict__ cnt, int32_t* __restrict__ apos,
                int32_t* __restrict__ bpos, const int32_t* __restrict__ rows,
                const int32_t* __restrict__ nrows_dev, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  u64* key = reinterpret_cast<u64*>(smem_raw);
  __shared__ int scratch[33];
  __shared__ int flags[2];
  const int tid = threadIdx.x;
  const int nrows = *nrows_dev;
  for (int q = blockIdx.x; q < nrows; q += gridDim.x) {
    const int r = rows[q];
    const int pa = A.rowptr[r], la = A.rowptr[r + 1] - pa;
    const int pb = B.rowptr[r], lb = B.rowptr[r + 1] - pb;
    const int L = la + lb;
    if (L > kAddCtaMax) {
      if (tid == 0) set_status(status, KK_ERR_CAPACITY);
      continue;
    }
    if (tid == 0) {
      flags[0] = 0;
      flags[1] = 0;
    }
    int n = 32;
    while (n < L) n <<= 1;
    int unsorted = 0, bad = 0;
    add_load<kAddCtaThreads>(A, B, pa, la, pb, lb, n, key, tid, unsorted, bad);
    if (unsorted) flags[0] = 1;
    if (bad) flags[1] = 1;
    __syncthreads();
    const bool merge_only = flags[0] == 0;
    if (tid == 0 && flags[1]) set_status(status, KK_ERR_BAD_INDEX);
    add_sort<kAddCtaThreads>(key, n, tid, merge_only);
    int run = 0;
    for (int t0 = 0; t0 < L; t0 += kAddCtaThreads) {
      const int t = t0 + tid;
      u64 k = 0;
      int first = 0;
      if (t < L) {
        k = key[t];
        first = (t == 0 || (key[t - 1] >> 32) != (k >> 32)) ? 1 : 0;
      }
      int tot;
      const int ex = add_block_scan(first, scratch, &tot);
      if (t < L) {
        const int slot = run + ex + first - 1;
        const int idx = (int)(k & 0x7fffffffull);
        if (k & (1ull << 31)) bpos[pb + idx] = slot;
        else apos[pa + idx] = slot;
      }
      run += tot;
    }
    if (tid == 0) cnt[r] = run;
    __syncthreads();
  }
}

// Numeric: one warp per row; every entry adds its scaled value at its slot.
__global__ void __launch_bounds__(256)
k_spadd_num(CsrView A, CsrView B, double alpha, double beta, const int64_t* __restrict__ c_rowptr,
            const int32_t* __restrict__ apos, const int32_t* __restrict__ bpos,
            int32_t* __restrict__ c_colind, double* __restrict__ c_vals) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  // coefficients of 1 skip the float64 multiply (FP64 is the scarce pipe): the
  // branches are uniform over the grid, so no multiply is issued at all
  const bool a1 = alpha == 1.0, b1 = beta == 1.0;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < A.m; r += nw) {
    const int64_t off = c_rowptr[r];
    const int pa = A.rowptr[r], pae = A.rowptr[r + 1];
    if (a1) {
      for (int p = pa + lane; p < pae; p += 32) {
        const int64_t s = off + apos[p];
        c_colind[s] = A.colind[p];
        atomicAdd(&c_vals[s], A.vals[p]);
      }
    } else {
      for (int p = pa + lane; p < pae; p += 32) {
        const int64_t s = off + apos[p];
        c_colind[s] = A.colind[p];
        atomicAdd(&c_vals[s], alpha * A.vals[p]);
      }
    }
    const int pb = B.rowptr[r], pbe = B.rowptr[r + 1];
    if (b1) {
      for (int p = pb + lane; p < pbe; p += 32) {
        const int64_t s = off + bpos[p];
        c_colind[s] = B.colind[p];
        atomicAdd(&c_vals[s], B.vals[p]);
      }
    } else {
      for (int p = pb + lane; p < pbe; p += 32) {
        const int64_t s = off + bpos[p];
        c_colind[s] = B.colind[p];
        atomicAdd(&c_vals[s], beta * B.vals[p]);
      }
    }
  }
}

}  // namespace

cudaError_t launch_spadd_symbolic(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, int32_t* cnt,
                                  int32_t* apos, int32_t* bpos, int32_t* long_rows,
                                  int32_t* long_count) {
  if (A.m <= 0) return cudaSuccess;
  long long blocks = ((long long)A.m + kAddWarps - 1) / kAddWarps;
  const long long cap = (long long)ctx.num_sms * 16;
  if (blocks > cap) blocks = cap;
  k_spadd_sym_warp<<<(int)blocks, kAddWarps * 32, 0, ctx.stream>>>(A, B, cnt, apos, bpos, long_rows,
                                                                   long_count, ctx.status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)kAddCtaMax * 8;
  e = cudaFuncSetAttribute(k_spadd_sym_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // the long-row count is on the device: one wave of CTAs strides over it
  k_spadd_sym_cta<<<ctx.num_sms * 2, kAddCtaThreads, smem, ctx.stream>>>(A, B, cnt, apos, bpos, long_rows,
                                                                         long_count, ctx.status);
  return cudaGetLastError();
}

cudaError_t launch_spadd_numeric(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, double alpha,
                                 double beta, const int64_t* c_rowptr, const int32_t* apos,
                                 const int32_t* bpos, int32_t* c_colind, double* c_vals) {
  if (A.m <= 0) return cudaSuccess;
  long long blocks = ((long long)A.m * 32 + 255) / 256;
  const long long cap = (long long)ctx.num_sms * 8;
  if (blocks > cap) blocks = cap;
  k_spadd_num<<<(int)blocks, 256, 0, ctx.stream>>>(A, B, alpha, beta, c_rowptr, apos, bpos, c_colind,
                                                   c_vals);
  return cudaGetLastError();
}

}  // namespace kk
