// Per-row helpers shared by the numeric kernels of the plain, learned and
// batched forms: B-row ranges, A-value payloads, accumulator updates, the
// team / block bitonic sorts and scans, and the DF32 / float64 output.
#pragma once

#include "kk_device.cuh"
#include "kk_internal.h"

namespace kk {

using u64 = unsigned long long;

struct FullRange {
  const int32_t* acol;
  const int32_t* brp;
  __device__ __forceinline__ void operator()(int p, int& bs, int& bl) const {
    const int j = acol[p];
    bs = brp[j];
    bl = brp[j + 1] - bs;
  }
};

// A's value at entry p of the row (row i of A; see a_value), as float64 or
// split into DF32.
struct PrepF64 {
  const double* av;
  ARowScale r;
  __device__ PrepF64(const CsrView& A, int i) : av(A.vals), r(a_row_scale(A, i)) {}
  __device__ __forceinline__ double operator()(int p) const { return a_scaled(r, p, av[p]); }
};
struct PrepDF {
  const double* av;
  ARowScale r;
  __device__ PrepDF(const CsrView& A, int i) : av(A.vals), r(a_row_scale(A, i)) {}
  __device__ __forceinline__ DF operator()(int p) const {
    DF t;
    df_split(a_scaled(r, p, av[p]), t);
    return t;
  }
};

__device__ __forceinline__ DF load_b(const float2* bs, int q) {
  const float2 v = bs[q];
  DF d;
  d.hi = v.x;
  d.lo = v.y;
  return d;
}

// Accumulate one product into slot `slot` of a u64 value array.
__device__ __forceinline__ void upd_df(u64* vals, int slot, DF a, DF b, bool atomic, int* status) {
  if (atomic) {
    df_atomic_fma(&vals[slot], a, b, status);
  } else {
    DF s = df_unpack(vals[slot]);
    df_fma(s, a, b);
    vals[slot] = df_pack(s);
  }
}
__device__ __forceinline__ void upd_f64(u64* vals, int slot, double a, double b, bool atomic) {
  double* v = reinterpret_cast<double*>(&vals[slot]);
  if (atomic) atomicAdd(v, a * b);
  else *v = fma(a, b, *v);
}

// True if every A value of the row lies in the DF32 window (team vote).
template <int TEAM>
__device__ __forceinline__ bool row_df_ok(const double* av, int pa, int pe, int tl, unsigned mask) {
  int bad = 0;
  for (int p = pa + tl; p < pe; p += TEAM) {
    DF t;
    bad |= df_split(av[p], t) ? 0 : 1;
  }
  return __any_sync(mask, bad) == 0;
}

__device__ __forceinline__ bool block_df_ok(const double* av, int pa, int pe, int* flag) {
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  for (int p = pa + threadIdx.x; p < pe; p += blockDim.x) {
    DF t;
    if (!df_split(av[p], t)) *flag = 1;
  }
  __syncthreads();
  const bool ok = *flag == 0;
  __syncthreads();
  return ok;
}

__device__ __forceinline__ double out_value(u64 v, bool df) {
  return df ? df_to_double(df_unpack(v)) : __longlong_as_double((long long)v);
}

// Bitonic sort of P (a power of two) u64 items in shared memory by a team.
template <int TEAM>
__device__ __forceinline__ void team_bitonic(u64* buf, int P, int tl, unsigned mask) {
  for (int kk = 2; kk <= P; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int t = tl; t < (P >> 1); t += TEAM) {
        const int lo = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int hi = lo + j;
        const bool up = (lo & kk) == 0;
        const u64 x = buf[lo], y = buf[hi];
        if ((x > y) == up) {
          buf[lo] = y;
          buf[hi] = x;
        }
      }
      __syncwarp(mask);
    }
  }
}

__device__ __forceinline__ void block_bitonic(u64* buf, int P) {
  for (int kk = 2; kk <= P; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const int lo = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int hi = lo + j;
        const bool up = (lo & kk) == 0;
        const u64 x = buf[lo], y = buf[hi];
        if ((x > y) == up) {
          buf[lo] = y;
          buf[hi] = x;
        }
      }
      __syncthreads();
    }
  }
}

// Exclusive scan of v over the block (blockDim.x a multiple of 32, <= 1024);
// returns this thread's prefix and the block total in *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  int incl = team_inclusive_scan<32>(v, lane, 0xffffffffu);
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? scratch[lane] : 0;
    int wi = team_inclusive_scan<32>(w, lane, 0xffffffffu);
    if (lane < nw) scratch[lane] = wi - w;
    if (lane == 31) scratch[32] = wi;
  }
  __syncthreads();
  const int r = scratch[warp] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int pow2ceil(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}


}  // namespace kk
