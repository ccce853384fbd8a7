// Row traversal of Gustavson's product (Kokkos Kernels paper, Eq. 1): for row i
// of A, every product A(i,j) * B(j,c) is one (A entry p, B entry q) pair.
//
// A team of TEAM lanes walks the A entries of the row in chunks of TEAM.  Two
// lane mappings (the paper's two parallelisation methods, Sec. "Standard SpGEMM
// Kernel", last paragraph):
//   - vector (FLAT = false): the A entries of a chunk are taken one after the
//     other and the lanes split the entries of the referenced B row; products
//     reach each output column in A-row storage order, so a row-private
//     accumulator needs no atomics when B's rows have distinct columns;
//   - flattened (FLAT = true): the lanes split the flattened (A entry, B entry)
//     index space of the chunk evenly, which keeps every lane busy when B's rows
//     are short; accumulation then needs atomics.
#pragma once

#include "kk_device.cuh"

namespace kk {

struct NoPayload {};

__device__ __forceinline__ NoPayload shfl_payload(unsigned, NoPayload v, int, int) { return v; }
__device__ __forceinline__ double shfl_payload(unsigned mask, double v, int src, int width) {
  return __shfl_sync(mask, v, src, width);
}
__device__ __forceinline__ DF shfl_payload(unsigned mask, DF v, int src, int width) {
  DF r;
  r.hi = __shfl_sync(mask, v.hi, src, width);
  r.lo = __shfl_sync(mask, v.lo, src, width);
  return r;
}

// Visit the products of A entries [pa, pe).  Chunks of TEAM entries are taken
// starting at chunk index first_chunk and stepping by chunk_step (so several
// teams may share one row).  For each A entry p the lane holding it calls
// range(p, bs, bl) (the B entries [bs, bs+bl) to visit) and prep(p) (a payload,
// e.g. the split value A(i,j), broadcast to the lanes that use it).  visit(pay,
// p, q) is then called exactly once per product, on some lane of the team.
template <int TEAM, bool FLAT, class Payload, class RangeFn, class PrepFn, class VisitFn>
__device__ __forceinline__ void visit_products(int pa, int pe, int first_chunk, int chunk_step,
                                               int tl, unsigned mask, RangeFn range, PrepFn prep,
                                               VisitFn visit) {
  for (int p0 = pa + first_chunk * TEAM; p0 < pe; p0 += chunk_step * TEAM) {
    const int p = p0 + tl;
    int bs = 0, bl = 0;
    Payload pay{};
    if (p < pe) {
      range(p, bs, bl);
      pay = prep(p);
    }
    if (FLAT) {
      const int incl = team_inclusive_scan<TEAM>(bl, tl, mask);
      const int total = __shfl_sync(mask, incl, TEAM - 1, TEAM);
      const int base = bs - (incl - bl);
      for (int f0 = 0; f0 < total; f0 += TEAM) {
        const int f = f0 + tl;
        int own = 0;
#pragma unroll
        for (int step = TEAM / 2; step > 0; step >>= 1) {
          const int v = __shfl_sync(mask, incl, own + step - 1, TEAM);
          if (v <= f) own += step;
        }
        const int qb = __shfl_sync(mask, base, own, TEAM);
        const Payload po = shfl_payload(mask, pay, own, TEAM);
        if (f < total) visit(po, p0 + own, qb + f);
      }
    } else {
      const int nch = min(TEAM, pe - p0);
      for (int t = 0; t < nch; ++t) {
        const int s = __shfl_sync(mask, bs, t, TEAM);
        const int l = __shfl_sync(mask, bl, t, TEAM);
        const Payload pt = shfl_payload(mask, pay, t, TEAM);
        for (int q = tl; q < l; q += TEAM) visit(pt, p0 + t, s + q);
        __syncwarp(mask);  // updates of this A entry are visible to the next one
      }
    }
  }
}

// First index in the sorted segment col[lo, hi) whose value is >= key.
__device__ __forceinline__ int lower_bound_i32(const int32_t* __restrict__ col, int lo, int hi,
                                               int32_t key) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace kk
