// Value pass of the window rows through a small word table (shared by the
// kept-structure numeric kernel and the learned one-pass kernel).
//
// A row's non-empty 32-column words (index relative to the word of its first
// column) sit in a 256-slot open-addressing table, slot = word mod 256, one
// u64 per word: bits (low 32), the word's prefix count (bits 32..47) and the
// word index (48..63).  A product's slot in the row's value array is its rank:
// prefix + popc(bits below the column).  Values are DF32 pairs (or float64),
// updated in A-row storage order without atomics.
#pragma once

#include "kk_internal.h"
#include "kk_rowops.cuh"

namespace kk {
namespace {

constexpr int kKeptSlots = 256;
constexpr unsigned long long kKeptEmpty = ~0ull;
// A entries whose B loads are issued together: 3 keeps the kernel within 40
// registers (six 256-thread CTAs per SM); measured on the 27-point product in
// float64 against 2, 4 and 5 (1.90 ms against 1.90, 1.98 and 2.23) and 8.
constexpr int kKeptBatch = 3;

// Rank of column o (relative to the row's first word) through the table, or
// the spare slot kWindowMaxNnz when o is not a column of the row.  CHECK =
// false trusts that o is a column of the row (the caller has verified the
// structure otherwise); the rank is still clamped to the spare slot.
template <bool PROBE, bool CHECK>
__device__ __forceinline__ int kept_rank(const unsigned long long* table, uint32_t o, bool ok, int& missing) {
  const uint32_t w = o >> 5;
  uint32_t s = w & (kKeptSlots - 1);
  unsigned long long e = table[s];
  if (PROBE) {
    for (int k = 0; k < kKeptSlots && e != kKeptEmpty && (uint32_t)(e >> 48) != w; ++k) {
      s = (s + 1) & (kKeptSlots - 1);
      e = table[s];
    }
  }
  const uint32_t word = (uint32_t)e;
  bool member = ok;
  if (CHECK) {
    member = ok && (uint32_t)(e >> 48) == w && ((word >> (o & 31)) & 1u);
    if (ok && !member) missing = 1;
  }
  const int r = (int)((e >> 32) & 0xFFFFu) + __popc(word & ((1u << (o & 31)) - 1u));
  return member ? min(r, kWindowMaxNnz) : kWindowMaxNnz;
}

// One batch of NB A entries of a chunk (ainfo: B row start and length, A
// value as two 32-bit halves; entries past the chunk have length 0): every
// lane loads its products of the batch and ranks them, then the batch's
// updates go in entry order; lanes without a product update the spare slot,
// so nothing branches per entry.
template <int NB, bool DFM, bool PROBE, bool CHECK>
__device__ __forceinline__ void kept_batch(const int4* ainfo, int t0, int lo_c, const unsigned long long* table,
                                           unsigned long long* vacc, const int32_t* __restrict__ bcol,
                                           const float2* __restrict__ bspl,
                                           const double* __restrict__ bval, int lane,
                                           int& missing) {
  float2 bv[NB];
  int rk[NB];
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int2 in = *reinterpret_cast<const int2*>(&ainfo[t0 + u]);
    const bool ok = lane < in.y;
    const int q = in.x + lane;
    int c = 0;
    bv[u] = make_float2(0.f, 0.f);
    if (ok) {
      c = bcol[q];
      if (DFM) {
        bv[u] = bspl[q];
      } else {
        const long long bb = __double_as_longlong(bval[q]);
        bv[u] = make_float2(__int_as_float((int)(bb & 0xffffffffll)), __int_as_float((int)(bb >> 32)));
      }
    }
    rk[u] = kept_rank<PROBE, CHECK>(table, (uint32_t)(c - lo_c), ok, missing);
  }
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int2 az = *reinterpret_cast<const int2*>(&ainfo[t0 + u].z);
    // lanes without a product (or with a column outside the kept structure)
    // skip the update and its shared-memory traffic
    if (rk[u] < kWindowMaxNnz) {
      if (DFM) {
        DF a, b;
        a.hi = __int_as_float(az.x);
        a.lo = __int_as_float(az.y);
        b.hi = bv[u].x;
        b.lo = bv[u].y;
        DF s = df_unpack(vacc[rk[u]]);
        df_fma(s, a, b);
        vacc[rk[u]] = df_pack(s);
      } else {
        const double x = __longlong_as_double(((long long)az.y << 32) | (unsigned)az.x);
        const double y = __longlong_as_double(((long long)__float_as_int(bv[u].y) << 32) |
                                              (unsigned)__float_as_int(bv[u].x));
        double* v = reinterpret_cast<double*>(&vacc[rk[u]]);
        *v = fma(x, y, *v);
      }
    }
    __syncwarp();  // this A entry's updates are visible before the next one's
  }
}

// Value pass over one chunk of at most 32 A entries: batches of kKeptBatch,
// a tail of more than 2 in one more batch (entries past the chunk have length
// 0), a tail of 1 or 2 in a batch of 2.
template <bool DFM, bool PROBE, bool CHECK>
__device__ __forceinline__ void kept_chunk(const int4* ainfo, int nch, int lo_c, const unsigned long long* table,
                                           unsigned long long* vacc, const int32_t* __restrict__ bcol,
                                           const float2* __restrict__ bspl,
                                           const double* __restrict__ bval, int lane,
                                           int& missing) {
  int t0 = 0;
  for (; t0 + kKeptBatch <= nch; t0 += kKeptBatch)
    kept_batch<kKeptBatch, DFM, PROBE, CHECK>(ainfo, t0, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
  const int rem = nch - t0;
  if (rem > 2)
    kept_batch<kKeptBatch, DFM, PROBE, CHECK>(ainfo, t0, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
  else if (rem > 0)
    kept_batch<2, DFM, PROBE, CHECK>(ainfo, t0, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
}

// Value pass for B rows longer than 32: one A entry at a time, lanes stride
// the B row.
template <bool DFM, bool PROBE, bool CHECK>
__device__ __forceinline__ void kept_chunk_long(const int4* ainfo, int nch, int lo_c,
                                                const unsigned long long* table, unsigned long long* vacc,
                                                const int32_t* __restrict__ bcol,
                                                const float2* __restrict__ bspl,
                                                const double* __restrict__ bval, int lane,
                                                int& missing) {
  for (int t = 0; t < nch; ++t) {
    const int4 in = ainfo[t];
    for (int q0 = 0; q0 < in.y; q0 += 32) {
      const int q = in.x + q0 + lane;
      const bool ok = q0 + lane < in.y;
      const int c = ok ? bcol[q] : 0;
      const int rank = kept_rank<PROBE, CHECK>(table, (uint32_t)(c - lo_c), ok, missing);
      if (rank < kWindowMaxNnz) {
        if (DFM) {
          DF a, b;
          a.hi = __int_as_float(in.z);
          a.lo = __int_as_float(in.w);
          const float2 bb = bspl[q];
          b.hi = bb.x;
          b.lo = bb.y;
          DF s = df_unpack(vacc[rank]);
          df_fma(s, a, b);
          vacc[rank] = df_pack(s);
        } else {
          const double x = __longlong_as_double(((long long)in.w << 32) | (unsigned)in.z);
          double* v = reinterpret_cast<double*>(&vacc[rank]);
          *v = fma(x, bval[q], *v);
        }
      }
      __syncwarp();
    }
  }
}

// Chunk setup: lane t holds A entry p0 + t (B row start, length, A value
// split for DF32 or as raw float64 halves).  Returns 1 if the lane's value is
// outside the DF32 window.
template <bool JAC>
__device__ __forceinline__ int kept_info(int p0, int pe, const CsrView& A, int i,
                                         const int32_t* __restrict__ brp, int lane, int4& info,
                                         DF& ad, double& a) {
  const int p = p0 + lane;
  info = make_int4(0, 0, 0, 0);
  a = 0.0;
  if (p < pe) {
    const int j = A.colind[p];
    info.x = brp[j];
    info.y = brp[j + 1] - info.x;
    a = JAC ? a_value(A, i, p) : A.vals[p];
  }
  return df_split(a, ad) ? 0 : 1;
}

template <bool PROBE, bool CHECK>
__device__ __forceinline__ void kept_store_and_run(int4 info, const DF& ad, double a, bool df,
                                                   int4* ainfo, int nch, int lo_c,
                                                   const unsigned long long* table, unsigned long long* vacc,
                                                   const int32_t* __restrict__ bcol,
                                                   const float2* __restrict__ bspl,
                                                   const double* __restrict__ bval, int lane,
                                                   int& missing) {
  if (df) {
    info.z = __float_as_int(ad.hi);
    info.w = __float_as_int(ad.lo);
  } else {
    const long long ab = __double_as_longlong(a);
    info.z = (int)(ab & 0xffffffffll);
    info.w = (int)(ab >> 32);
  }
  ainfo[lane] = info;
  __syncwarp();
  const bool shrt = __reduce_max_sync(0xffffffffu, (unsigned)info.y) <= 32u;
  if (df) {
    if (shrt) kept_chunk<true, PROBE, CHECK>(ainfo, nch, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
    else kept_chunk_long<true, PROBE, CHECK>(ainfo, nch, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
  } else {
    if (shrt) kept_chunk<false, PROBE, CHECK>(ainfo, nch, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
    else kept_chunk_long<false, PROBE, CHECK>(ainfo, nch, lo_c, table, vacc, bcol, bspl, bval, lane, missing);
  }
  __syncwarp();
}

// Value pass of a row; returns whether it ran in DF32.  Rows of at most 32 A
// entries decide the arithmetic from their own split values; longer rows
// check all their values first.
// JAC: A's values scaled for the Jacobi-fused product (a template switch so the
// plain product keeps its registers)
template <bool PROBE, bool CHECK, bool JAC = false>
__device__ __forceinline__ bool kept_values(int pa, int pe, bool df_all, const CsrView& A, int i,
                                            const int32_t* __restrict__ brp, int4* ainfo, int lo_c,
                                            const unsigned long long* table, unsigned long long* vacc,
                                            const int32_t* __restrict__ bcol,
                                            const float2* __restrict__ bspl,
                                            const double* __restrict__ bval, int lane, int& missing) {
  df_all = df_all && df_row_terms_ok(pa, pe);
  bool df = df_all;
  if (df_all && pe - pa > 32) df = row_df_ok<32>(A.vals, pa, pe, lane, 0xffffffffu);
  for (int p0 = pa; p0 < pe; p0 += 32) {
    int4 info;
    DF ad;
    double a;
    const int bad = kept_info<JAC>(p0, pe, A, i, brp, lane, info, ad, a);
    if (df_all && pe - pa <= 32) df = __any_sync(0xffffffffu, bad) == 0;
    kept_store_and_run<PROBE, CHECK>(info, ad, a, df, ainfo, min(32, pe - p0), lo_c, table, vacc, bcol,
                              bspl, bval, lane, missing);
  }
  return df;
}

}  // namespace
}  // namespace kk
