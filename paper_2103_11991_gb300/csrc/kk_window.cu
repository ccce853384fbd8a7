// Window tier: dense accumulators over a row's column span.
//
// The paper's dense accumulator (Sec. "Standard SpGEMM Kernel": a bit vector
// for the symbolic phase, a scalar array for the numeric phase) is kept in
// shared memory here, over the window [lo, lo + W) that holds every column of
// C(i,:) (lo = the smallest first column, lo + span - 1 the largest last column
// of the B rows that A(i,:) references; rows of B must be sorted).  One warp per
// row; lanes split each B row, A entries are taken in storage order.
//
//   symbolic: set the bit of every product's column (atomicOr), then
//             nnz(C(i,:)) = popcount of the window;
//   numeric:  same bits; per-word prefix counts give every column its rank
//             (its position in the sorted row), so the column indices are
//             written straight from the bits and each product adds into the
//             dense value slot rank = prefix[w] + popc(bits[w] & below(b)).
// There is no hashing, no probing and no sort: the bit vector is the sorted
// order.  Updates of one output entry happen in A-row order without atomics
// because the columns of a sorted B row are distinct.
#include "kk_internal.h"
#include "kk_visit.cuh"

namespace kk {
namespace {

using u64 = unsigned long long;
constexpr int kWinWarps = 4;  // warps (rows in flight) per CTA
constexpr int kWinBatch = 8;  // A entries whose B loads are issued together

template <int W>
struct SymWinGeom {
  static constexpr int WORDS = W / 32;
  static constexpr int SUMS = (WORDS + 31) / 32;  // summary words: one bit per word
  // bits u32[WORDS] | sum u32[SUMS] (padded to 16 B) | ainfo int2[32]
  static constexpr size_t kSumOff = (size_t)WORDS * 4;
  static constexpr size_t kInfoOff = kSumOff + (size_t)((SUMS + 3) / 4) * 16;
  static constexpr size_t kWarpBytes = kInfoOff + 32 * 8;
};

template <int W>
struct NumWinGeom {
  static constexpr int WORDS = W / 32;
  static constexpr int SUMS = (WORDS + 31) / 32;
  // bits u32[WORDS] | sum u32[SUMS] | prefix u16[WORDS] | list u16[kWindowMaxNnz]
  // | vacc u64[kWindowMaxNnz] | ainfo int4[32]
  static constexpr size_t kSumOff = (size_t)WORDS * 4;
  static constexpr size_t kPreOff = kSumOff + (size_t)((SUMS + 3) / 4) * 16;
  static constexpr size_t kListOff = kPreOff + (size_t)WORDS * 2;
  static constexpr size_t kValOff = kListOff + (size_t)kWindowMaxNnz * 2;
  static constexpr size_t kInfoOff = kValOff + (size_t)(kWindowMaxNnz + 2) * 8;  // + spare slot
  static constexpr size_t kWarpBytes = kInfoOff + 32 * 16;
};

// Set bit o of the window and, the first time a word becomes non-empty, its
// summary bit.
__device__ __forceinline__ void window_set(uint32_t* bits, uint32_t* sum, uint32_t o) {
  const uint32_t w = o >> 5;
  const uint32_t old = atomicOr(&bits[w], 1u << (o & 31));
  if (old == 0u) atomicOr(&sum[w >> 5], 1u << (w & 31));
}

// Set the window bits of every product of row entries [pa, pe).  ainfo2 is
// the warp's staging area for (B row start, length).
template <int W>
__device__ __forceinline__ void window_set_bits(uint32_t* bits, uint32_t* sum, int2* ainfo2, int lo,
                                                int pa, int pe, const int32_t* __restrict__ acol,
                                                const int32_t* __restrict__ brp,
                                                const int32_t* __restrict__ bcol, int lane,
                                                int* status) {
  for (int p0 = pa; p0 < pe; p0 += 32) {
    const int p = p0 + lane;
    int2 info = make_int2(0, 0);
    if (p < pe) {
      const int j = acol[p];
      info.x = brp[j];
      info.y = brp[j + 1] - info.x;
    }
    ainfo2[lane] = info;
    __syncwarp();
    const int nch = min(32, pe - p0);
    const unsigned maxlen = __reduce_max_sync(0xffffffffu, (unsigned)info.y);
    int bad = 0;
    if (maxlen <= 32u) {
      for (int t0 = 0; t0 < nch; t0 += kWinBatch) {
        int cols[kWinBatch];
#pragma unroll
        for (int u = 0; u < kWinBatch; ++u) {
          cols[u] = -1;
          if (t0 + u < nch) {
            const int2 in = ainfo2[t0 + u];
            if (lane < in.y) cols[u] = bcol[in.x + lane];
          }
        }
#pragma unroll
        for (int u = 0; u < kWinBatch; ++u) {
          if (cols[u] >= 0) {
            const uint32_t o = (uint32_t)(cols[u] - lo);
            if (o < (uint32_t)W) window_set(bits, sum, o);
            else bad = 1;
          }
        }
      }
    } else {
      for (int t = 0; t < nch; ++t) {
        const int2 in = ainfo2[t];
        for (int q = lane; q < in.y; q += 32) {
          const uint32_t o = (uint32_t)(bcol[in.x + q] - lo);
          if (o < (uint32_t)W) window_set(bits, sum, o);
          else bad = 1;
        }
      }
    }
    if (bad) set_status(status, KK_ERR_CAPACITY);
    __syncwarp();
  }
}

// Value pass of a compact row (columns of the lane's products in pcol[],
// -1 where the lane has no product).  Ranks are computed for a whole batch
// before the updates; lanes without a product update a spare slot
// (kWindowMaxNnz) instead of branching, so the update path does not diverge.
template <int W, bool DFM>
__device__ __forceinline__ void compact_values(const int (&pcol)[32], const int4* ainfo, int nch,
                                               int lo, const uint32_t* bits, const uint16_t* pre,
                                               u64* vacc, const float2* __restrict__ bspl,
                                               const double* __restrict__ bval, int lane) {
  constexpr int WORDS = W / 32;
#pragma unroll
  for (int t0 = 0; t0 < 32; t0 += kWinBatch) {
    if (t0 < nch) {
      float2 bv[kWinBatch];
      int rk[kWinBatch];
#pragma unroll
      for (int u = 0; u < kWinBatch; ++u) {
        const int c = pcol[t0 + u];
        const bool ok = c >= 0;
        const int q = ainfo[t0 + u].x + lane;
        if (DFM) {
          bv[u] = ok ? bspl[q] : make_float2(0.f, 0.f);
        } else {
          const long long bb = ok ? __double_as_longlong(bval[q]) : 0ll;
          bv[u] = make_float2(__int_as_float((int)(bb & 0xffffffffll)), __int_as_float((int)(bb >> 32)));
        }
        const uint32_t o = ok ? (uint32_t)(c - lo) : 0u;
        const uint32_t w = min(o >> 5, (uint32_t)(WORDS - 1));
        const int r = (int)pre[w] + __popc(bits[w] & ((1u << (o & 31)) - 1u));
        rk[u] = (ok && o < (uint32_t)W) ? min(r, kWindowMaxNnz) : kWindowMaxNnz;
      }
#pragma unroll
      for (int u = 0; u < kWinBatch; ++u) {
        if (t0 + u < nch) {
          const int2 az = *reinterpret_cast<const int2*>(&ainfo[t0 + u].z);
          if (DFM) {
            DF a, b;
            a.hi = __int_as_float(az.x);
            a.lo = __int_as_float(az.y);
            b.hi = bv[u].x;
            b.lo = bv[u].y;
            DF acc = df_unpack(vacc[rk[u]]);
            df_fma(acc, a, b);
            vacc[rk[u]] = df_pack(acc);
          } else {
            const double a = __longlong_as_double(((long long)az.y << 32) | (unsigned)az.x);
            const double b = __longlong_as_double(((long long)__float_as_int(bv[u].y) << 32) |
                                                  (unsigned)__float_as_int(bv[u].x));
            double* v = reinterpret_cast<double*>(&vacc[rk[u]]);
            *v = fma(a, b, *v);
          }
          __syncwarp();  // this A entry's updates are visible before the next one's
        }
      }
    }
  }
}

template <int W>
__global__ void __launch_bounds__(kWinWarps * 32, 8)
k_sym_window(CsrView A, CsrView B, const int32_t* __restrict__ row_lo,
             const int32_t* __restrict__ rows, int32_t nrows, int32_t* __restrict__ cnt,
             int* status) {
  using G = SymWinGeom<W>;
  constexpr int WORDS = G::WORDS;
  constexpr int SUMS = G::SUMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * G::kWarpBytes;
  uint32_t* bits = reinterpret_cast<uint32_t*>(base);
  uint32_t* sum = reinterpret_cast<uint32_t*>(base + G::kSumOff);
  int2* ainfo2 = reinterpret_cast<int2*>(base + G::kInfoOff);
  // whole window cleared once; afterwards each row clears only what it set
  for (int w = lane * 4; w < WORDS; w += 128)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int w = lane; w < SUMS; w += 32) sum[w] = 0u;
  __syncwarp();
  const int per_cta = (nrows + gridDim.x - 1) / gridDim.x;
  const int r_begin = blockIdx.x * per_cta;
  const int r_end = min(nrows, r_begin + per_cta);
  for (int r = r_begin + warp; r < r_end; r += kWinWarps) {
    const int i = rows[r];
    const int lo = row_lo[i];
    window_set_bits<W>(bits, sum, ainfo2, lo, A.rowptr[i], A.rowptr[i + 1], A.colind, B.rowptr,
                       B.colind, lane, status);
    int c = 0;
    for (int sw = lane; sw < SUMS; sw += 32) {
      uint32_t m = sum[sw];
      sum[sw] = 0u;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int w = sw * 32 + b;
        c += __popc(bits[w]);
        bits[w] = 0u;
      }
    }
    c = team_sum<32>(c, 0xffffffffu);
    if (lane == 0) cnt[i] = c;
    __syncwarp();
  }
}

// SPEC = true: speculative one-pass of the learned form.  c_rowptr then holds
// staging offsets, c_colind / c_vals the staging arrays, cap[i] the row's
// predicted capacity; a row with more columns than its capacity overflows
// (cnt_out[i] = -1, re-run by the plain path), otherwise cnt_out[i] = nnz.
template <int W, bool SPEC>
__global__ void __launch_bounds__(kWinWarps * 32, 4)
k_num_window(CsrView A, CsrView B, const int32_t* __restrict__ row_lo, const float2* __restrict__ bspl,
             const int32_t* __restrict__ b_range_bad, int32_t arith,
             const int64_t* __restrict__ c_rowptr, const int32_t* __restrict__ rows, int32_t nrows,
             int32_t* __restrict__ c_colind, double* __restrict__ c_vals, int* status,
             const int32_t* __restrict__ cap, int32_t* __restrict__ cnt_out) {
  using G = NumWinGeom<W>;
  constexpr int WORDS = G::WORDS;
  constexpr int SUMS = G::SUMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * G::kWarpBytes;
  uint32_t* bits = reinterpret_cast<uint32_t*>(base);
  uint32_t* sum = reinterpret_cast<uint32_t*>(base + G::kSumOff);
  uint16_t* pre = reinterpret_cast<uint16_t*>(base + G::kPreOff);
  uint16_t* list = reinterpret_cast<uint16_t*>(base + G::kListOff);
  u64* vacc = reinterpret_cast<u64*>(base + G::kValOff);
  int4* ainfo = reinterpret_cast<int4*>(base + G::kInfoOff);
  int2* ainfo2 = reinterpret_cast<int2*>(base + G::kInfoOff);
  const bool df_all = arith == kArithDF32 && *b_range_bad == 0;
  const int32_t* __restrict__ acol = A.colind;
  const double* __restrict__ aval = A.vals;
  const int32_t* __restrict__ brp = B.rowptr;
  const int32_t* __restrict__ bcol = B.colind;
  const double* __restrict__ bval = B.vals;
  for (int w = lane * 4; w < WORDS; w += 128)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int w = lane; w < SUMS; w += 32) sum[w] = 0u;
  __syncwarp();
  const int per_cta = (nrows + gridDim.x - 1) / gridDim.x;
  const int r_begin = blockIdx.x * per_cta;
  const int r_end = min(nrows, r_begin + per_cta);
  for (int r = r_begin + warp; r < r_end; r += kWinWarps) {
    const int i = rows[r];
    const int lo = row_lo[i];
    const int64_t off = c_rowptr[i];
    const int cnt = SPEC ? min(cap[i], kWindowMaxNnz) : (int)(c_rowptr[i + 1] - off);
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    for (int e = lane; e < kWindowMaxNnz; e += 32) vacc[e] = 0ull;
    // Compact rows (at most 32 A entries, every B row at most 32 long): each
    // lane keeps the columns of its products in registers for both passes.
    int4 cinfo = make_int4(0, 0, 0, 0);
    if (pa + lane < pe) {
      const int j = acol[pa + lane];
      cinfo.x = brp[j];
      cinfo.y = brp[j + 1] - cinfo.x;
    }
    const bool compact =
        (pe - pa <= 32) && __reduce_max_sync(0xffffffffu, (unsigned)cinfo.y) <= 32u;
    int pcol[32];
    if (compact) {
      ainfo2[lane] = make_int2(cinfo.x, cinfo.y);
      __syncwarp();
      const int nch = pe - pa;
      int bad = 0;
#pragma unroll
      for (int t0 = 0; t0 < 32; t0 += kWinBatch) {
        if (t0 < nch) {
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) {
            pcol[t0 + u] = -1;
            if (t0 + u < nch) {
              const int2 in = ainfo2[t0 + u];
              if (lane < in.y) pcol[t0 + u] = bcol[in.x + lane];
            }
          }
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) {
            if (pcol[t0 + u] >= 0) {
              const uint32_t o = (uint32_t)(pcol[t0 + u] - lo);
              if (o < (uint32_t)W) window_set(bits, sum, o);
              else bad = 1;
            }
          }
        } else {
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) pcol[t0 + u] = -1;
        }
      }
      if (bad) set_status(status, KK_ERR_CAPACITY);
      __syncwarp();
    } else {
      // pass 1: structure bits (and summary bits of the non-empty words)
      window_set_bits<W>(bits, sum, ainfo2, lo, pa, pe, acol, brp, bcol, lane, status);
    }
    // ordered list of non-empty words (summary words in order, bits in order)
    int nsum[(SUMS + 31) / 32];
    int mine = 0;
#pragma unroll
    for (int k = 0; k < (SUMS + 31) / 32; ++k) {
      const int sw = k * 32 + lane;
      nsum[k] = sw < SUMS ? __popc(sum[sw]) : 0;
      mine += nsum[k];
    }
    // lane-major order is not word order when SUMS > 32: scan per round
    int carry = 0;
#pragma unroll
    for (int k = 0; k < (SUMS + 31) / 32; ++k) {
      const int sw = k * 32 + lane;
      const int incl = team_inclusive_scan<32>(nsum[k], lane, 0xffffffffu);
      int pos = carry + incl - nsum[k];
      carry += __shfl_sync(0xffffffffu, incl, 31);
      if (sw < SUMS) {
        uint32_t m = sum[sw];
        sum[sw] = 0u;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          if (pos < kWindowMaxNnz) list[pos] = (uint16_t)(sw * 32 + b);
          ++pos;
        }
      }
    }
    (void)mine;
    const int L = min(carry, kWindowMaxNnz);
    __syncwarp();
    // prefix counts of the listed words, column indices written from the bits
    int run = 0;
    for (int e0 = 0; e0 < L; e0 += 32) {
      const int e = e0 + lane;
      const int w = e < L ? (int)list[e] : 0;
      const uint32_t word = e < L ? bits[w] : 0u;
      const int c = __popc(word);
      const int incl = team_inclusive_scan<32>(c, lane, 0xffffffffu);
      int pos = run + incl - c;
      run += __shfl_sync(0xffffffffu, incl, 31);
      if (e < L) {
        pre[w] = (uint16_t)pos;
        uint32_t m = word;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          if (pos < cnt) c_colind[off + pos] = lo + w * 32 + b;
          ++pos;
        }
      }
    }
    if (!SPEC && run != cnt && lane == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    if (SPEC) {
      if (run > cnt) {  // overflow: abandon the row, clear what it set
        if (lane == 0) cnt_out[i] = -1;
        if (carry > kWindowMaxNnz) {
          for (int w = lane * 4; w < WORDS; w += 128)
            *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
        } else {
          for (int e = lane; e < L; e += 32) bits[list[e]] = 0u;
        }
        __syncwarp();
        continue;
      }
      if (lane == 0) cnt_out[i] = run;
    }
    __syncwarp();
    // arithmetic of this row: DF32 unless a value of the row is outside its window
    bool df = df_all;
    if (df_all) {
      int bad = 0;
      for (int p = pa + lane; p < pe; p += 32) {
        DF t;
        bad |= df_split(aval[p], t) ? 0 : 1;
      }
      df = __any_sync(0xffffffffu, bad) == 0;
    }
    // pass 2: values; rank = prefix + popc(bits below the column)
    if (compact) {
      int4 info = make_int4(cinfo.x, cinfo.y, 0, 0);
      if (pa + lane < pe) {
        const double a = aval[pa + lane];
        if (df) {
          DF ad;
          df_split(a, ad);
          info.z = __float_as_int(ad.hi);
          info.w = __float_as_int(ad.lo);
        } else {
          const long long ab = __double_as_longlong(a);
          info.z = (int)(ab & 0xffffffffll);
          info.w = (int)(ab >> 32);
        }
      }
      ainfo[lane] = info;
      __syncwarp();
      const int nch = pe - pa;
      if (df) compact_values<W, true>(pcol, ainfo, nch, lo, bits, pre, vacc, bspl, bval, lane);
      else compact_values<W, false>(pcol, ainfo, nch, lo, bits, pre, vacc, bspl, bval, lane);
    }
    for (int p0 = pa; p0 < (compact ? pa : pe); p0 += 32) {
      const int p = p0 + lane;
      int4 info = make_int4(0, 0, 0, 0);
      if (p < pe) {
        const int j = acol[p];
        info.x = brp[j];
        info.y = brp[j + 1] - info.x;
        const double a = aval[p];
        if (df) {
          DF ad;
          df_split(a, ad);
          info.z = __float_as_int(ad.hi);
          info.w = __float_as_int(ad.lo);
        } else {
          const long long ab = __double_as_longlong(a);
          info.z = (int)(ab & 0xffffffffll);
          info.w = (int)(ab >> 32);
        }
      }
      ainfo[lane] = info;
      __syncwarp();
      const int nch = min(32, pe - p0);
      const unsigned maxlen = __reduce_max_sync(0xffffffffu, (unsigned)info.y);
      if (maxlen <= 32u) {
        for (int t0 = 0; t0 < nch; t0 += kWinBatch) {
          int cols[kWinBatch];
          float2 bv[kWinBatch];
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) {
            cols[u] = -1;
            bv[u] = make_float2(0.f, 0.f);
            if (t0 + u < nch) {
              const int2 in = *reinterpret_cast<const int2*>(&ainfo[t0 + u]);
              if (lane < in.y) {
                const int q = in.x + lane;
                cols[u] = bcol[q];
                if (df) {
                  bv[u] = bspl[q];
                } else {
                  const long long bb = __double_as_longlong(bval[q]);
                  bv[u] = make_float2(__int_as_float((int)(bb & 0xffffffffll)), __int_as_float((int)(bb >> 32)));
                }
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) {
            if (t0 + u < nch) {
              if (cols[u] >= 0) {
                const uint32_t o = (uint32_t)(cols[u] - lo);
                if (o < (uint32_t)W) {
                  const int rank = (int)pre[o >> 5] + __popc(bits[o >> 5] & ((1u << (o & 31)) - 1u));
                  if (rank < kWindowMaxNnz) {
                    const int2 az = *reinterpret_cast<const int2*>(&ainfo[t0 + u].z);
                    if (df) {
                      DF a, b;
                      a.hi = __int_as_float(az.x);
                      a.lo = __int_as_float(az.y);
                      b.hi = bv[u].x;
                      b.lo = bv[u].y;
                      DF s = df_unpack(vacc[rank]);
                      df_fma(s, a, b);
                      vacc[rank] = df_pack(s);
                    } else {
                      const double a = __longlong_as_double(((long long)az.y << 32) | (unsigned)az.x);
                      const double b = __longlong_as_double(((long long)__float_as_int(bv[u].y) << 32) |
                                                            (unsigned)__float_as_int(bv[u].x));
                      double* v = reinterpret_cast<double*>(&vacc[rank]);
                      *v = fma(a, b, *v);
                    }
                  }
                }
              }
              __syncwarp();  // this A entry's updates are visible before the next one's
            }
          }
        }
      } else {
        for (int t = 0; t < nch; ++t) {
          const int4 in = ainfo[t];
          for (int q = lane; q < in.y; q += 32) {
            const int qq = in.x + q;
            const uint32_t o = (uint32_t)(bcol[qq] - lo);
            if (o >= (uint32_t)W) continue;
            const int rank = (int)pre[o >> 5] + __popc(bits[o >> 5] & ((1u << (o & 31)) - 1u));
            if (rank >= kWindowMaxNnz) continue;
            if (df) {
              DF a, b;
              a.hi = __int_as_float(in.z);
              a.lo = __int_as_float(in.w);
              const float2 bb = bspl[qq];
              b.hi = bb.x;
              b.lo = bb.y;
              DF s = df_unpack(vacc[rank]);
              df_fma(s, a, b);
              vacc[rank] = df_pack(s);
            } else {
              const double a = __longlong_as_double(((long long)in.w << 32) | (unsigned)in.z);
              double* v = reinterpret_cast<double*>(&vacc[rank]);
              *v = fma(a, bval[qq], *v);
            }
          }
          __syncwarp();  // this A entry's updates are visible before the next one's
        }
      }
      __syncwarp();
    }
    const int n = min(SPEC ? run : cnt, kWindowMaxNnz);
    for (int e = lane; e < n; e += 32) {
      const u64 v = vacc[e];
      c_vals[off + e] = df ? df_to_double(df_unpack(v)) : __longlong_as_double((long long)v);
    }
    // clear the words this row set (listed) for the next row
    for (int e = lane; e < L; e += 32) bits[list[e]] = 0u;
    __syncwarp();
  }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

int grid_for_rows(const LaunchCtx& ctx, int nrows) {
  long long blocks = (nrows + kWinWarps * 4 - 1) / (kWinWarps * 4);
  const long long cap = (long long)ctx.num_sms * 32;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <int W>
cudaError_t sym_window(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                       const int32_t* rows, int32_t nrows, int32_t* cnt) {
  const size_t smem = (size_t)kWinWarps * SymWinGeom<W>::kWarpBytes;
  auto kern = k_sym_window<W>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid_for_rows(ctx, nrows), kWinWarps * 32, smem, ctx.stream>>>(A, B, ctx.row_lo, rows,
                                                                        nrows, cnt, ctx.status);
  return cudaGetLastError();
}

template <int W, bool SPEC = false>
cudaError_t num_window(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                       const float2* b_split, const int32_t* b_range_bad, int32_t arith,
                       const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                       int32_t* c_colind, double* c_vals, const int32_t* cap = nullptr,
                       int32_t* cnt_out = nullptr) {
  const size_t smem = (size_t)kWinWarps * NumWinGeom<W>::kWarpBytes;
  auto kern = k_num_window<W, SPEC>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<grid_for_rows(ctx, nrows), kWinWarps * 32, smem, ctx.stream>>>(
      A, B, ctx.row_lo, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals,
      ctx.status, cap, cnt_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_symbolic_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                   const CsrView& B, const int32_t* rows, int32_t nrows,
                                   int32_t* cnt) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "sym_window");
  cudaError_t e = cudaErrorInvalidValue;
  switch (bin.slots) {
    case 4096: e = sym_window<4096>(ctx, A, B, rows, nrows, cnt); break;
    case 12288: e = sym_window<12288>(ctx, A, B, rows, nrows, cnt); break;
    case 24576: e = sym_window<24576>(ctx, A, B, rows, nrows, cnt); break;
    case 40960: e = sym_window<40960>(ctx, A, B, rows, nrows, cnt); break;
    case 65536: e = sym_window<65536>(ctx, A, B, rows, nrows, cnt); break;
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

cudaError_t launch_numeric_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                  const CsrView& B, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith,
                                  const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                  int32_t* c_colind, double* c_vals) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "num_window");
  cudaError_t e = cudaErrorInvalidValue;
  switch (bin.slots) {
    case 4096: e = num_window<4096>(ctx, A, B, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals); break;
    case 12288: e = num_window<12288>(ctx, A, B, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals); break;
    case 24576: e = num_window<24576>(ctx, A, B, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals); break;
    case 40960: e = num_window<40960>(ctx, A, B, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals); break;
    case 65536: e = num_window<65536>(ctx, A, B, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals); break;
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

}  // namespace kk

namespace kk {

cudaError_t launch_onepass_window(const LaunchCtx& ctx, int32_t wclass, const CsrView& A,
                                  const CsrView& B, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith, const int64_t* soff,
                                  const int32_t* cap, const int32_t* rows, int32_t nrows,
                                  int32_t* scol, double* sval, int32_t* cnt_out) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "onepass_window");
  cudaError_t e = cudaErrorInvalidValue;
  switch (kWindowBits[wclass]) {
    case 4096: e = num_window<4096, true>(ctx, A, B, b_split, b_range_bad, arith, soff, rows, nrows, scol, sval, cap, cnt_out); break;
    case 12288: e = num_window<12288, true>(ctx, A, B, b_split, b_range_bad, arith, soff, rows, nrows, scol, sval, cap, cnt_out); break;
    case 24576: e = num_window<24576, true>(ctx, A, B, b_split, b_range_bad, arith, soff, rows, nrows, scol, sval, cap, cnt_out); break;
    case 40960: e = num_window<40960, true>(ctx, A, B, b_split, b_range_bad, arith, soff, rows, nrows, scol, sval, cap, cnt_out); break;
    case 65536: e = num_window<65536, true>(ctx, A, B, b_split, b_range_bad, arith, soff, rows, nrows, scol, sval, cap, cnt_out); break;
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

}  // namespace kk
