// Speculative one-pass of the learned form for window rows: structure and
// values of a row in one kernel, written to a staging area of the row's
// predicted capacity.
//
// The row's compressed B rows (the paper's B_C: (column >> 5, 32-bit mask)
// pairs) are inserted into a 256-slot word table (slot = word mod 256, linear
// probing, masks ORed), with one presence bit per word to list the words in
// column order; the words' prefix counts give the row's columns and the rank
// of every product, and the value pass is the one of the kept-structure
// numeric kernel (kk_kept.cuh).  A row with more distinct columns than its
// predicted capacity (or more words than the table holds) overflows: its
// count is -1 and the plain two-phase path computes it (the speculate /
// detect / redo pattern of the paper's Sec. "Distance-1 Graph Coloring").
// About 5.4 KB of shared memory per warp, whatever the row's span.
#include "kk_internal.h"
#include "kk_kept.cuh"

namespace kk {
namespace {

using u64 = unsigned long long;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kOpWarps = 8;
constexpr int kOpPresWords = 68;              // presence bits of up to 2176 words
constexpr int kOpMaxWords = kOpPresWords * 32;  // a 65,536-column window spans 2049 words

constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }
struct OpGeom {
  // table u64[256] | vacc u64[kWindowMaxNnz + 2] | ainfo int4[32] | pres u32[68] | list u16[256]
  static constexpr size_t kValOff = (size_t)kKeptSlots * 8;
  static constexpr size_t kInfoOff = al16(kValOff + (size_t)(kWindowMaxNnz + 2) * 8);
  static constexpr size_t kPresOff = kInfoOff + 32 * 16;
  static constexpr size_t kListOff = al16(kPresOff + (size_t)kOpPresWords * 4);
  static constexpr size_t kWarpBytes = al16(kListOff + (size_t)kKeptSlots * 2);
};

// Insert the pair (word w, bits m); returns 0 when the table has no room.
__device__ __forceinline__ int op_insert(u64* table, uint32_t* pres, uint32_t w, uint32_t m,
                                         int& probe) {
  uint32_t s = w & (kKeptSlots - 1);
  for (int k = 0; k < kKeptSlots; ++k) {
    u64 e = table[s];
    if (e == kKeptEmpty) {
      const u64 prev = atomicCAS(&table[s], kKeptEmpty, ((u64)w << 48) | m);
      if (prev == kKeptEmpty) {
        atomicOr(&pres[w >> 5], 1u << (w & 31));
        return 1;
      }
      e = prev;
    }
    if ((uint32_t)(e >> 48) == w) {
      atomicOr(&table[s], (u64)m);
      return 1;
    }
    probe = 1;
    s = (s + 1) & (kKeptSlots - 1);
  }
  return 0;
}

__global__ void __launch_bounds__(kOpWarps * 32, 4)
k_onepass_table(CsrView A, CsrView B, BComp bcomp, const int32_t* __restrict__ row_lo,
                const float2* __restrict__ bspl, const int32_t* __restrict__ b_range_bad,
                int32_t arith, const int64_t* __restrict__ soff, const int32_t* __restrict__ cap,
                const int32_t* __restrict__ rows, int32_t nrows, int32_t* __restrict__ scol,
                double* __restrict__ sval, int32_t* __restrict__ cnt_out, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * OpGeom::kWarpBytes;
  u64* table = reinterpret_cast<u64*>(base);
  u64* vacc = reinterpret_cast<u64*>(base + OpGeom::kValOff);
  int4* ainfo = reinterpret_cast<int4*>(base + OpGeom::kInfoOff);
  uint32_t* pres = reinterpret_cast<uint32_t*>(base + OpGeom::kPresOff);
  uint16_t* list = reinterpret_cast<uint16_t*>(base + OpGeom::kListOff);
  const bool df_all = arith == kArithDF32 && *b_range_bad == 0;
  for (int s = lane; s < kKeptSlots; s += 32) table[s] = kKeptEmpty;
  for (int s = lane; s < kOpPresWords; s += 32) pres[s] = 0u;
  __syncwarp();
  const int nw = gridDim.x * kOpWarps;  // rows dealt round-robin over the grid
  for (int r = blockIdx.x * kOpWarps + warp; r < nrows; r += nw) {
    const int i = rows[r];
    const int lo_w = row_lo[i] >> 5;
    const int lo_c = lo_w * 32;
    const int64_t off = soff[i];
    const int capi = min(cap[i], kWindowMaxNnz);
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    int full = 0, probe = 0;
    // 1. structure: OR the compressed B rows into the word table
    for (int p0 = pa; p0 < pe; p0 += 32) {
      const int p = p0 + lane;
      int x = 0, y = 0;
      if (p < pe) {
        const int j = A.colind[p];
        x = B.rowptr[j];
        y = bcomp.len[j];
      }
      const int nch = min(32, pe - p0);
      const unsigned maxlen = __reduce_max_sync(kFull, (unsigned)y);
      if (maxlen <= 16u) {
        const int lg = maxlen <= 1u ? 0 : maxlen <= 2u ? 1 : maxlen <= 4u ? 2 : maxlen <= 8u ? 3 : 4;
        const int per = 32 >> lg;
        const int sub = lane >> lg, e = lane & ((1 << lg) - 1);
        for (int t0 = 0; t0 < nch; t0 += 4 * per) {
          int2 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * per + sub;
            const int xs = __shfl_sync(kFull, x, t & 31);
            const int ys = __shfl_sync(kFull, y, t & 31);
            v[u] = make_int2(0, 0);
            if (t < nch && e < ys) v[u] = bcomp.bc[xs + e];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (v[u].y != 0) {
              const uint32_t w = (uint32_t)(v[u].x - lo_w);
              if (w >= (uint32_t)kOpMaxWords || !op_insert(table, pres, w, (uint32_t)v[u].y, probe))
                full = 1;
            }
          }
        }
      } else {
        for (int t = 0; t < nch; ++t) {
          const int xs = __shfl_sync(kFull, x, t);
          const int ys = __shfl_sync(kFull, y, t);
          for (int e = lane; e < ys; e += 32) {
            const int2 v = bcomp.bc[xs + e];
            const uint32_t w = (uint32_t)(v.x - lo_w);
            if (w >= (uint32_t)kOpMaxWords || !op_insert(table, pres, w, (uint32_t)v.y, probe))
              full = 1;
          }
        }
      }
    }
    __syncwarp();
    full = __any_sync(kFull, full);
    probe = __any_sync(kFull, probe);
    // 2. the row's words in column order (presence bits, cleared as listed)
    int L = 0;
#pragma unroll
    for (int k = 0; k < (kOpPresWords + 31) / 32; ++k) {
      const int sw = k * 32 + lane;
      uint32_t m = sw < kOpPresWords ? pres[sw] : 0u;
      const int c = __popc(m);
      const int incl = team_inclusive_scan<32>(c, lane, kFull);
      int pos = L + incl - c;
      L += __shfl_sync(kFull, incl, 31);
      if (sw < kOpPresWords) pres[sw] = 0u;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        if (pos < kKeptSlots) list[pos] = (uint16_t)(sw * 32 + b);
        ++pos;
      }
    }
    __syncwarp();
    const int Lk = min(L, kKeptSlots);
    // 3. prefix counts, columns, prefix stored with each word
    int run = 0;
    for (int e0 = 0; e0 < Lk; e0 += 32) {
      const int e = e0 + lane;
      uint32_t w = 0u, m = 0u, s = 0u;
      if (e < Lk) {
        w = list[e];
        s = w & (kKeptSlots - 1);
        u64 ent = table[s];
        for (int k = 0; k < kKeptSlots && (uint32_t)(ent >> 48) != w; ++k) {
          s = (s + 1) & (kKeptSlots - 1);
          ent = table[s];
        }
        m = (uint32_t)ent;
      }
      const int c = __popc(m);
      const int incl = team_inclusive_scan<32>(c, lane, kFull);
      int pos = run + incl - c;
      run += __shfl_sync(kFull, incl, 31);
      if (e < Lk) {
        table[s] = ((u64)w << 48) | ((u64)(uint32_t)pos << 32) | m;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          if (pos < capi) scol[off + pos] = lo_c + (int)w * 32 + b;
          ++pos;
        }
      }
    }
    __syncwarp();
    const bool over = full || run > capi;
    if (lane == 0) cnt_out[i] = over ? -1 : run;
    if (!over) {
      for (int e = lane; e < run; e += 32) vacc[e] = 0ull;
      __syncwarp();
      int missing = 0;
      const bool df =
          probe ? kept_values<true, true>(pa, pe, df_all, A, i, B.rowptr, ainfo, lo_c, table,
                                    vacc, B.colind, bspl, B.vals, lane, missing)
                : kept_values<false, true>(pa, pe, df_all, A, i, B.rowptr, ainfo, lo_c, table,
                                     vacc, B.colind, bspl, B.vals, lane, missing);
      for (int e = lane; e < run; e += 32) {
        const u64 v = vacc[e];
        sval[off + e] = df ? df_to_double(df_unpack(v)) : __longlong_as_double((long long)v);
      }
    }
    // 4. empty the table for the next row: without collisions every word sits
    // in its home slot
    if (full || probe) {
      for (int s = lane; s < kKeptSlots; s += 32) table[s] = kKeptEmpty;
    } else {
      for (int e = lane; e < Lk; e += 32) table[list[e] & (kKeptSlots - 1)] = kKeptEmpty;
    }
    __syncwarp();
  }
  (void)status;
}

}  // namespace

cudaError_t launch_onepass_table(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                 const BComp& bcomp, const float2* b_split,
                                 const int32_t* b_range_bad, int32_t arith, const int64_t* soff,
                                 const int32_t* cap, const int32_t* rows, int32_t nrows,
                                 int32_t* scol, double* sval, int32_t* cnt_out) {
  if (nrows <= 0) return cudaSuccess;
  if (!bcomp.bc || !bcomp.len) return cudaErrorInvalidValue;
  timer_begin(ctx.timer, ctx.stream, "onepass_table");
  const size_t smem = (size_t)kOpWarps * OpGeom::kWarpBytes;
  cudaError_t e = cudaFuncSetAttribute(k_onepass_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    long long blocks = (nrows + kOpWarps * 4 - 1) / (kOpWarps * 4);
    const long long capb = (long long)ctx.num_sms * 16;
    if (blocks > capb) blocks = capb;
    if (blocks < 1) blocks = 1;
    k_onepass_table<<<(int)blocks, kOpWarps * 32, smem, ctx.stream>>>(
        A, B, bcomp, ctx.row_lo, b_split, b_range_bad, arith, soff, cap, rows, nrows, scol, sval,
        cnt_out, ctx.status);
    e = cudaGetLastError();
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

}  // namespace kk
