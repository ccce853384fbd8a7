// Window tier: dense accumulators over a row's column span.
//
// The paper's dense accumulator (Sec. "Standard SpGEMM Kernel": a bit vector
// for the symbolic phase, a scalar array for the numeric phase) is kept in
// shared memory here, over a window of 32-column words starting at the word
// that holds lo = the smallest first column of the B rows A(i,:) references
// (rows of B must be sorted, so the window spans at most W + 31 columns).  One
// warp per row.
//
//   symbolic: OR every (word, mask) pair of the compressed rows B_C(j,:)
//             (the paper's B_C, Sec. "Standard SpGEMM Kernel": columns stored
//             as bits, accumulation = bitwise OR) into the window; nnz(C(i,:))
//             is the popcount of the non-empty words, found through one
//             summary bit per word.  The row's non-empty words (up to
//             kCacheWords) are kept as its structure for the numeric phase.
//   numeric:  the words come from that structure (or are rebuilt from B_C);
//             per-word prefix counts give every column its rank (its position
//             in the sorted row), so column indices are written straight from
//             the bits and each product adds into the dense value slot
//             rank = prefix[w] + popc(bits[w] & below(b)).
// There is no hashing, no probing and no sort: the bit vector is the sorted
// order.  Updates of one output entry happen in A-row order without atomics
// because the columns of a sorted B row are distinct.
#include "kk_internal.h"
#include "kk_rowops.cuh"
#include "kk_visit.cuh"

namespace kk {
namespace {

using u64 = unsigned long long;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kWinWarps = 4;  // warps (rows in flight) per CTA
constexpr int kWinBatch = 8;  // A entries whose B loads are issued together
constexpr int kSetBatch = 8;  // groups of compressed-row loads in flight in bc_set_bits

constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Words of a W-bit window that may start anywhere inside its first word,
// padded to a multiple of 4; one summary bit per word.
template <int W>
struct WinWords {
  static constexpr int WORDS = W / 32 + 4;
  static constexpr int SUMS = (WORDS + 31) / 32;
};

template <int W>
struct SymWinGeom : WinWords<W> {
  using WinWords<W>::WORDS;
  // one mark byte per group of 32 words
  static constexpr int GROUPS = (WORDS + 31) / 32;
  // bits u32[WORDS] | gmark u8[GROUPS]
  static constexpr size_t kMarkOff = al16((size_t)WORDS * 4);
  static constexpr size_t kWarpBytes = al16(kMarkOff + (size_t)GROUPS);
};

template <int W, int VMAX = kWindowMaxNnz>
struct NumWinGeom : WinWords<W> {
  using WinWords<W>::WORDS;
  using WinWords<W>::SUMS;
  // bits u32[WORDS] | sum u32[SUMS] | prefix u16[WORDS] | list u16[VMAX]
  // | vacc u64[VMAX + 2] (the last ones: spare slot) | ainfo int4[32]
  static constexpr size_t kSumOff = al16((size_t)WORDS * 4);
  static constexpr size_t kPreOff = al16(kSumOff + (size_t)SUMS * 4);
  static constexpr size_t kListOff = al16(kPreOff + (size_t)WORDS * 2);
  static constexpr size_t kValOff = al16(kListOff + (size_t)VMAX * 2);
  static constexpr size_t kInfoOff = al16(kValOff + (size_t)(VMAX + 2) * 8);
  static constexpr size_t kWarpBytes = kInfoOff + 32 * 16;
};

// Compressed row bounds of A entry p (0, 0 past the row's end).
__device__ __forceinline__ void bc_bounds(int p, int pe, const int32_t* __restrict__ acol,
                                          const int32_t* __restrict__ brp,
                                          const int32_t* __restrict__ bclen, int& x, int& y) {
  x = 0;
  y = 0;
  if (p < pe) {
    const int j = acol[p];
    x = brp[j];
    y = bclen[j];
  }
}

// (Numeric phases: a pair outside the window means B's structure is not the
// one the symbolic phase sized the window for: KK_ERR_STRUCTURE_MISMATCH.)
// OR the compressed rows B_C(j,:) of the entries [pa, pe) of A(i,:) into the
// window whose word 0 is column word lo_w, and the word's summary bit.  Lanes
// take the pairs of 32 / G A entries at a time, G the power of two that covers
// the longest compressed row of the chunk, with the loads of SETB such groups
// in flight (the numeric kernels take 4: their register budget is tighter).  x0 / y0:
// the lane's bounds for the first chunk, already loaded (PRE), else loaded here.
template <int WORDS, bool PRE = false, int SETB = kSetBatch>
__device__ __forceinline__ void bc_set_bits(uint32_t* bits, uint32_t* sum, int lo_w, int pa, int pe,
                                            const int32_t* __restrict__ acol,
                                            const int32_t* __restrict__ brp,
                                            const int2* __restrict__ bc,
                                            const int32_t* __restrict__ bclen, int lane,
                                            int* status, int x0 = 0, int y0 = 0) {
  int bad = 0;
  for (int p0 = pa; p0 < pe; p0 += 32) {
    int x, y;
    if (PRE && p0 == pa) {
      x = x0;
      y = y0;
    } else {
      bc_bounds(p0 + lane, pe, acol, brp, bclen, x, y);
    }
    const int nch = min(32, pe - p0);
    const unsigned maxlen = __reduce_max_sync(kFull, (unsigned)y);
    if (maxlen <= 16u) {
      const int lg = maxlen <= 1u ? 0 : maxlen <= 2u ? 1 : maxlen <= 4u ? 2 : maxlen <= 8u ? 3 : 4;
      const int per = 32 >> lg;
      const int sub = lane >> lg, e = lane & ((1 << lg) - 1);
      for (int t0 = 0; t0 < nch; t0 += SETB * per) {
        int2 v[SETB];
#pragma unroll
        for (int u = 0; u < SETB; ++u) {
          const int t = t0 + u * per + sub;
          const int xs = __shfl_sync(kFull, x, t & 31);
          const int ys = __shfl_sync(kFull, y, t & 31);
          v[u] = make_int2(0, 0);
          if (t < nch && e < ys) v[u] = bc[xs + e];
        }
#pragma unroll
        for (int u = 0; u < SETB; ++u) {
          if (v[u].y != 0) {
            const uint32_t w = (uint32_t)(v[u].x - lo_w);
            if (w < (uint32_t)WORDS) {
              // no returned value to wait for: the summary bit is set every time
              atomicOr(&bits[w], (uint32_t)v[u].y);
              atomicOr(&sum[w >> 5], 1u << (w & 31));
            } else {
              bad = 1;
            }
          }
        }
      }
    } else {
      for (int t = 0; t < nch; ++t) {
        const int xs = __shfl_sync(kFull, x, t);
        const int ys = __shfl_sync(kFull, y, t);
        for (int e = lane; e < ys; e += 32) {
          const int2 v = bc[xs + e];
          const uint32_t w = (uint32_t)(v.x - lo_w);
          if (w < (uint32_t)WORDS) {
            // long compressed rows (scattered columns): only the first setter of
            // a word sets its summary bit, which keeps lanes off shared summary words
            const uint32_t old = atomicOr(&bits[w], (uint32_t)v.y);
            if (old == 0u) atomicOr(&sum[w >> 5], 1u << (w & 31));
          } else {
            bad = 1;
          }
        }
      }
    }
  }
  if (bad) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  __syncwarp();
}

// The symbolic kernel's OR of the compressed rows B_C(j,:) of A entries
// [pa, pe) into the window (word 0 = column word lo_w), with a mark byte per
// group of 32 words (plain stores: lanes that mark the same group write the
// same value).  Pairs are loaded 16 bytes (two pairs) at a time from the even
// pair index at or below the row's start (the compressed B is padded so the
// last load stays inside it), by a team of G lanes per entry with 2G covering
// the chunk's longest row span: one load instruction then fetches all of an
// entry's pairs, so it touches each entry's cache line once (the kernel was
// bound by L1 tag lookups of narrower loads that revisited the same lines).
// Two steps' loads are in flight.  Rows spanning more than 64 pairs are walked
// an entry at a time.  x0 / y0: the lane's bounds for the first chunk.
template <int WORDS>
__device__ __forceinline__ void or_pair(uint32_t* bits, uint8_t* gmark, int lo_w, int wc, uint32_t m,
                                        int& bad) {
  const uint32_t w = (uint32_t)(wc - lo_w);
  if (w < (uint32_t)WORDS) {
    atomicOr(&bits[w], m);
    gmark[w >> 5] = 1;
  } else {
    bad = 1;
  }
}

template <int WORDS>
__device__ __forceinline__ void bc_or_marked(uint32_t* bits, uint8_t* gmark, int lo_w, int pa, int pe,
                                             const int32_t* __restrict__ acol,
                                             const int32_t* __restrict__ brp,
                                             const int2* __restrict__ bc,
                                             const int32_t* __restrict__ bclen, int lane, int* status,
                                             int x0, int y0) {
  int bad = 0;
  const int4* __restrict__ bc4 = reinterpret_cast<const int4*>(bc);
  for (int p0 = pa; p0 < pe; p0 += 32) {
    int x = x0, y = y0;
    if (p0 != pa) bc_bounds(p0 + lane, pe, acol, brp, bclen, x, y);
    const int nch = min(32, pe - p0);
    // pairs to fetch from the even index below the row's start
    const unsigned span = y > 0 ? (unsigned)((x & 1) + y) : 0u;
    const unsigned maxspan = __reduce_max_sync(kFull, span);
    if (maxspan <= 64u) {
      const int lg = maxspan <= 2u ? 0 : maxspan <= 4u ? 1 : maxspan <= 8u ? 2 : maxspan <= 16u ? 3
                   : maxspan <= 32u ? 4 : 5;
      const int E = 32 >> lg;
      const int sub = lane >> lg, e2 = 2 * (lane & ((1 << lg) - 1));
      for (int t0 = 0; t0 < nch; t0 += 2 * E) {
        const int ta = t0 + sub, tb = t0 + E + sub;
        const int xa = __shfl_sync(kFull, x, ta & 31), ya = __shfl_sync(kFull, y, ta & 31);
        const int xb = __shfl_sync(kFull, x, tb & 31), yb = __shfl_sync(kFull, y, tb & 31);
        // pair indices [qa, qa + 2) of the row's [xa, xa + ya)
        const int qa = (xa & ~1) + e2, qb = (xb & ~1) + e2;
        const bool la = ta < nch && qa + 1 >= xa && qa < xa + ya;
        const bool lb = tb < nch && qb + 1 >= xb && qb < xb + yb;
        int4 va = make_int4(0, 0, 0, 0), vb = make_int4(0, 0, 0, 0);
        if (la) va = bc4[qa >> 1];
        if (lb) vb = bc4[qb >> 1];
        if (la && qa >= xa) or_pair<WORDS>(bits, gmark, lo_w, va.x, (uint32_t)va.y, bad);
        if (la && qa + 1 < xa + ya) or_pair<WORDS>(bits, gmark, lo_w, va.z, (uint32_t)va.w, bad);
        if (lb && qb >= xb) or_pair<WORDS>(bits, gmark, lo_w, vb.x, (uint32_t)vb.y, bad);
        if (lb && qb + 1 < xb + yb) or_pair<WORDS>(bits, gmark, lo_w, vb.z, (uint32_t)vb.w, bad);
      }
    } else {
      for (int t = 0; t < nch; ++t) {
        const int xs = __shfl_sync(kFull, x, t);
        const int ys = __shfl_sync(kFull, y, t);
        for (int e = lane; e < ys; e += 32) {
          const int2 v = bc[xs + e];
          or_pair<WORDS>(bits, gmark, lo_w, v.x, (uint32_t)v.y, bad);
        }
      }
    }
  }
  if (bad) set_status(status, KK_ERR_CAPACITY);
  __syncwarp();
}

// Ordered list of the window's non-empty words from the summary bits (which
// are cleared); list receives the first `cap` of them.  Returns their number.
template <int SUMS>
__device__ __forceinline__ int window_list(uint32_t* sum, uint16_t* list, int cap, int lane) {
  int carry = 0;
#pragma unroll
  for (int k = 0; k < (SUMS + 31) / 32; ++k) {
    const int sw = k * 32 + lane;
    uint32_t m = sw < SUMS ? sum[sw] : 0u;
    const int c = __popc(m);
    const int incl = team_inclusive_scan<32>(c, lane, kFull);
    int pos = carry + incl - c;
    carry += __shfl_sync(kFull, incl, 31);
    if (sw < SUMS) sum[sw] = 0u;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      if (pos < cap) list[pos] = (uint16_t)(sw * 32 + b);
      ++pos;
    }
  }
  __syncwarp();
  return carry;
}

// Popcount of the whole window, clearing it (rows with more non-empty words
// than the list holds).
template <int WORDS>
__device__ __forceinline__ int window_count_clear(uint32_t* bits, int lane) {
  int c = 0;
  for (int w = lane * 4; w < WORDS; w += 128) {
    uint4* q = reinterpret_cast<uint4*>(&bits[w]);
    const uint4 v = *q;
    c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    *q = make_uint4(0u, 0u, 0u, 0u);
  }
  return c;
}

template <int W>
__global__ void __launch_bounds__(kWinWarps * 32, 8)
k_sym_window(CsrView A, CsrView B, BComp bcomp, const int32_t* __restrict__ row_lo,
             const int32_t* __restrict__ rows, int32_t nrows, int32_t* __restrict__ cnt,
             WinCache cache, int* status) {
  using G = SymWinGeom<W>;
  constexpr int WORDS = G::WORDS;
  constexpr int GROUPS = G::GROUPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * G::kWarpBytes;
  uint32_t* bits = reinterpret_cast<uint32_t*>(base);
  uint8_t* gmark = base + G::kMarkOff;
  // whole window cleared once; afterwards each row clears what it set
  for (int w = lane * 4; w < WORDS; w += 128)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int g = lane; g < GROUPS; g += 32) gmark[g] = 0;
  __syncwarp();
  // Rows are dealt to warps round-robin over the whole grid, so the rows in
  // flight at any time are neighbours and the B rows they share stay in L2.
  const int nw = gridDim.x * kWinWarps;
  const int r_end = nrows;
  int kept = 0;
  // Rows are software-pipelined: while a row is processed, the next row's
  // bounds and then its first chunk of compressed-row bounds are loaded, so
  // the chain row id -> A row -> A columns -> B_C bounds is off the critical
  // path (the kernel is bound by those dependent loads otherwise).
  int r = blockIdx.x * kWinWarps + warp;
  int i = 0, pa = 0, pe = 0, lo = 0, x = 0, y = 0, i_n = -1;
  if (r < r_end) {
    i = rows[r];
    pa = A.rowptr[i];
    pe = A.rowptr[i + 1];
    lo = row_lo[i];
    bc_bounds(pa + lane, pe, A.colind, B.rowptr, bcomp.len, x, y);
    if (r + nw < r_end) i_n = rows[r + nw];
  }
  for (; r < r_end; r += nw) {
    int pa_n = 0, pe_n = 0, lo_n = 0;
    if (i_n >= 0) {
      pa_n = A.rowptr[i_n];
      pe_n = A.rowptr[i_n + 1];
      lo_n = row_lo[i_n];
    }
    const int i_nn = r + 2 * nw < r_end ? rows[r + 2 * nw] : -1;
    bc_or_marked<WORDS>(bits, gmark, lo >> 5, pa, pe, A.colind, B.rowptr, bcomp.bc, bcomp.len, lane, status,
                        x, y);
    int j_n = -1;
    if (i_n >= 0 && pa_n + lane < pe_n) j_n = A.colind[pa_n + lane];
    // The marked groups of 32 words in order: a lane per word of the group
    // finds the non-empty ones (ballot), counts their columns, clears them and
    // stores the word and its bits as the row's kept structure (in order).
    int c = 0, L = 0;
    {
      const unsigned below = (1u << lane) - 1u;
      uint16_t* cw = cache.w ? cache.w + (size_t)i * kCacheWords : nullptr;
      uint32_t* cm = cache.w ? cache.m + (size_t)i * kCacheWords : nullptr;
#pragma unroll
      for (int g0 = 0; g0 < GROUPS; g0 += 32) {
        const int g = g0 + lane;
        const bool mk = g < GROUPS && gmark[g] != 0;
        unsigned gm = __ballot_sync(kFull, mk);
        if (mk) gmark[g] = 0;
        while (gm) {
          const int gb = __ffs(gm) - 1;
          gm &= gm - 1;
          const int w = (g0 + gb) * 32 + lane;
          const uint32_t m = w < WORDS ? bits[w] : 0u;
          const unsigned nz = __ballot_sync(kFull, m != 0u);
          const int pos = L + __popc(nz & below);
          if (m != 0u) {
            bits[w] = 0u;
            c += __popc(m);
            if (cw && pos < kCacheWords) {
              cw[pos] = (uint16_t)w;
              cm[pos] = m;
            }
          }
          L += __popc(nz);
        }
      }
    }
    int x_n = 0, y_n = 0;
    if (j_n >= 0) {
      x_n = B.rowptr[j_n];
      y_n = bcomp.len[j_n];
    }
    c = team_sum<32>(c, kFull);
    if (lane == 0) {
      cnt[i] = c;
      if (cache.n) cache.n[i] = L <= kCacheWords ? L : -1;
    }
    kept += (cache.n && L <= kCacheWords) ? 1 : 0;
    __syncwarp();
    i = i_n;
    pa = pa_n;
    pe = pe_n;
    lo = lo_n;
    x = x_n;
    y = y_n;
    i_n = i_nn;
  }
  if (lane == 0 && kept) atomicAdd(cache.kept, (unsigned long long)kept);
}

// Rank of column o (relative to the window) from the bits and prefixes, or
// the spare slot VMAX when o is not a column of the row.
template <int WORDS, int VMAX>
__device__ __forceinline__ int window_rank(const uint32_t* bits, const uint16_t* pre, uint32_t o,
                                           bool ok, int& missing) {
  const uint32_t w = min(o >> 5, (uint32_t)(WORDS - 1));
  const uint32_t word = bits[w];
  const bool member = ok && o < (uint32_t)(WORDS * 32) && ((word >> (o & 31)) & 1u);
  if (ok && !member) missing = 1;
  const int r = (int)pre[w] + __popc(word & ((1u << (o & 31)) - 1u));
  return member ? min(r, VMAX) : VMAX;
}

// SPEC = true: speculative one-pass of the learned form.  c_rowptr then holds
// staging offsets, c_colind / c_vals the staging arrays, cap[i] the row's
// predicted capacity; a row with more columns than its capacity overflows
// (cnt_out[i] = -1, re-run by the plain path), otherwise cnt_out[i] = nnz.
template <int W, bool SPEC, int VMAX = kWindowMaxNnz>
__global__ void __launch_bounds__(kWinWarps * 32, 4)
k_num_window(CsrView A, CsrView B, BComp bcomp, WinCacheView cache,
             const int32_t* __restrict__ row_lo, const float2* __restrict__ bspl,
             const int32_t* __restrict__ b_range_bad, int32_t arith,
             const int64_t* __restrict__ c_rowptr, const int32_t* __restrict__ rows, int32_t nrows,
             int32_t* __restrict__ c_colind, double* __restrict__ c_vals, int* status,
             const int32_t* __restrict__ cap, int32_t* __restrict__ cnt_out,
             const int32_t* __restrict__ nrows_dev) {
  using G = NumWinGeom<W, VMAX>;
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
  const bool df_all = arith == kArithDF32 && *b_range_bad == 0;
  const int32_t* __restrict__ acol = A.colind;
  const double* __restrict__ aval = A.vals;
  const int32_t* __restrict__ brp = B.rowptr;
  const int32_t* __restrict__ bcol = B.colind;
  const double* __restrict__ bval = B.vals;
  if (nrows_dev) nrows = *nrows_dev;
  const int nw = gridDim.x * kWinWarps;  // rows dealt round-robin over the grid
  if (blockIdx.x * kWinWarps + warp >= nrows) return;  // warps share no shared memory or barrier
  for (int w = lane * 4; w < WORDS; w += 128)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int w = lane; w < SUMS; w += 32) sum[w] = 0u;
  __syncwarp();
  for (int r = blockIdx.x * kWinWarps + warp; r < nrows; r += nw) {
    const int i = rows[r];
    const int lo_w = row_lo[i] >> 5;
    const int lo_c = lo_w * 32;
    const int64_t off = c_rowptr[i];
    const int cnt = SPEC ? min(cap[i], VMAX) : (int)(c_rowptr[i + 1] - off);
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    const int Lc = (!SPEC && cache.n) ? cache.n[i] : -1;
    // value slots of the row's columns (a rank past cnt goes to the spare slot
    // VMAX, which is never read)
    for (int e = lane; e < min(cnt, VMAX); e += 32) vacc[e] = 0ull;
    int L, run = 0, bad = 0;
    if (Lc >= 0 && Lc <= kCacheWords) {
      // structure kept by the symbolic phase: words, bits, prefixes, columns
      L = Lc;
      for (int e0 = 0; e0 < L; e0 += 32) {
        const int e = e0 + lane;
        int w = 0;
        uint32_t m = 0u;
        if (e < L) {
          w = cache.w[(size_t)i * kCacheWords + e];
          m = cache.m[(size_t)i * kCacheWords + e];
          if (w >= WORDS) {
            bad = 1;
            m = 0u;
            w = 0;
          }
        }
        const int c = __popc(m);
        const int incl = team_inclusive_scan<32>(c, lane, kFull);
        int pos = run + incl - c;
        run += __shfl_sync(kFull, incl, 31);
        if (e < L) {
          list[e] = (uint16_t)w;
          bits[w] = m;
          pre[w] = (uint16_t)pos;
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (pos < cnt) c_colind[off + pos] = lo_c + w * 32 + b;
            ++pos;
          }
        }
      }
    } else {
      // rebuild: bits from B_C, ordered word list, prefixes and columns
      bc_set_bits<WORDS, false, 4>(bits, sum, lo_w, pa, pe, acol, brp, bcomp.bc, bcomp.len, lane, status);
      L = window_list<SUMS>(sum, list, VMAX, lane);
      if (L > VMAX) {  // more words than a window row has columns
        for (int w = lane * 4; w < WORDS; w += 128)
          *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
        if (lane == 0) {
          if (SPEC) cnt_out[i] = -1;
          else set_status(status, KK_ERR_STRUCTURE_MISMATCH);
        }
        __syncwarp();
        continue;
      }
      for (int e0 = 0; e0 < L; e0 += 32) {
        const int e = e0 + lane;
        const int w = e < L ? (int)list[e] : 0;
        uint32_t m = e < L ? bits[w] : 0u;
        const int c = __popc(m);
        const int incl = team_inclusive_scan<32>(c, lane, kFull);
        int pos = run + incl - c;
        run += __shfl_sync(kFull, incl, 31);
        if (e < L) {
          pre[w] = (uint16_t)pos;
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (pos < cnt) c_colind[off + pos] = lo_c + w * 32 + b;
            ++pos;
          }
        }
      }
    }
    if (bad) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    if (!SPEC && run != cnt && lane == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    if (SPEC) {
      if (run > cnt) {  // overflow: abandon the row, clear what it set
        if (lane == 0) cnt_out[i] = -1;
        for (int e = lane; e < L; e += 32) bits[list[e]] = 0u;
        __syncwarp();
        continue;
      }
      if (lane == 0) cnt_out[i] = run;
    }
    __syncwarp();
    // arithmetic of this row: DF32 unless a value of the row is outside its
    // window (rows of up to 32 entries decide from the split below)
    const bool df_row = df_all && df_row_terms_ok(pa, pe);
    bool df = df_row;
    if (df_row && pe - pa > 32) df = row_df_ok<32>(aval, pa, pe, lane, kFull);
    int missing = 0;
    for (int p0 = pa; p0 < pe; p0 += 32) {
      const int p = p0 + lane;
      int4 info = make_int4(0, 0, 0, 0);
      double a = 0.0;
      if (p < pe) {
        const int j = acol[p];
        info.x = brp[j];
        info.y = brp[j + 1] - info.x;
        a = a_value(A, i, p);
      }
      DF ad;
      const int split_bad = df_row ? (df_split(a, ad) ? 0 : 1) : 1;
      if (df_row && pe - pa <= 32) df = __any_sync(kFull, split_bad) == 0;
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
      const int nch = min(32, pe - p0);
      const unsigned maxlen = __reduce_max_sync(kFull, (unsigned)info.y);
      if (maxlen <= 32u) {
        for (int t0 = 0; t0 < nch; t0 += kWinBatch) {
          float2 bv[kWinBatch];
          int rk[kWinBatch];
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) {
            int c = 0;
            bool ok = false;
            bv[u] = make_float2(0.f, 0.f);
            if (t0 + u < nch) {
              const int2 in = *reinterpret_cast<const int2*>(&ainfo[t0 + u]);
              if (lane < in.y) {
                const int q = in.x + lane;
                ok = true;
                c = bcol[q];
                if (df) {
                  bv[u] = bspl[q];
                } else {
                  const long long bb = __double_as_longlong(bval[q]);
                  bv[u] = make_float2(__int_as_float((int)(bb & 0xffffffffll)),
                                      __int_as_float((int)(bb >> 32)));
                }
              }
            }
            rk[u] = window_rank<WORDS, VMAX>(bits, pre, (uint32_t)(c - lo_c), ok, missing);
          }
#pragma unroll
          for (int u = 0; u < kWinBatch; ++u) {
            if (t0 + u < nch) {
              const int2 az = *reinterpret_cast<const int2*>(&ainfo[t0 + u].z);
              if (df) {
                DF av2, b2;
                av2.hi = __int_as_float(az.x);
                av2.lo = __int_as_float(az.y);
                b2.hi = bv[u].x;
                b2.lo = bv[u].y;
                DF s = df_unpack(vacc[rk[u]]);
                df_fma(s, av2, b2);
                vacc[rk[u]] = df_pack(s);
              } else {
                const double x = __longlong_as_double(((long long)az.y << 32) | (unsigned)az.x);
                const double y = __longlong_as_double(((long long)__float_as_int(bv[u].y) << 32) |
                                                      (unsigned)__float_as_int(bv[u].x));
                double* v = reinterpret_cast<double*>(&vacc[rk[u]]);
                *v = fma(x, y, *v);
              }
              __syncwarp();  // this A entry's updates are visible before the next one's
            }
          }
        }
      } else {
        for (int t = 0; t < nch; ++t) {
          const int4 in = ainfo[t];
          for (int q0 = 0; q0 < in.y; q0 += 32) {
            const int q = in.x + q0 + lane;
            const bool ok = q0 + lane < in.y;
            const int c = ok ? bcol[q] : 0;
            const int rank = window_rank<WORDS, VMAX>(bits, pre, (uint32_t)(c - lo_c), ok, missing);
            if (df) {
              DF av2, b2;
              av2.hi = __int_as_float(in.z);
              av2.lo = __int_as_float(in.w);
              const float2 bb = ok ? bspl[q] : make_float2(0.f, 0.f);
              b2.hi = bb.x;
              b2.lo = bb.y;
              DF s = df_unpack(vacc[rank]);
              df_fma(s, av2, b2);
              vacc[rank] = df_pack(s);
            } else {
              const double x = __longlong_as_double(((long long)in.w << 32) | (unsigned)in.z);
              double* v = reinterpret_cast<double*>(&vacc[rank]);
              *v = fma(x, ok ? bval[q] : 0.0, *v);
            }
            __syncwarp();
          }
        }
      }
      __syncwarp();
    }
    if (missing) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    const int n = min(SPEC ? run : cnt, VMAX);
    for (int e = lane; e < n; e += 32) {
      const u64 v = vacc[e];
      c_vals[off + e] = df ? df_to_double(df_unpack(v)) : __longlong_as_double((long long)v);
    }
    // clear the words this row set for the next row
    for (int e = lane; e < L; e += 32) bits[list[e]] = 0u;
    __syncwarp();
  }
}

// DF32 s += b (two-sum of the high parts, renormalised).
__device__ __forceinline__ void df_add(DF& s, const DF b) {
  const float sh = s.hi + b.hi;
  const float bb = sh - s.hi;
  const float err = (s.hi - (sh - bb)) + (b.hi - bb);
  const float lo = s.lo + (b.lo + err);
  const float hi = sh + lo;
  s.lo = lo - (hi - sh);
  s.hi = hi;
}

// Value pass over the A entries [p_lo, p_hi) of a window row into vacc: DF32
// pairs when df, else float64 in storage order; ranks from the window's bits
// and prefix counts.  One warp.
template <int WORDS, int VMAX>
__device__ __forceinline__ void window_values(int p_lo, int p_hi, bool df, const CsrView& A, int i,
                                              const int32_t* __restrict__ brp,
                                              const int32_t* __restrict__ bcol,
                                              const float2* __restrict__ bspl,
                                              const double* __restrict__ bval, const uint32_t* bits,
                                              const uint16_t* pre, int lo_c, u64* vacc, int4* ainfo,
                                              int lane, int& missing) {
  for (int p0 = p_lo; p0 < p_hi; p0 += 32) {
    const int p = p0 + lane;
    int4 info = make_int4(0, 0, 0, 0);
    double a = 0.0;
    if (p < p_hi) {
      const int j = A.colind[p];
      info.x = brp[j];
      info.y = brp[j + 1] - info.x;
      a = a_value(A, i, p);
    }
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
    ainfo[lane] = info;
    __syncwarp();
    const int nch = min(32, p_hi - p0);
    const unsigned maxlen = __reduce_max_sync(kFull, (unsigned)info.y);
    if (maxlen <= 32u) {
      // B rows of at most 32 entries: the loads of kWinBatch A entries in flight
      for (int t0 = 0; t0 < nch; t0 += kWinBatch) {
        float2 bv[kWinBatch];
        int rk[kWinBatch];
#pragma unroll
        for (int u = 0; u < kWinBatch; ++u) {
          int c = 0;
          bool ok = false;
          bv[u] = make_float2(0.f, 0.f);
          if (t0 + u < nch) {
            const int2 in = *reinterpret_cast<const int2*>(&ainfo[t0 + u]);
            if (lane < in.y) {
              const int q = in.x + lane;
              ok = true;
              c = bcol[q];
              if (df) {
                bv[u] = bspl[q];
              } else {
                const long long bb = __double_as_longlong(bval[q]);
                bv[u] = make_float2(__int_as_float((int)(bb & 0xffffffffll)),
                                    __int_as_float((int)(bb >> 32)));
              }
            }
          }
          rk[u] = window_rank<WORDS, VMAX>(bits, pre, (uint32_t)(c - lo_c), ok, missing);
        }
#pragma unroll
        for (int u = 0; u < kWinBatch; ++u) {
          if (t0 + u < nch) {
            const int2 az = *reinterpret_cast<const int2*>(&ainfo[t0 + u].z);
            if (df) {
              DF av2, b2;
              av2.hi = __int_as_float(az.x);
              av2.lo = __int_as_float(az.y);
              b2.hi = bv[u].x;
              b2.lo = bv[u].y;
              DF sv = df_unpack(vacc[rk[u]]);
              df_fma(sv, av2, b2);
              vacc[rk[u]] = df_pack(sv);
            } else {
              const double x = __longlong_as_double(((long long)az.y << 32) | (unsigned)az.x);
              const double y = __longlong_as_double(((long long)__float_as_int(bv[u].y) << 32) |
                                                    (unsigned)__float_as_int(bv[u].x));
              double* v = reinterpret_cast<double*>(&vacc[rk[u]]);
              *v = fma(x, y, *v);
            }
            __syncwarp();  // this A entry's updates are visible before the next one's
          }
        }
      }
      __syncwarp();
      continue;
    }
    for (int t = 0; t < nch; ++t) {
      const int4 in = ainfo[t];
      for (int q0 = 0; q0 < in.y; q0 += 32) {
        const int q = in.x + q0 + lane;
        const bool ok = q0 + lane < in.y;
        const int c = ok ? bcol[q] : 0;
        const int rank = window_rank<WORDS, VMAX>(bits, pre, (uint32_t)(c - lo_c), ok, missing);
        if (df) {
          DF av2, b2;
          av2.hi = __int_as_float(in.z);
          av2.lo = __int_as_float(in.w);
          const float2 bb = ok ? bspl[q] : make_float2(0.f, 0.f);
          b2.hi = bb.x;
          b2.lo = bb.y;
          DF sv = df_unpack(vacc[rank]);
          df_fma(sv, av2, b2);
          vacc[rank] = df_pack(sv);
        } else {
          const double x = __longlong_as_double(((long long)in.w << 32) | (unsigned)in.z);
          double* v = reinterpret_cast<double*>(&vacc[rank]);
          *v = fma(x, ok ? bval[q] : 0.0, *v);
        }
        __syncwarp();  // this B entry set's updates are visible before the next one's
      }
    }
    __syncwarp();
  }
}

// Large-value window rows (more than kWindowMaxNnz columns), one CTA of
// kWinCtaWarps warps per row.  The window (bits, summary bits, prefix counts,
// word list) is shared by the CTA instead of one per warp, so an SM holds
// about twice as many warps of these rows; the warps split the row's A entries
// into contiguous shares, OR their compressed rows into the shared window,
// and add their products into a value array of their own; the arrays are
// summed in warp order, so the result does not depend on scheduling.  A row
// whose values leave the DF32 window is added by warp 0 alone, in float64 and
// storage order.  The structure is always rebuilt from B_C.
constexpr int kWinCtaWarps = 4;
template <int W, int VMAX>
struct CtaWinGeom : WinWords<W> {
  using WinWords<W>::WORDS;
  using WinWords<W>::SUMS;
  // bits u32[WORDS] | sum u32[SUMS] | prefix u16[WORDS] | list u16[VMAX]
  // | vacc u64[kWinCtaWarps][VMAX + 2] | ainfo int4[kWinCtaWarps][32] | int[8]
  static constexpr size_t kSumOff = al16((size_t)WORDS * 4);
  static constexpr size_t kPreOff = al16(kSumOff + (size_t)SUMS * 4);
  static constexpr size_t kListOff = al16(kPreOff + (size_t)WORDS * 2);
  static constexpr size_t kValOff = al16(kListOff + (size_t)VMAX * 2);
  static constexpr size_t kValStride = (size_t)(VMAX + 2);
  static constexpr size_t kInfoOff = al16(kValOff + kWinCtaWarps * kValStride * 8);
  static constexpr size_t kShOff = kInfoOff + (size_t)kWinCtaWarps * 32 * 16;
  static constexpr size_t kBytes = kShOff + 8 * 4;
};

template <int W, int VMAX>
__global__ void __launch_bounds__(kWinCtaWarps * 32)
k_num_window_cta(CsrView A, CsrView B, BComp bcomp, const int32_t* __restrict__ row_lo,
                 const float2* __restrict__ bspl, const int32_t* __restrict__ b_range_bad,
                 int32_t arith, const int64_t* __restrict__ c_rowptr, const int32_t* __restrict__ rows,
                 int32_t nrows, int32_t* __restrict__ c_colind, double* __restrict__ c_vals, int* status) {
  using G = CtaWinGeom<W, VMAX>;
  constexpr int WORDS = G::WORDS;
  constexpr int SUMS = G::SUMS;
  constexpr int NT = kWinCtaWarps * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* sum = reinterpret_cast<uint32_t*>(smem_raw + G::kSumOff);
  uint16_t* pre = reinterpret_cast<uint16_t*>(smem_raw + G::kPreOff);
  uint16_t* list = reinterpret_cast<uint16_t*>(smem_raw + G::kListOff);
  u64* vacc_all = reinterpret_cast<u64*>(smem_raw + G::kValOff);
  u64* vacc = vacc_all + warp * G::kValStride;
  int4* ainfo = reinterpret_cast<int4*>(smem_raw + G::kInfoOff) + warp * 32;
  int* sh = reinterpret_cast<int*>(smem_raw + G::kShOff);
  const bool df_all = arith == kArithDF32 && *b_range_bad == 0;
  const int32_t* __restrict__ acol = A.colind;
  const double* __restrict__ aval = A.vals;
  for (int w = tid * 4; w < WORDS; w += NT * 4)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int w = tid; w < SUMS; w += NT) sum[w] = 0u;
  __syncthreads();
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int lo_w = row_lo[i] >> 5;
    const int lo_c = lo_w * 32;
    const int64_t off = c_rowptr[i];
    const int cnt = (int)(c_rowptr[i + 1] - off);
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    for (int e = lane; e < min(cnt, VMAX); e += 32) vacc[e] = 0ull;
    // this warp's share of the A entries
    const int na = pe - pa;
    const int qa = (na + kWinCtaWarps - 1) / kWinCtaWarps;
    const int p_lo = pa + min(na, warp * qa), p_hi = pa + min(na, (warp + 1) * qa);
    bc_set_bits<WORDS, false, 4>(bits, sum, lo_w, p_lo, p_hi, acol, B.rowptr, bcomp.bc, bcomp.len, lane, status);
    __syncthreads();
    if (warp == 0) {
      const int L0 = window_list<SUMS>(sum, list, VMAX, lane);
      if (lane == 0) sh[0] = L0;
    }
    __syncthreads();
    const int L = sh[0];
    if (L > VMAX) {  // more words than a window row has columns
      for (int w = tid * 4; w < WORDS; w += NT * 4)
        *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
      if (tid == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
      __syncthreads();
      continue;
    }
    // prefix counts and columns: warp w takes a contiguous part of the list
    const int lq = (L + NT - 1) / NT * 32;
    const int e_lo = min(L, warp * lq), e_hi = min(L, (warp + 1) * lq);
    int part = 0;
    for (int e = e_lo + lane; e < e_hi; e += 32) part += __popc(bits[list[e]]);
    part = team_sum<32>(part, kFull);
    if (lane == 0) sh[1 + warp] = part;
    __syncthreads();
    int run = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kWinCtaWarps; ++k) {
      run += k < warp ? sh[1 + k] : 0;
      total += sh[1 + k];
    }
    for (int e0 = e_lo; e0 < e_hi; e0 += 32) {
      const int e = e0 + lane;
      const int w = e < e_hi ? (int)list[e] : 0;
      uint32_t m = e < e_hi ? bits[w] : 0u;
      const int c = __popc(m);
      const int incl = team_inclusive_scan<32>(c, lane, kFull);
      int pos = run + incl - c;
      run += __shfl_sync(kFull, incl, 31);
      if (e < e_hi) {
        pre[w] = (uint16_t)pos;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          if (pos < cnt) c_colind[off + pos] = lo_c + w * 32 + b;
          ++pos;
        }
      }
    }
    if (tid == 0 && total != cnt) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    __syncthreads();
    // arithmetic of this row: DF32 unless one of its A values is outside the window
    const bool df = df_all && df_row_terms_ok(pa, pe) && row_df_ok<32>(aval, pa, pe, lane, kFull);
    int missing = 0;
    if (df)
      window_values<WORDS, VMAX>(p_lo, p_hi, true, A, i, B.rowptr, B.colind, bspl, B.vals, bits, pre,
                                 lo_c, vacc, ainfo, lane, missing);
    else if (warp == 0)
      window_values<WORDS, VMAX>(pa, pe, false, A, i, B.rowptr, B.colind, bspl, B.vals, bits, pre,
                                 lo_c, vacc, ainfo, lane, missing);
    if (missing) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    __syncthreads();
    const int n = min(cnt, VMAX);
    for (int e = tid; e < n; e += NT) {
      if (df) {
        DF v = df_unpack(vacc_all[e]);
#pragma unroll
        for (int k = 1; k < kWinCtaWarps; ++k) df_add(v, df_unpack(vacc_all[k * G::kValStride + e]));
        c_vals[off + e] = df_to_double(v);
      } else {
        c_vals[off + e] = __longlong_as_double((long long)vacc_all[e]);
      }
    }
    for (int e = tid; e < L; e += NT) bits[list[e]] = 0u;
    __syncthreads();
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

// One resident wave of a row-striding kernel: the SMs' count times the CTAs
// of `kern` an SM holds at once (never more than the rows need).  With every
// CTA resident, the rows in flight are one contiguous band that advances
// through the matrix, so the B rows they share stay in L2; a grid of several
// waves would run bands far apart in the matrix at once.
template <class K>
int resident_grid(const LaunchCtx& ctx, K kern, int threads, size_t smem, int nrows, int rows_per_cta) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  long long blocks = (nrows + rows_per_cta - 1) / rows_per_cta;
  const long long cap = (long long)ctx.num_sms * per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <int W>
cudaError_t sym_window(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, const BComp& bcomp,
                       const int32_t* rows, int32_t nrows, int32_t* cnt, const WinCache& cache) {
  const size_t smem = (size_t)kWinWarps * SymWinGeom<W>::kWarpBytes;
  auto kern = k_sym_window<W>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<resident_grid(ctx, kern, kWinWarps * 32, smem, nrows, kWinWarps), kWinWarps * 32, smem, ctx.stream>>>(
      A, B, bcomp, ctx.row_lo, rows, nrows, cnt, cache, ctx.status);
  return cudaGetLastError();
}

template <int W, bool SPEC = false, int VMAX = kWindowMaxNnz>
cudaError_t num_window(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, const BComp& bcomp,
                       const WinCacheView& cache, const float2* b_split,
                       const int32_t* b_range_bad, int32_t arith, const int64_t* c_rowptr,
                       const int32_t* rows, int32_t nrows, int32_t* c_colind, double* c_vals,
                       const int32_t* cap = nullptr, int32_t* cnt_out = nullptr,
                       const int32_t* nrows_dev = nullptr) {
  const size_t smem = (size_t)kWinWarps * NumWinGeom<W, VMAX>::kWarpBytes;
  auto kern = k_num_window<W, SPEC, VMAX>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int grid = grid_for_rows(ctx, nrows);
  // a device-side row count (the leftover pass) is usually small or zero:
  // one wave of the kernel's minimum residency strides over it
  if (nrows_dev && grid > ctx.num_sms * 4) grid = ctx.num_sms * 4;
  kern<<<grid, kWinWarps * 32, smem, ctx.stream>>>(
      A, B, bcomp, cache, ctx.row_lo, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind,
      c_vals, ctx.status, cap, cnt_out, nrows_dev);
  return cudaGetLastError();
}

template <int W, int VMAX>
cudaError_t num_window_cta(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, const BComp& bcomp,
                           const float2* b_split, const int32_t* b_range_bad, int32_t arith,
                           const int64_t* c_rowptr, const int32_t* rows, int32_t nrows, int32_t* c_colind,
                           double* c_vals) {
  const size_t smem = CtaWinGeom<W, VMAX>::kBytes;
  auto kern = k_num_window_cta<W, VMAX>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  // persistent: one resident wave strides over the rows
  static int per_sm = 0;
  if (per_sm == 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWinCtaWarps * 32, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  long long grid = (long long)ctx.num_sms * (per_sm > 0 ? per_sm : 1);
  if (grid > nrows) grid = nrows;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, kWinCtaWarps * 32, smem, ctx.stream>>>(A, B, bcomp, ctx.row_lo, b_split, b_range_bad,
                                                           arith, c_rowptr, rows, nrows, c_colind, c_vals,
                                                           ctx.status);
  return cudaGetLastError();
}

}  // namespace


cudaError_t launch_symbolic_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                   const CsrView& B, const BComp& bcomp, const int32_t* rows,
                                   int32_t nrows, int32_t* cnt, const WinCache& cache) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "sym_window");
  cudaError_t e = cudaErrorInvalidValue;
  switch (bin.slots) {
    case 4096: e = sym_window<4096>(ctx, A, B, bcomp, rows, nrows, cnt, cache); break;
    case 12288: e = sym_window<12288>(ctx, A, B, bcomp, rows, nrows, cnt, cache); break;
    case 24576: e = sym_window<24576>(ctx, A, B, bcomp, rows, nrows, cnt, cache); break;
    case 40960: e = sym_window<40960>(ctx, A, B, bcomp, rows, nrows, cnt, cache); break;
    case 65536: e = sym_window<65536>(ctx, A, B, bcomp, rows, nrows, cnt, cache); break;
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

cudaError_t launch_numeric_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                  const CsrView& B, const BComp& bcomp, const WinCacheView& cache,
                                  const WinScratch& scratch, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith,
                                  const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                  int32_t* c_colind, double* c_vals) {
  if (nrows <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (bin.hi > kWindowMaxNnz) {  // rows of up to kWindowMaxNnzWide columns: large value array
    timer_begin(ctx.timer, ctx.stream, "num_window");
    e = cudaErrorInvalidValue;
#define KK_NUM_WIN_LARGE(WB, VM)                                                                 \
  case WB:                                                                                       \
    e = num_window_cta<WB, VM>(ctx, A, B, bcomp, b_split, b_range_bad, arith, c_rowptr, rows, nrows, \
                               c_colind, c_vals);                                                \
    break;
    if (bin.hi <= kWindowMidNnz) {
      switch (bin.slots) {
        KK_NUM_WIN_LARGE(24576, kWindowMidNnz)
        KK_NUM_WIN_LARGE(40960, kWindowMidNnz)
        KK_NUM_WIN_LARGE(65536, kWindowMidNnz)
      }
    } else {
      switch (bin.slots) {
        KK_NUM_WIN_LARGE(24576, kWindowMaxNnzWide)
        KK_NUM_WIN_LARGE(40960, kWindowMaxNnzWide)
        KK_NUM_WIN_LARGE(65536, kWindowMaxNnzWide)
      }
    }
#undef KK_NUM_WIN_LARGE
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  // rows of at most kWindowMaxNnz columns: with the automatic arithmetic in
  // float64, whether the kept structure or the rebuild serves them (so that a
  // row's values do not depend on which one did)
  if (ctx.kept_f64) arith = kArithF64;
  const int32_t* wrows = rows;
  const int32_t* wcount = nullptr;
  if (cache.n && scratch.rows) {
    timer_begin(ctx.timer, ctx.stream, "num_kept");
    e = cudaMemsetAsync(scratch.count, 0, sizeof(int32_t), ctx.stream);
    if (e == cudaSuccess)
      e = launch_num_kept(ctx, A, B, cache, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind,
                   c_vals, scratch.rows, scratch.count);
    timer_end(ctx.timer, ctx.stream);
    if (e != cudaSuccess) return e;
    wrows = scratch.rows;
    wcount = scratch.count;
  }
  timer_begin(ctx.timer, ctx.stream, "num_window");
  e = cudaErrorInvalidValue;
#define KK_NUM_WIN(WB)                                                                          \
  case WB:                                                                                      \
    e = num_window<WB>(ctx, A, B, bcomp, cache, b_split, b_range_bad, arith, c_rowptr, wrows,   \
                       nrows, c_colind, c_vals, nullptr, nullptr, wcount);                      \
    break;
  switch (bin.slots) {
    KK_NUM_WIN(4096)
    KK_NUM_WIN(12288)
    KK_NUM_WIN(24576)
    KK_NUM_WIN(40960)
    KK_NUM_WIN(65536)
  }
#undef KK_NUM_WIN
  timer_end(ctx.timer, ctx.stream);
  return e;
}

cudaError_t launch_onepass_window(const LaunchCtx& ctx, int32_t wclass, const CsrView& A,
                                  const CsrView& B, const BComp& bcomp, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith, const int64_t* soff,
                                  const int32_t* cap, const int32_t* rows, int32_t nrows,
                                  int32_t* scol, double* sval, int32_t* cnt_out) {
  if (nrows <= 0) return cudaSuccess;
  timer_begin(ctx.timer, ctx.stream, "onepass_window");
  cudaError_t e = cudaErrorInvalidValue;
  const WinCacheView none{nullptr, nullptr, nullptr};
#define KK_ONE_WIN(WB)                                                                          \
  case WB:                                                                                      \
    e = num_window<WB, true>(ctx, A, B, bcomp, none, b_split, b_range_bad, arith, soff, rows,   \
                             nrows, scol, sval, cap, cnt_out);                                  \
    break;
  switch (kWindowBits[wclass]) {
    KK_ONE_WIN(4096)
    KK_ONE_WIN(12288)
    KK_ONE_WIN(24576)
    KK_ONE_WIN(40960)
    KK_ONE_WIN(65536)
  }
#undef KK_ONE_WIN
  timer_end(ctx.timer, ctx.stream);
  return e;
}

}  // namespace kk
