// Wide tier: rows too heavy for a team hash (the CTA and dense bins), when the
// bit vector of all k columns of C fits in shared memory.
//
// The paper's dense accumulator (Sec. "Standard SpGEMM Kernel") over the full
// column range: one CTA per row keeps a k-bit vector in shared memory, plus
// one summary bit per 32-bit word for rows whose products touch few words.
//   symbolic: every product ORs its column bit (no probing, no chunk passes);
//             nnz(C(i,:)) = popcount of the touched words, cleared as they are
//             counted;
//   numeric:  the same bits; prefix counts over the touched words give every
//             column its rank, the column indices are written from the bits
//             in order, and each product adds a*b into value slot `rank`: in
//             shared memory when the row's nnz fits, else directly into C's
//             values (zeroed first) with global float64 atomics.  The order of
//             the additions is not fixed, so the values carry the float64 bound
//             of an unordered sum.
// Rows whose values go to C with atomics keep their bit vector from the
// symbolic phase (a slot of ceil(k/32) words in global memory, while the
// handle's budget lasts), so the numeric phase loads it instead of walking the
// row's products a second time for the structure.
// The CTA walks the row's products (the flattened (A entry, B entry) pairs in
// storage order) in work items of kItem products that warps claim from a
// shared counter, so one long B row does not leave the other warps waiting at
// the row's barrier; each lane issues kWideU loads before it uses them.
#include "kk_internal.h"
#include "kk_device.cuh"

namespace kk {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWideU = 4;      // warp steps whose loads are issued together
constexpr int kWideBlock = 1024;
constexpr int kKeepU = 4;      // 16-byte loads in flight per thread when a kept bit vector is loaded

// Words of the column bit vector: ceil(k / 32) rounded up to a multiple of
// 1024 (one run of 32 words per lane of every warp of the CTA).
__host__ __device__ inline int wide_words(int k) { return (((k + 31) >> 5) + 1023) & ~1023; }

// Shared memory: bits u32[words] | sum u32[words / 32] | region u8[2 * words]
// | values f64[vcap].  The region holds either per-word prefixes (u16, rows
// with values in shared memory) or per-group (8 words) u32 prefixes and
// per-word u8 offsets (rows with values in C); the ordered list of touched
// words (u16) is built in the value area before the values are zeroed.
struct WideGeom {
  size_t sum_off, reg_off, val_off, bytes;
  int vcap;
};
inline WideGeom wide_geom(int words, size_t max_smem, bool numeric) {
  WideGeom g;
  g.sum_off = (size_t)words * 4;
  g.reg_off = g.sum_off + (size_t)words / 32 * 4;
  g.reg_off = (g.reg_off + 15) / 16 * 16;
  g.val_off = numeric ? g.reg_off + (size_t)words * 2 : g.reg_off;
  const long long left = (long long)max_smem - (long long)g.val_off;
  g.vcap = (numeric && left > 0) ? (int)(left / 8) : 0;
  if (g.vcap > 32768) g.vcap = 32768;
  g.bytes = g.val_off + (size_t)g.vcap * 8;
  return g;
}

// Exclusive block scan of v (blockDim.x <= 1024); *total receives the sum.
template <class T>
__device__ __forceinline__ T block_exscan(T v, T* tmp, T* total) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += n;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const T x = lane < nwarps ? tmp[lane] : T(0);
    T xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T n = __shfl_up_sync(kFull, xi, o);
      if (lane >= o) xi += n;
    }
    tmp[lane] = xi - x;
    if (lane == 31) tmp[32] = xi;
  }
  __syncthreads();
  const T r = tmp[warp] + incl - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

// Shared scratch of the product walk: the segment's product prefix and B row
// starts, the work-item counter and the scan buffer.
constexpr int kSeg = kWideBlock;       // A entries per segment (one per thread)
constexpr int kItem = 32 * kWideU * 2;  // products per work item
struct WalkSmem {
  long long pre[kSeg + 1];
  int bst[kSeg];
  long long tmp[33];
  int next;
};

// Visit every product A(i,j)*B(j,c) of the A entries [pa, pe) of a row with
// the whole CTA, balanced to kItem products: the row's A entries are taken
// kSeg at a time; their products, flattened in storage order, are cut into
// items of kItem that warps claim from a shared counter; a warp walks its item
// with lanes over consecutive products, 32 A entries' bounds held in lanes,
// and issues kWideU steps of loads before using them.  use(c, ab, ok) gets
// the column (and with VALS the product a*b in float64).  Ends with a barrier.
template <bool VALS, class Use>
__device__ __forceinline__ void wide_walk(const CsrView& A, const CsrView& B, int pa, int pe,
                                          WalkSmem& ws, int& bad, Use use, int row = 0) {
  const int lane = threadIdx.x & 31;
  const int32_t* __restrict__ bcol = B.colind;
  const double* __restrict__ bval = B.vals;
  for (int s0 = pa; s0 < pe; s0 += kSeg) {
    const int ns = min(kSeg, pe - s0);
    {
      const int t = threadIdx.x;
      int bs = 0;
      long long len = 0;
      if (t < ns) {
        const int j = A.colind[s0 + t];
        if ((unsigned)j < (unsigned)B.m) {
          bs = B.rowptr[j];
          len = B.rowptr[j + 1] - bs;
        } else {
          bad = 1;
        }
      }
      long long total;
      const long long ex = block_exscan<long long>(len, ws.tmp, &total);
      ws.pre[t] = ex;
      ws.bst[t] = bs;
      if (t == 0) {
        ws.pre[ns] = total;
        ws.next = 0;
      }
      __syncthreads();
    }
    const long long total = ws.pre[ns];
    for (;;) {
      int it = 0;
      if (lane == 0) it = atomicAdd(&ws.next, 1);
      it = __shfl_sync(kFull, it, 0);
      const long long fb = (long long)it * kItem;
      if (fb >= total) break;
      const int ilen = (int)min((long long)kItem, total - fb);
      // entry holding product fb: last t with pre[t] <= fb (32-ary search)
      int lo = 0, hi = ns;
      while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int cand = lo + lane * step;
        const bool le = cand < hi && ws.pre[cand] <= fb;
        const unsigned m = __ballot_sync(kFull, le);
        const int last = 31 - __clz(m);
        lo = lo + last * step;
        hi = min(hi, lo + step);
      }
      int done = 0, t0 = lo;
      while (done < ilen) {
        // window of A entries t0 .. t0 + 31: starts relative to fb
        const int tl = t0 + lane;
        const long long P = tl < ns ? ws.pre[tl] : total;
        int rel = (int)max(min(P - fb, (long long)0x7fffffff), -(long long)0x7fffffff);
        if (tl >= ns) rel = 0x7fffffff;
        const int bsl = tl < ns ? ws.bst[tl] : 0;
        double al = 0.0;
        if (VALS && tl < ns) al = a_value(A, row, s0 + tl);
        const long long wend = t0 + 32 < ns ? ws.pre[t0 + 32] : total;
        const int lim = (int)min((long long)ilen, wend - fb);
        for (int g = done; g < lim; g += 32 * kWideU) {
          int col[kWideU];
          double ab[kWideU];
#pragma unroll
          for (int u = 0; u < kWideU; ++u) {
            const int f = g + u * 32 + lane;
            int own = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
              const int v = __shfl_sync(kFull, rel, own + st);
              if (own + st < 32 && v <= f) own += st;
            }
            const int q = __shfl_sync(kFull, bsl, own) + (f - __shfl_sync(kFull, rel, own));
            const double a = VALS ? __shfl_sync(kFull, al, own) : 0.0;
            col[u] = -1;
            ab[u] = 0.0;
            if (f < lim) {
              col[u] = bcol[q];
              if (VALS) ab[u] = a * bval[q];
            }
          }
#pragma unroll
          for (int u = 0; u < kWideU; ++u) use(col[u], ab[u]);
        }
        done = lim;
        t0 += 32;
      }
    }
    __syncthreads();
  }
}

// Bulk-copy staging of long B-row pieces (symbolic wide kernel).  Each warp
// owns two shared-memory buffers of kStageCols columns (+ alignment slack) and
// an mbarrier per buffer.  A piece of at least 2 * kStageCols products is cut
// into sub-pieces; lane 0 copies sub-piece k + 2 with cp.async.bulk while the
// warp ORs sub-piece k from the other buffer, so the row's columns arrive by
// the copy unit in large transfers instead of per-lane loads.  The copied
// range is widened to 16-byte boundaries (the copy unit's rule) and clipped to
// the last 16-byte boundary inside B's columns; anything past it is read with
// plain loads.
constexpr int kStageCols = 256;
constexpr int kStageSlots = kStageCols + 8;  // int32 per buffer: widening slack
struct StageState {
  int32_t* buf;               // this warp's two buffers (2 * kStageSlots)
  unsigned long long* bar;    // this warp's two mbarriers
  uint32_t phase;             // bit b: parity the next wait on buffer b expects
  bool ok;                    // false after a wait ran out: plain loads only
};

// Issue the copy of sub-piece k of the piece [q0, q0 + n) of B's columns into
// buffer k & 1 (lane 0).
__device__ __forceinline__ void stage_issue(const CsrView& B, StageState& st, int q0, int n, int k) {
  const int q = q0 + k * kStageCols;
  const int e = q + min(kStageCols, n - k * kStageCols);
  const int a0 = q & ~3;
  const int ce = min((e + 3) & ~3, B.nnz & ~3);
  unsigned long long* bar = st.bar + (k & 1);
  if (ce > a0) {
    const uint32_t bytes = (uint32_t)(ce - a0) * 4u;
    proxy_async_fence();  // the warp's reads of this buffer come before the copy's writes
    mbar_arrive_expect(bar, bytes);
    bulk_copy_g2s(st.buf + (k & 1) * kStageSlots, B.colind + a0, bytes, bar);
  } else {
    mbar_arrive(bar);
  }
}

// The columns of the piece [q0, q0 + n) (n >= 2 * kStageCols) through the
// staging buffers; use(col) per column.  Falls back to plain loads (and
// disables staging) if a wait runs out.
template <class Use>
__device__ __forceinline__ void stage_walk(const CsrView& B, StageState& st, int q0, int n, int* status,
                                           Use use) {
  const int lane = threadIdx.x & 31;
  const int nsub = (n + kStageCols - 1) / kStageCols;
  if (lane == 0) {
    stage_issue(B, st, q0, n, 0);
    stage_issue(B, st, q0, n, 1);
  }
  int k = 0;
  for (; k < nsub; ++k) {
    const int b = k & 1;
    const bool got = mbar_wait(st.bar + b, (st.phase >> b) & 1u, status);
    if (!__all_sync(kFull, got)) {
      // give the copies in flight a second bounded wait, then go on without them
      if (lane == 0) {
        mbar_wait(st.bar + b, (st.phase >> b) & 1u, status);
        if (k + 1 < nsub) mbar_wait(st.bar + (b ^ 1), (st.phase >> (b ^ 1)) & 1u, status);
      }
      __syncwarp();
      st.ok = false;
      break;
    }
    st.phase ^= 1u << b;
    const int q = q0 + k * kStageCols;
    const int e = q + min(kStageCols, n - k * kStageCols);
    const int a0 = q & ~3;
    const int ce = min((e + 3) & ~3, B.nnz & ~3);
    const int32_t* bufb = st.buf + b * kStageSlots;
    for (int x = q + lane; x < e; x += 32) use(x < ce ? bufb[x - a0] : B.colind[x]);
    __syncwarp();  // every lane is done with buffer b before it is refilled
    if (lane == 0 && k + 2 < nsub) stage_issue(B, st, q0, n, k + 2);
  }
  for (int x = q0 + k * kStageCols + lane; x < q0 + n; x += 32) use(B.colind[x]);  // after a give-up
  __syncwarp();
}

// Walk for rows whose B rows are long (mean length >= kLongMean): work items
// are the row's A entries cut into pieces of at most psz products (sized per
// row by wide_piece so that every warp gets several; with one or two items per
// warp the row's closing barrier waited for the largest piece); a warp
// claims an item from a shared counter, finds its entry by a 32-ary search over
// the item prefix (once per item, not per product) and its lanes stride the
// piece's B entries, kWideU loads in flight.  Same contract as wide_walk.
constexpr int kPieceMin = 256, kPieceMax = 2048;
constexpr long long kLongMean = 64;
struct LongSmem {
  int ipre[kSeg + 1];
  int bst[kSeg];
  int blen[kSeg];
  int tmp[33];
  int next;
};

template <bool VALS, class Use>
__device__ __forceinline__ void wide_walk_long(const CsrView& A, const CsrView& B, int pa, int pe,
                                               LongSmem& ls, int psz, int& bad, Use use, StageState* st = nullptr,
                                               int* status = nullptr, int row = 0) {
  const int lane = threadIdx.x & 31;
  const int32_t* __restrict__ bcol = B.colind;
  const double* __restrict__ bval = B.vals;
  for (int s0 = pa; s0 < pe; s0 += kSeg) {
    const int ns = min(kSeg, pe - s0);
    {
      const int t = threadIdx.x;
      int bs = 0, len = 0;
      if (t < ns) {
        const int j = A.colind[s0 + t];
        if ((unsigned)j < (unsigned)B.m) {
          bs = B.rowptr[j];
          len = B.rowptr[j + 1] - bs;
        } else {
          bad = 1;
        }
      }
      int total;
      const int ex = block_exscan<int>((len + psz - 1) / psz, ls.tmp, &total);
      ls.ipre[t] = ex;
      ls.bst[t] = bs;
      ls.blen[t] = len;
      if (t == 0) {
        ls.ipre[ns] = total;
        ls.next = 0;
      }
      __syncthreads();
    }
    const int nitems = ls.ipre[ns];
    for (;;) {
      int it = 0;
      if (lane == 0) it = atomicAdd(&ls.next, 1);
      it = __shfl_sync(kFull, it, 0);
      if (it >= nitems) break;
      // entry of item it: last t with ipre[t] <= it (32-ary search)
      int lo = 0, hi = ns;
      while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int cand = lo + lane * step;
        const bool le = cand < hi && ls.ipre[cand] <= it;
        const unsigned m = __ballot_sync(kFull, le);
        const int last = 31 - __clz(m);
        lo = lo + last * step;
        hi = min(hi, lo + step);
      }
      const int t = lo;
      const int piece = it - ls.ipre[t];
      const int q0 = ls.bst[t] + piece * psz;
      const int n = min(psz, ls.blen[t] - piece * psz);
      if (!VALS && st != nullptr && st->ok && n >= 2 * kStageCols) {
        stage_walk(B, *st, q0, n, status, [&](int c) { use(c, 0.0); });
        continue;
      }
      const double a = VALS ? a_value(A, row, s0 + t) : 0.0;
      for (int g = 0; g < n; g += 32 * kWideU) {
        int col[kWideU];
        double ab[kWideU];
#pragma unroll
        for (int u = 0; u < kWideU; ++u) {
          const int f = g + u * 32 + lane;
          col[u] = -1;
          ab[u] = 0.0;
          if (f < n) {
            col[u] = bcol[q0 + f];
            if (VALS) ab[u] = a * bval[q0 + f];
          }
        }
#pragma unroll
        for (int u = 0; u < kWideU; ++u) use(col[u], ab[u]);
      }
    }
    __syncthreads();
  }
}

// The two walks' shared state (never used at the same time).
union WideWalkSmem {
  WalkSmem ws;
  LongSmem ls;
};

// Walk of row i: 0 for the flattened walk, else the piece size of the
// entry-piece walk.  The mean B-row length of the row's A entries decides the
// walk; the pieces spread the row's products over about eight items per warp
// of the CTA, kPieceMin .. kPieceMax products each.
__device__ __forceinline__ int wide_piece(const long long* flop, int i, int pa, int pe) {
  if (flop == nullptr || pe <= pa || flop[i] < kLongMean * (long long)(pe - pa)) return 0;
  const long long per = flop[i] / (kWideBlock / 32 * 8);
  return per <= kPieceMin ? kPieceMin : per >= kPieceMax ? kPieceMax : (int)per;
}

// OR the column bits of the products of A entries [pa, pe) into bits (and,
// with SUM, the summary bits of their words).  Ends with a barrier.
template <bool SUM>
__device__ __forceinline__ void wide_set_bits(const CsrView& A, const CsrView& B, int pa, int pe,
                                              int psz, WideWalkSmem& wsm, uint32_t* bits,
                                              uint32_t* sum, int words, int& bad, StageState* st = nullptr,
                                              int* status = nullptr) {
  auto set = [&](int c, double) {
    if (c >= 0) {
      if ((unsigned)c < (unsigned)(words * 32)) {
        atomicOr(&bits[c >> 5], 1u << (c & 31));
        if (SUM) atomicOr(&sum[c >> 10], 1u << ((c >> 5) & 31));
      } else {
        bad = 1;
      }
    }
  };
  if (psz > 0) wide_walk_long<false>(A, B, pa, pe, wsm.ls, psz, bad, set, st, status);
  else wide_walk<false>(A, B, pa, pe, wsm.ws, bad, set);
}

__global__ void __launch_bounds__(kWideBlock, 1)
k_sym_wide(CsrView A, CsrView B, int32_t words, uint32_t sum_off, uint32_t stage_off,
           const long long* __restrict__ flop, const int32_t* __restrict__ rows, int32_t nrows,
           int32_t* __restrict__ cnt, WideKeep keep, int* status) {
  extern __shared__ __align__(16) unsigned char wsm[];
  uint32_t* bits = reinterpret_cast<uint32_t*>(wsm);
  uint32_t* sum = reinterpret_cast<uint32_t*>(wsm + sum_off);
  __shared__ WideWalkSmem walk;
  __shared__ int tmp[33];
  __shared__ int s_slot;
  __shared__ unsigned long long sbar[kWideBlock / 32 * 2];
  const int nsum = words >> 5;
  // staging of long B-row pieces through bulk copies (stage_off = 0: off)
  StageState stage{nullptr, nullptr, 0u, stage_off != 0};
  if (stage_off != 0) {
    const int wp = threadIdx.x >> 5;
    stage.buf = reinterpret_cast<int32_t*>(wsm + stage_off) + (size_t)wp * 2 * kStageSlots;
    stage.bar = &sbar[wp * 2];
    if ((threadIdx.x & 31) == 0) {
      mbar_init(stage.bar, 1);
      mbar_init(stage.bar + 1, 1);
      mbar_init_fence();
    }
  }
  for (int w = threadIdx.x * 4; w < words; w += blockDim.x * 4)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int s = threadIdx.x; s < nsum; s += blockDim.x) sum[s] = 0u;
  __syncthreads();
  int bad = 0;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const bool sparse = flop[i] < (long long)words;  // few words touched: walk the summary
    const int lng = wide_piece(flop, i, A.rowptr[i], A.rowptr[i + 1]);
    int c = 0;
    if (sparse) {
      // few words touched: count and clear them through the summary (such rows
      // keep nothing: walking their products again costs less than storing
      // and reloading a k-bit vector)
      wide_set_bits<true>(A, B, A.rowptr[i], A.rowptr[i + 1], lng, walk, bits, sum, words, bad,
                          stage_off ? &stage : nullptr, status);
      for (int s = threadIdx.x; s < nsum; s += blockDim.x) {
        uint32_t m = sum[s];
        sum[s] = 0u;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          const int w = s * 32 + b;
          c += __popc(bits[w]);
          bits[w] = 0u;
        }
      }
      int tot;
      block_exscan<int>(c, tmp, &tot);
      if (threadIdx.x == 0) cnt[i] = tot;
    } else {
      wide_set_bits<false>(A, B, A.rowptr[i], A.rowptr[i + 1], lng, walk, bits, sum, words, bad,
                           stage_off ? &stage : nullptr, status);
      for (int w = threadIdx.x * 4; w < words; w += blockDim.x * 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(&bits[w]);
        c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
      }
      int tot;
      block_exscan<int>(c, tmp, &tot);
      // rows whose values will go to C by atomics keep their bits for the
      // numeric phase, while slots last
      if (threadIdx.x == 0) {
        int sl = -1;
        if (keep.max_slots > 0 && tot > keep.min_cnt) {
          sl = atomicAdd(keep.next, 1);
          if (sl >= keep.max_slots) sl = -1;
          if (sl >= 0) keep.slot[i] = sl;
        }
        s_slot = sl;
      }
      __syncthreads();
      const int sl = s_slot;
      uint32_t* dst = sl >= 0 ? keep.bits + (size_t)sl * words : nullptr;
      for (int w = threadIdx.x * 4; w < words; w += blockDim.x * 4) {
        uint4* q = reinterpret_cast<uint4*>(&bits[w]);
        if (dst) *reinterpret_cast<uint4*>(&dst[w]) = *q;
        *q = make_uint4(0u, 0u, 0u, 0u);
      }
      if (threadIdx.x == 0) cnt[i] = tot;
      __syncthreads();
    }
  }
  if (bad) set_status(status, KK_ERR_BAD_INDEX);
}

// Rank tables of a row whose values go to C (rank of column c = gpre[c >> 8]
// + wpre8[c >> 5] + the popcount of its word's bits below c), from one block
// scan: thread t owns the wpt consecutive words [t * wpt, (t + 1) * wpt),
// wpt in {8, 16, 32}, and visits its 16-byte pieces in the lane-rotated order
// q = k ^ (lane & (wpt / 4 - 1)), so that a warp's loads spread over the
// shared-memory banks.  Pass 1 sums the popcounts of the thread's 8-word
// groups, the block scan gives the thread's base (and *total, the row's
// count), pass 2 writes each group's prefix and each word's offset in its
// group (at most 7 * 32, a byte).  Ends with the scan's barrier behind it; the
// caller synchronises before the tables are read.
__device__ __forceinline__ void wide_prefix_owned(const uint32_t* bits, uint32_t* gpre, uint8_t* wpre8, int wpt,
                                                  int* tmp, int* total) {
  const int t = threadIdx.x;
  const int nq = wpt >> 2;  // 16-byte pieces per thread: 2, 4 or 8
  const int sw = (t & 31) & (nq - 1);
  const uint4* b4 = reinterpret_cast<const uint4*>(bits) + (size_t)t * nq;
  int gs0 = 0, gs1 = 0, gs2 = 0, gs3 = 0;  // the thread's group popcounts (nq / 2 <= 4 groups)
  for (int k = 0; k < nq; ++k) {
    const int q = k ^ sw;
    const uint4 v = b4[q];
    const int p = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    const int g = q >> 1;
    gs0 += g == 0 ? p : 0;
    gs1 += g == 1 ? p : 0;
    gs2 += g == 2 ? p : 0;
    gs3 += g == 3 ? p : 0;
  }
  const int base = block_exscan<int>(gs0 + gs1 + gs2 + gs3, tmp, total);
  const int ng = nq >> 1;
  uint32_t* gp = gpre + (size_t)t * ng;
  gp[0] = (uint32_t)base;
  if (ng > 1) gp[1] = (uint32_t)(base + gs0);
  if (ng > 2) {
    gp[2] = (uint32_t)(base + gs0 + gs1);
    gp[3] = (uint32_t)(base + gs0 + gs1 + gs2);
  }
  uint32_t* w8 = reinterpret_cast<uint32_t*>(wpre8) + (size_t)t * nq;
  for (int k = 0; k < nq; ++k) {
    const int q = k ^ sw;
    const uint4 v = b4[q];
    int o = 0;
    if (q & 1) {  // second piece of its group: after the first piece's columns
      const uint4 e = b4[q ^ 1];
      o = __popc(e.x) + __popc(e.y) + __popc(e.z) + __popc(e.w);
    }
    const int o1 = o + __popc(v.x), o2 = o1 + __popc(v.y), o3 = o2 + __popc(v.z);
    w8[q] = (uint32_t)o | ((uint32_t)o1 << 8) | ((uint32_t)o2 << 16) | ((uint32_t)o3 << 24);
  }
}

// C's columns of a row from its bit vector and rank tables, written to
// out[0..cnt): the row's words in rounds of 32 consecutive words that warps
// claim from the shared counter *next (dense rounds cost more; claiming
// balances them across the warps, where fixed word ranges left the warps
// holding a row's dense columns behind).  In a round lane l holds word
// 32 r + l and its rank from the tables; a round whose words hold at most one
// column each is written by the lanes directly (consecutive entries), any
// other by the warp-cooperative expansion.
__device__ __forceinline__ void wide_write_columns(const uint32_t* bits, const uint32_t* gpre, const uint8_t* wpre8,
                                                   int words, int cnt, int32_t* __restrict__ out, int* next) {
  const int lane = threadIdx.x & 31;
  const int nr = words >> 5;
  for (;;) {
    int r = 0;
    if (lane == 0) r = atomicAdd(next, 1);
    r = __shfl_sync(kFull, r, 0);
    if (r >= nr) break;
    const int w = r * 32 + lane;
    const uint32_t m = bits[w];
    const int pos = (int)gpre[w >> 3] + (int)wpre8[w];
    const int c = __popc(m);
    if (__all_sync(kFull, c <= 1)) {
      if (c != 0 && pos < cnt) out[pos] = w * 32 + (__ffs(m) - 1);
    } else {
      const int p0 = __shfl_sync(kFull, pos, 0);
      const int incl = pos - p0 + c;
      const int rtot = __shfl_sync(kFull, incl, 31);
      warp_expand_bits(w, m, incl, rtot, [&](int e, int col) {
        if (p0 + e < cnt) out[p0 + e] = col;
      });
    }
  }
}

__global__ void __launch_bounds__(kWideBlock, 1)
k_num_wide(CsrView A, CsrView B, int32_t words, int32_t vcap, uint32_t sum_off, uint32_t reg_off,
           uint32_t val_off, const int64_t* __restrict__ c_rowptr, const long long* __restrict__ flop,
           const int32_t* __restrict__ rows, int32_t nrows, int32_t* __restrict__ c_colind,
           double* __restrict__ c_vals, WideKeep keep, int* status) {
  extern __shared__ __align__(16) unsigned char wsm[];
  uint32_t* bits = reinterpret_cast<uint32_t*>(wsm);
  uint32_t* sum = reinterpret_cast<uint32_t*>(wsm + sum_off);
  uint16_t* wpre16 = reinterpret_cast<uint16_t*>(wsm + reg_off);  // rows with values here
  uint32_t* gpre = reinterpret_cast<uint32_t*>(wsm + reg_off);    // rows with values in C
  uint8_t* wpre8 = wsm + reg_off + (size_t)(words / 8) * 4;       // rows with values in C
  double* vals = reinterpret_cast<double*>(wsm + val_off);
  uint16_t* list = reinterpret_cast<uint16_t*>(wsm + val_off);
  __shared__ WideWalkSmem walk;
  __shared__ int tmp[33];
  __shared__ int col_next;
  const int nsum = words >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps_blk = blockDim.x >> 5;
  for (int w = threadIdx.x * 4; w < words; w += blockDim.x * 4)
    *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
  for (int s = threadIdx.x; s < nsum; s += blockDim.x) sum[s] = 0u;
  __syncthreads();
  int bad = 0, mismatch = 0;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    const int64_t off = c_rowptr[i];
    const int cnt = (int)(c_rowptr[i + 1] - off);
    const int lng = wide_piece(flop, i, pa, pe);
    // values in shared memory (and the word list in their place) when the row fits
    const bool sparse = cnt <= vcap && cnt <= 65535;
    bool row_bad = false;
    int total;
    if (sparse) {
      wide_set_bits<true>(A, B, pa, pe, lng, walk, bits, sum, words, bad);
      // ordered list of touched words: summary words in order, bits in order,
      // in rounds of blockDim summary words
      int L = 0;
      for (int s0 = 0; s0 < nsum; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        uint32_t m = s < nsum ? sum[s] : 0u;
        int t;
        int pos = L + block_exscan<int>(__popc(m), tmp, &t);
        L += t;
        if (s < nsum) sum[s] = 0u;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          if (pos < cnt) list[pos] = (uint16_t)(s * 32 + b);
          ++pos;
        }
      }
      __syncthreads();
      if (L > cnt) {  // more touched words than the row has columns
        row_bad = true;
        L = cnt;
      }
      // per-word prefixes over the list, columns written in order
      int run = 0;
      for (int e0 = 0; e0 < L; e0 += blockDim.x) {
        const int e = e0 + threadIdx.x;
        const int w = e < L ? (int)list[e] : 0;
        uint32_t m = e < L ? bits[w] : 0u;
        int t;
        int pos = run + block_exscan<int>(__popc(m), tmp, &t);
        run += t;
        if (e < L) {
          wpre16[w] = (uint16_t)pos;
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (pos < cnt) c_colind[off + pos] = w * 32 + b;
            ++pos;
          }
        }
      }
      total = run;
      __syncthreads();
      // the list area now holds the values; the touched words are found again
      // from C's columns when they are cleared
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) vals[e] = 0.0;
    } else {
      const int sl = keep.max_slots > 0 ? keep.slot[i] : -1;
      if (sl >= 0) {  // the symbolic phase kept this row's bits
        // kKeepU 16-byte pieces per thread in flight at once; read once, so
        // streamed past L2
        const uint4* src = reinterpret_cast<const uint4*>(keep.bits + (size_t)sl * words);
        uint4* dst4 = reinterpret_cast<uint4*>(bits);
        const int n4 = words >> 2;
        for (int v0 = threadIdx.x; v0 < n4; v0 += blockDim.x * kKeepU) {
          uint4 t[kKeepU];
#pragma unroll
          for (int u = 0; u < kKeepU; ++u) {
            const int v = v0 + u * blockDim.x;
            if (v < n4) t[u] = __ldcs(&src[v]);
          }
#pragma unroll
          for (int u = 0; u < kKeepU; ++u) {
            const int v = v0 + u * blockDim.x;
            if (v < n4) dst4[v] = t[u];
          }
        }
        __syncthreads();
      } else {
        wide_set_bits<false>(A, B, pa, pe, lng, walk, bits, sum, words, bad);
      }
      const int wpw = words / nwarps_blk;  // words per warp (words is a multiple of 32 * 32)
      const int w0 = warp * wpw;
      const int wpt = words / (int)blockDim.x;
      if (wpt == 8 || wpt == 16 || wpt == 32) {
        // prefixes from one block scan over threads owning consecutive words
        if (threadIdx.x == 0) col_next = 0;  // read after the scan's barriers
        wide_prefix_owned(bits, gpre, wpre8, wpt, tmp, &total);
        __syncthreads();
        // C's columns: rounds of 32 words claimed by the warps
        wide_write_columns(bits, gpre, wpre8, words, cnt, c_colind + off, &col_next);
      } else {
        // Each warp owns a contiguous range of words, its lanes consecutive
        // words in it (conflict-free shared loads, and consecutive lanes write
        // consecutive columns of C): a warp sum, the block scan of the warp
        // sums, then per round of 32 words a warp scan gives every word its
        // prefix, kept as a u32 per 8-word group plus a byte per word.
        int mine = 0;
        for (int j = lane; j < wpw; j += 32) mine += __popc(bits[w0 + j]);
        mine = team_sum<32>(mine, kFull);
        int run = block_exscan<int>(lane == 0 ? mine : 0, tmp, &total);
        run = __shfl_sync(kFull, run, 0);
        for (int j0 = 0; j0 < wpw; j0 += 32) {
          const int w = w0 + j0 + lane;
          uint32_t m = bits[w];
          const int c = __popc(m);
          const int incl = team_inclusive_scan<32>(c, lane, kFull);
          int pos = run + incl - c;
          run += __shfl_sync(kFull, incl, 31);
          const int gbase = __shfl_sync(kFull, pos, lane & ~7);
          if ((lane & 7) == 0) gpre[w >> 3] = (uint32_t)pos;
          wpre8[w] = (uint8_t)(pos - gbase);
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (pos < cnt) c_colind[off + pos] = w * 32 + b;
            ++pos;
          }
        }
      }
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) c_vals[off + e] = 0.0;
    }
    if (total != cnt) row_bad = true;
    if (row_bad) mismatch = 1;
    __syncthreads();
    // values: rank = prefix of the word + popc(bits below the column); one
    // walk per accumulator (shared memory or C), so that a product carries
    // only its own rank lookup and add
    auto add_smem = [&](int c, double ab) {
      if ((unsigned)c < (unsigned)(words * 32)) {  // also skips the idle lanes' -1
        const int w = c >> 5;
        const uint32_t word = bits[w];
        if (!((word >> (c & 31)) & 1u)) {  // a column outside the (kept) structure
          mismatch = 1;
          return;
        }
        const int rank = (int)wpre16[w] + __popc(word & ((1u << (c & 31)) - 1u));
        if (rank < cnt) atomicAdd(&vals[rank], ab);
      }
    };
    double* __restrict__ crow = c_vals + off;
    auto add_glob = [&](int c, double ab) {
      if ((unsigned)c < (unsigned)(words * 32)) {  // also skips the idle lanes' -1
        const int w = c >> 5;
        const uint32_t word = bits[w];
        if (!((word >> (c & 31)) & 1u)) {  // a column outside the (kept) structure
          mismatch = 1;
          return;
        }
        const int rank = (int)gpre[w >> 3] + (int)wpre8[w] + __popc(word & ((1u << (c & 31)) - 1u));
        if (rank < cnt) atomicAdd(&crow[rank], ab);
      }
    };
    if (sparse) {
      if (lng) wide_walk_long<true>(A, B, pa, pe, walk.ls, lng, bad, add_smem, nullptr, nullptr, i);
      else wide_walk<true>(A, B, pa, pe, walk.ws, bad, add_smem, i);
    } else {
      if (lng) wide_walk_long<true>(A, B, pa, pe, walk.ls, lng, bad, add_glob, nullptr, nullptr, i);
      else wide_walk<true>(A, B, pa, pe, walk.ws, bad, add_glob, i);
    }
    if (sparse) {
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) c_vals[off + e] = vals[e];
    }
    if (sparse && !row_bad) {
      // clear the touched words: they are the words of this row's columns
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) bits[c_colind[off + e] >> 5] = 0u;
    } else {
      for (int w = threadIdx.x * 4; w < words; w += blockDim.x * 4)
        *reinterpret_cast<uint4*>(&bits[w]) = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
  }
  if (bad) set_status(status, KK_ERR_BAD_INDEX);
  if (mismatch) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
}

// Dynamic shared memory available to the wide kernels (their static arrays
// take the rest of the opt-in limit).
size_t wide_budget(const LaunchCtx& ctx) {
  const size_t stat = sizeof(WideWalkSmem) + 33 * sizeof(int) + 512;
  return (size_t)ctx.max_smem_optin > stat ? (size_t)ctx.max_smem_optin - stat : 0;
}

int wide_grid(const LaunchCtx& ctx, size_t smem, int nrows) {
  int per_sm = (int)(((size_t)ctx.max_smem_optin + 1024) / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2048 / kWideBlock) per_sm = 2048 / kWideBlock;
  long long g = (long long)ctx.num_sms * per_sm;
  if (g > nrows) g = nrows;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int32_t wide_word_count(int32_t k) { return wide_words(k); }

int32_t wide_keep_min_cnt(const LaunchCtx& ctx, int32_t k) {
  const WideGeom g = wide_geom(wide_words(k), wide_budget(ctx), true);
  return g.vcap < 65535 ? g.vcap : 65535;
}

bool wide_symbolic_fits(const LaunchCtx& ctx, int32_t k) {
  if (k <= 0) return false;
  return wide_geom(wide_words(k), wide_budget(ctx), false).bytes <= wide_budget(ctx);
}

bool wide_numeric_fits(const LaunchCtx& ctx, int32_t k) {
  if (k <= 0) return false;
  const WideGeom g = wide_geom(wide_words(k), wide_budget(ctx), true);
  return g.val_off <= wide_budget(ctx) && g.vcap >= 64;
}

cudaError_t launch_symbolic_wide(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                 const long long* flop, const int32_t* rows, int32_t nrows,
                                 int32_t* cnt) {
  if (nrows <= 0) return cudaSuccess;
  const int words = wide_words(B.n);
  const WideGeom g = wide_geom(words, wide_budget(ctx), false);
  // staging buffers after the bit vector, when they fit and B's columns start
  // on a 16-byte boundary (the bulk copies' rule)
  size_t bytes = g.bytes;
  uint32_t stage_off = 0;
  const size_t stage_bytes = (size_t)(kWideBlock / 32) * 2 * kStageSlots * 4;
  const size_t st_off = (g.bytes + 15) / 16 * 16;
  if (ctx.stage_long_rows && ((uintptr_t)B.colind & 15) == 0 && st_off + stage_bytes <= wide_budget(ctx) - 1024) {
    stage_off = (uint32_t)st_off;
    bytes = st_off + stage_bytes;
  }
  cudaError_t e = cudaFuncSetAttribute(k_sym_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_sym_wide<<<wide_grid(ctx, bytes, nrows), kWideBlock, bytes, ctx.stream>>>(
      A, B, words, (uint32_t)g.sum_off, stage_off, flop, rows, nrows, cnt, ctx.keep, ctx.status);
  return cudaGetLastError();
}

cudaError_t launch_numeric_wide(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                int32_t* c_colind, double* c_vals) {
  if (nrows <= 0) return cudaSuccess;
  const int words = wide_words(B.n);
  const WideGeom g = wide_geom(words, wide_budget(ctx), true);
  cudaError_t e = cudaFuncSetAttribute(k_num_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.bytes);
  if (e != cudaSuccess) return e;
  k_num_wide<<<wide_grid(ctx, g.bytes, nrows), kWideBlock, g.bytes, ctx.stream>>>(
      A, B, words, g.vcap, (uint32_t)g.sum_off, (uint32_t)g.reg_off, (uint32_t)g.val_off, c_rowptr,
      ctx.flop, rows, nrows, c_colind, c_vals, ctx.keep, ctx.status);
  return cudaGetLastError();
}

}  // namespace kk
