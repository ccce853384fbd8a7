// Analysis of B (the first pass of the symbolic phase, before the paper's
// symbolic kernel of Sec. "Standard SpGEMM Kernel"): are B's rows strictly
// ascending, are its columns inside [0, k), and -- when bc is given -- the
// compressed rows B_C of the same section: row j as (column >> 5, OR of
// 1 << (column & 31)) pairs in column order, stored at B's own row offsets,
// len[j] = number of pairs (meaningful only if B turns out sorted).
//
// One team of T lanes per row.  The team walks the row in chunks of T entries;
// the word being built when a chunk ends is carried into the next chunk, so
// every word of a sorted row gives exactly one pair.  The kernel is bound by
// the latency of its loads, so the columns of U chunks are loaded together and
// the next row's bounds are loaded while a row is walked; T and U follow B's
// mean row length (short rows: small teams, more rows in flight).
#include "kk_internal.h"
#include "kk_device.cuh"

namespace kk {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int T, int U>
__global__ void __launch_bounds__(256, 6)
k_analyze_b(CsrView B, int32_t* sorted_flag, int* status, int2* __restrict__ bc,
            int32_t* __restrict__ len, unsigned long long* pairs) {
  const int lane = threadIdx.x & 31;
  const int tl = lane & (T - 1);
  const int tbase = lane & ~(T - 1);
  const unsigned mask = team_mask<T>();
  const unsigned lt = (1u << tl) - 1u;
  const long long team0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / T;
  const long long nteams = (long long)gridDim.x * blockDim.x / T;
  int unsorted = 0, bad = 0;
  unsigned long long tot = 0;
  if (team0 == 0 && tl == 0 && B.rowptr[0] != 0) bad = 1;
  long long r = team0;
  int bs_n = 0, be_n = 0;
  if (r < B.m) {
    bs_n = B.rowptr[r];
    be_n = B.rowptr[r + 1];
  }
  for (; r < B.m; r += nteams) {
    const int bs = bs_n, be = be_n;
    if (r + nteams < B.m) {  // next row's bounds in flight while this row is walked
      bs_n = B.rowptr[r + nteams];
      be_n = B.rowptr[r + nteams + 1];
    }
    if (bs < 0 || be < bs || be > B.nnz) {
      bad = 1;
      continue;
    }
    int cw = -1, n = 0;
    uint32_t cm = 0u;
    int prev = 0;  // last column of the previous chunk
    for (int qb = bs; qb < be; qb += T * U) {
      int cu[U];  // the columns of U chunks, loaded together
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = qb + u * T + tl;
        cu[u] = q < be ? B.colind[q] : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q0 = qb + u * T;
        if (q0 >= be) break;  // uniform over the team
        const int q = q0 + tl;
        const bool valid = q < be;
        const int c = cu[u];
        int pc = __shfl_up_sync(mask, c, 1, T);
        if (tl == 0) pc = prev;
        prev = __shfl_sync(mask, c, T - 1, T);
        if (valid) {
          if ((unsigned)c >= (unsigned)B.n) bad = 1;
          if (q > bs && pc >= c) unsorted = 1;
        }
        if (!bc) continue;
        const int w = valid ? (c >> 5) : (-2 - tl);  // invalid lanes match nothing
        uint32_t acc = valid ? (1u << (c & 31)) : 0u;
        int pw = __shfl_up_sync(mask, w, 1, T);
        if (tl == 0) pw = cw;
        const bool head = valid && w != pw;
#pragma unroll
        for (int d = 1; d < T; d <<= 1) {
          const uint32_t v = __shfl_down_sync(mask, acc, d, T);
          const int w2 = __shfl_down_sync(mask, w, d, T);
          if (tl + d < T && w2 == w) acc |= v;
        }
        // a chunk that starts inside the carried word adds its first segment to it
        const uint32_t acc0 = __shfl_sync(mask, acc, 0, T);
        const bool cont0 = __shfl_sync(mask, (int)(valid && !head), 0, T) != 0;
        if (cont0) cm |= acc0;
        const unsigned hm = (__ballot_sync(mask, head) >> tbase) & ((1u << T) - 1u);
        if (hm) {
          // a new word started: the carried pair is complete
          if (cm) {
            if (tl == 0) bc[bs + n] = make_int2(cw, (int)cm);
            ++n;
          }
          const int last = 31 - __clz(hm);
          if (head && tl != last) bc[bs + n + __popc(hm & lt)] = make_int2(w, (int)acc);
          n += __popc(hm) - 1;
          cw = __shfl_sync(mask, w, last, T);
          cm = __shfl_sync(mask, acc, last, T);
        }
      }
    }
    if (bc) {
      if (cm) {
        if (tl == 0) bc[bs + n] = make_int2(cw, (int)cm);
        ++n;
      }
      if (tl == 0) {
        len[r] = n;
        tot += (unsigned long long)n;
      }
    }
  }
  unsorted = __any_sync(kFull, unsorted);
  bad = __any_sync(kFull, bad);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(kFull, tot, o);
  if (lane == 0) {
    if (unsorted) atomicAnd(sorted_flag, 0);
    if (bad) set_status(status, KK_ERR_BAD_INDEX);
    if (tot && pairs) atomicAdd(pairs, tot);
  }
}


}  // namespace

template <int T, int U>
static cudaError_t analyze_b_tu(const LaunchCtx& ctx, const CsrView& B, int32_t* sorted_flag,
                                int2* bc, int32_t* len, unsigned long long* pairs) {
  // one resident wave: the kernel strides over rows, so blocks beyond what the
  // SMs hold at once would only start late
  static int per_sm = 0;
  if (per_sm == 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_analyze_b<T, U>, 256, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = 4;
  }
  long long blocks = ((long long)B.m * T + 255) / 256;
  const long long cap = (long long)ctx.num_sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_analyze_b<T, U><<<(int)blocks, 256, 0, ctx.stream>>>(B, sorted_flag, ctx.status, bc, len, pairs);
  return cudaGetLastError();
}

cudaError_t launch_analyze_b(const LaunchCtx& ctx, const CsrView& B, int32_t* sorted_flag,
                             int2* bc, int32_t* len, unsigned long long* pairs) {
  if (B.m <= 0) return cudaSuccess;
  const long long avg = (long long)B.nnz / B.m;
  if (avg <= 2) return analyze_b_tu<1, 2>(ctx, B, sorted_flag, bc, len, pairs);
  if (avg <= 8) return analyze_b_tu<4, 2>(ctx, B, sorted_flag, bc, len, pairs);
  return analyze_b_tu<8, 4>(ctx, B, sorted_flag, bc, len, pairs);
}

}  // namespace kk
