// Symbolic phase kernels: nnz(C(i,:)) for each row of a bin (Kokkos Kernels
// paper, Sec. "Standard SpGEMM Kernel": the symbolic phase computes the number
// of nonzeros in each row of C with an accumulator that is sparse (a hash map,
// level 1 in shared memory) or dense (a bit vector)).
//
// Tiers:
//   team  - TEAM lanes per row, a private shared-memory hash set of 2^LOG2S keys;
//   CTA   - one CTA (16 warps) per row sharing one shared-memory hash set;
//   dense - one CTA per row, a shared-memory bit vector over a window of columns,
//           swept across [0, k) in chunks (the level-2 role: rows too heavy for a
//           shared-memory hash).
#include "kk_internal.h"
#include "kk_visit.cuh"

namespace kk {
namespace {

constexpr int kTeamBlock = 256;
constexpr int kCtaBlock = 512;
constexpr int kDenseBlock = 512;

struct FullRange {
  const int32_t* acol;
  const int32_t* brp;
  __device__ __forceinline__ void operator()(int p, int& bs, int& bl) const {
    const int j = acol[p];
    bs = brp[j];
    bl = brp[j + 1] - bs;
  }
};

struct NoPrep {
  __device__ __forceinline__ NoPayload operator()(int) const { return NoPayload{}; }
};

// Teams per CTA for a team-tier table of 2^LOG2S int32 keys: at most 64 KB of
// tables per CTA.
template <int TEAM, int LOG2S>
struct SymTeamGeom {
  static constexpr int kByTable = (64 * 1024) / ((1 << LOG2S) * 4);
  static constexpr int TPB = (kTeamBlock / TEAM) < kByTable ? (kTeamBlock / TEAM)
                                                             : (kByTable < 1 ? 1 : kByTable);
};

template <int TEAM, int LOG2S, bool FLAT>
__global__ void __launch_bounds__(kTeamBlock)
k_sym_team(CsrView A, CsrView B, const int32_t* __restrict__ rows, int32_t nrows,
           int32_t* __restrict__ cnt, int* status) {
  extern __shared__ int smem_i[];
  constexpr int S = 1 << LOG2S;
  constexpr int TPB = SymTeamGeom<TEAM, LOG2S>::TPB;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x % TEAM;
  const unsigned mask = team_mask<TEAM>();
  int* tab = smem_i + team * S;
  const FullRange rng{A.colind, B.rowptr};
  for (int r = blockIdx.x * TPB + team; r < nrows; r += gridDim.x * TPB) {
    const int i = rows[r];
    for (int s = tl; s < S; s += TEAM) tab[s] = kEmptyKey;
    __syncwarp(mask);
    int mine = 0;
    const int32_t* bcol = B.colind;
    visit_products<TEAM, FLAT, NoPayload>(
        A.rowptr[i], A.rowptr[i + 1], 0, 1, tl, mask, rng, NoPrep{},
        [&](NoPayload, int, int q) { mine += set_insert(tab, bcol[q], LOG2S, status); });
    mine = team_sum<TEAM>(mine, mask);
    if (tl == 0) cnt[i] = mine;
    __syncwarp(mask);
  }
}

// Warp-per-row vector kernel: one warp per row, lanes split each B row, the
// row's A entries staged once in shared memory (bs, len) and read back as
// broadcasts.  Rows are split into contiguous shares per CTA so neighbouring
// rows reuse B rows through L1.
template <int LOG2S>
__global__ void __launch_bounds__(256)
k_sym_warp_vec(CsrView A, CsrView B, const int32_t* __restrict__ rows, int32_t nrows,
               int32_t* __restrict__ cnt, int* status) {
  constexpr int S = 1 << LOG2S;
  constexpr int WPB = 8;
  extern __shared__ __align__(16) int smem_w[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* tab = smem_w + warp * (S + 64);
  int2* ainfo = reinterpret_cast<int2*>(tab + S);
  const int32_t* __restrict__ acol = A.colind;
  const int32_t* __restrict__ brp = B.rowptr;
  const int32_t* __restrict__ bcol = B.colind;
  const int per_cta = (nrows + gridDim.x - 1) / gridDim.x;
  const int r_begin = blockIdx.x * per_cta;
  const int r_end = min(nrows, r_begin + per_cta);
  for (int r = r_begin + warp; r < r_end; r += WPB) {
    const int i = rows[r];
#pragma unroll
    for (int s = lane * 4; s < S; s += 128) *reinterpret_cast<int4*>(&tab[s]) = make_int4(-1, -1, -1, -1);
    __syncwarp();
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    int mine = 0;
    for (int p0 = pa; p0 < pe; p0 += 32) {
      const int p = p0 + lane;
      int2 info = make_int2(0, 0);
      if (p < pe) {
        const int j = acol[p];
        info.x = brp[j];
        info.y = brp[j + 1] - info.x;
      }
      ainfo[lane] = info;
      __syncwarp();
      const int nch = min(32, pe - p0);
      const unsigned maxlen = __reduce_max_sync(0xffffffffu, (unsigned)info.y);
      if (maxlen <= 32u) {
        // issue the loads of kBatch A entries' B rows before inserting them
        constexpr int kBatch = 8;
        for (int t0 = 0; t0 < nch; t0 += kBatch) {
          int cols[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            cols[u] = -1;
            if (t0 + u < nch) {
              const int2 in = ainfo[t0 + u];
              if (lane < in.y) cols[u] = bcol[in.x + lane];
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u)
            if (cols[u] >= 0) mine += set_insert(tab, cols[u], LOG2S, status);
        }
      } else {
        for (int t = 0; t < nch; ++t) {
          const int2 in = ainfo[t];
          for (int q0 = lane; q0 < in.y; q0 += 32) mine += set_insert(tab, bcol[in.x + q0], LOG2S, status);
        }
      }
      __syncwarp();
    }
    mine = team_sum<32>(mine, 0xffffffffu);
    if (lane == 0) cnt[i] = mine;
    __syncwarp();
  }
}

template <int LOG2S>
__global__ void __launch_bounds__(kCtaBlock)
k_sym_cta(CsrView A, CsrView B, const int32_t* __restrict__ rows, int32_t nrows,
          int32_t* __restrict__ cnt, int* status) {
  extern __shared__ int smem_i[];
  constexpr int S = 1 << LOG2S;
  __shared__ int red[kCtaBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  int* tab = smem_i;
  const FullRange rng{A.colind, B.rowptr};
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    for (int s = threadIdx.x; s < S; s += blockDim.x) tab[s] = kEmptyKey;
    __syncthreads();
    int mine = 0;
    const int32_t* bcol = B.colind;
    visit_products<32, true, NoPayload>(
        A.rowptr[i], A.rowptr[i + 1], warp, nwarps, lane, 0xffffffffu, rng, NoPrep{},
        [&](NoPayload, int, int q) { mine += set_insert(tab, bcol[q], LOG2S, status); });
    mine = team_sum<32>(mine, 0xffffffffu);
    if (lane == 0) red[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < nwarps; ++w) t += red[w];
      cnt[i] = t;
    }
    __syncthreads();
  }
}

// Dense tier: bit vector over columns [c0, c0 + W) in shared memory.  With
// several chunks and sorted B rows, each B row is cut to the chunk by binary
// search; unsorted B rows are filtered entry by entry.
__global__ void __launch_bounds__(kDenseBlock)
k_sym_dense(CsrView A, CsrView B, int32_t b_sorted, int32_t k, int32_t W,
            const int32_t* __restrict__ rows, int32_t nrows, int32_t* __restrict__ cnt,
            int* status) {
  extern __shared__ uint32_t bits[];
  __shared__ int red[kDenseBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int words = W >> 5;
  const int32_t* acol = A.colind;
  const int32_t* brp = B.rowptr;
  const int32_t* bcol = B.colind;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    int total = 0;
    for (long long c0l = 0; c0l < k; c0l += W) {
      const int c0 = (int)c0l;
      const int cend = (k - c0 > W) ? c0 + W : k;
      const bool whole = (k <= W) || !b_sorted;
      for (int w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
      __syncthreads();
      auto rng = [&](int p, int& bs, int& bl) {
        const int j = acol[p];
        int lo = brp[j], hi = brp[j + 1];
        if (!whole) {
          lo = lower_bound_i32(bcol, lo, hi, c0);
          hi = lower_bound_i32(bcol, lo, hi, cend);
        }
        bs = lo;
        bl = hi - lo;
      };
      visit_products<32, true, NoPayload>(
          pa, pe, warp, nwarps, lane, 0xffffffffu, rng, NoPrep{}, [&](NoPayload, int, int q) {
            const uint32_t off = (uint32_t)(bcol[q] - c0);
            if (off < (uint32_t)W) atomicOr(&bits[off >> 5], 1u << (off & 31));
          });
      __syncthreads();
      int mine = 0;
      for (int w = threadIdx.x; w < words; w += blockDim.x) mine += __popc(bits[w]);
      mine = team_sum<32>(mine, 0xffffffffu);
      if (lane == 0) red[warp] = mine;
      __syncthreads();
      for (int w = 0; w < nwarps; ++w) total += red[w];
      __syncthreads();
    }
    if (threadIdx.x == 0) cnt[i] = total;
  }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int TEAM, int LOG2S, bool FLAT>
cudaError_t launch_team(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                        const int32_t* rows, int32_t nrows, int32_t* cnt) {
  constexpr int tpb = SymTeamGeom<TEAM, LOG2S>::TPB;
  const size_t smem = (size_t)tpb * (1u << LOG2S) * sizeof(int);
  auto kern = k_sym_team<TEAM, LOG2S, FLAT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long blocks = (nrows + tpb - 1) / tpb;
  blocks = blocks > (long long)ctx.num_sms * 32 ? (long long)ctx.num_sms * 32 : blocks;
  kern<<<(unsigned)blocks, tpb * TEAM, smem, ctx.stream>>>(A, B, rows, nrows, cnt, ctx.status);
  return cudaGetLastError();
}

template <int TEAM, bool FLAT>
cudaError_t dispatch_team_slots(const LaunchCtx& ctx, int log2s, const CsrView& A,
                                const CsrView& B, const int32_t* rows, int32_t nrows,
                                int32_t* cnt) {
  switch (log2s) {
    case 5: return launch_team<TEAM, 5, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 6: return launch_team<TEAM, 6, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 7: return launch_team<TEAM, 7, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 8: return launch_team<TEAM, 8, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 9: return launch_team<TEAM, 9, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 10: return launch_team<TEAM, 10, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 11: return launch_team<TEAM, 11, FLAT>(ctx, A, B, rows, nrows, cnt);
    case 12: return launch_team<TEAM, 12, FLAT>(ctx, A, B, rows, nrows, cnt);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOG2S>
cudaError_t launch_warp_vec(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                            const int32_t* rows, int32_t nrows, int32_t* cnt) {
  const size_t smem = (size_t)8 * ((1u << LOG2S) + 64) * sizeof(int);
  auto kern = k_sym_warp_vec<LOG2S>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long blocks = (nrows + 31) / 32;
  const long long cap = (long long)ctx.num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, 256, smem, ctx.stream>>>(A, B, rows, nrows, cnt, ctx.status);
  return cudaGetLastError();
}

template <int LOG2S>
cudaError_t launch_cta(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                       const int32_t* rows, int32_t nrows, int32_t* cnt) {
  const size_t smem = (size_t)(1u << LOG2S) * sizeof(int);
  auto kern = k_sym_cta<LOG2S>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long blocks = nrows < ctx.num_sms * 8 ? nrows : ctx.num_sms * 8;
  kern<<<(unsigned)blocks, kCtaBlock, smem, ctx.stream>>>(A, B, rows, nrows, cnt, ctx.status);
  return cudaGetLastError();
}

}  // namespace

size_t symbolic_smem_bytes(const BinSpec& bin) {
  if (bin.tier == kTierTeam) {
    int tpb = kTeamBlock / bin.team, by = (64 * 1024) / (bin.slots * 4);
    if (by < 1) by = 1;
    return (size_t)(tpb < by ? tpb : by) * bin.slots * sizeof(int);
  }
  if (bin.tier == kTierCta) return (size_t)bin.slots * sizeof(int);
  return (size_t)bin.slots / 8;
}

cudaError_t launch_symbolic_bin(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                const CsrView& B, int32_t b_sorted, const int32_t* rows,
                                int32_t nrows, int32_t* cnt) {
  if (nrows <= 0) return cudaSuccess;
  if (bin.tier == kTierThread) return launch_symbolic_thread(ctx, A, B, rows, nrows, cnt);
  int log2s = 0;
  while ((1 << log2s) < bin.slots) ++log2s;
  if (bin.tier == kTierTeam && !bin.flat && bin.team == 32 && log2s >= 5 && log2s <= 12) {
    timer_begin(ctx.timer, ctx.stream, "sym_warp_vec");
    cudaError_t e = cudaErrorInvalidValue;
    switch (log2s) {
      case 5: e = launch_warp_vec<5>(ctx, A, B, rows, nrows, cnt); break;
      case 6: e = launch_warp_vec<6>(ctx, A, B, rows, nrows, cnt); break;
      case 7: e = launch_warp_vec<7>(ctx, A, B, rows, nrows, cnt); break;
      case 8: e = launch_warp_vec<8>(ctx, A, B, rows, nrows, cnt); break;
      case 9: e = launch_warp_vec<9>(ctx, A, B, rows, nrows, cnt); break;
      case 10: e = launch_warp_vec<10>(ctx, A, B, rows, nrows, cnt); break;
      case 11: e = launch_warp_vec<11>(ctx, A, B, rows, nrows, cnt); break;
      case 12: e = launch_warp_vec<12>(ctx, A, B, rows, nrows, cnt); break;
    }
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  if (bin.tier == kTierTeam) {
    timer_begin(ctx.timer, ctx.stream, bin.flat ? "sym_team_flat" : "sym_team_vec");
    cudaError_t e = cudaErrorInvalidValue;
    if (bin.flat) {
      if (bin.team == 8) e = dispatch_team_slots<8, true>(ctx, log2s, A, B, rows, nrows, cnt);
      else if (bin.team == 32) e = dispatch_team_slots<32, true>(ctx, log2s, A, B, rows, nrows, cnt);
    } else {
      if (bin.team == 8) e = dispatch_team_slots<8, false>(ctx, log2s, A, B, rows, nrows, cnt);
      else if (bin.team == 32) e = dispatch_team_slots<32, false>(ctx, log2s, A, B, rows, nrows, cnt);
    }
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  if ((bin.tier == kTierCta || bin.tier == kTierDense) && ctx.flop && wide_symbolic_fits(ctx, B.n)) {
    timer_begin(ctx.timer, ctx.stream, "sym_wide");
    cudaError_t e = launch_symbolic_wide(ctx, A, B, ctx.flop, rows, nrows, cnt);
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  if (bin.tier == kTierCta) {
    timer_begin(ctx.timer, ctx.stream, "sym_cta");
    cudaError_t e;
    switch (log2s) {
      case 13: e = launch_cta<13>(ctx, A, B, rows, nrows, cnt); break;
      case 14: e = launch_cta<14>(ctx, A, B, rows, nrows, cnt); break;
      case 15: e = launch_cta<15>(ctx, A, B, rows, nrows, cnt); break;
      default: e = cudaErrorInvalidValue;
    }
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  // dense
  timer_begin(ctx.timer, ctx.stream, "sym_dense");
  const size_t smem = (size_t)bin.slots / 8;
  cudaError_t e = set_smem(k_sym_dense, smem);
  if (e == cudaSuccess) {
    long long blocks = nrows < ctx.num_sms ? nrows : ctx.num_sms;
    k_sym_dense<<<(unsigned)blocks, kDenseBlock, smem, ctx.stream>>>(
        A, B, b_sorted, B.n, bin.slots, rows, nrows, cnt, ctx.status);
    e = cudaGetLastError();
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

}  // namespace kk
