// Batched form (kk_batched.h): all products of a batch share one global row
// space; rows are binned across the batch and one persistent kernel per phase
// drains a work queue of (bin, row tile) items.  The per-row routines are the
// warp and CTA hash accumulators of the plain form with the table size chosen
// at run time from the row's bin.
#include "kk_internal.h"
#include "kk_rowops.cuh"
#include "kk_visit.cuh"

namespace kk {
namespace {

constexpr int kBBlock = 256;            // 8 warps
constexpr int kBWarps = kBBlock / 32;
constexpr int kBSmem = 64 * 1024;       // dynamic shared memory per CTA
constexpr int kBWarpBytes = kBSmem / kBWarps;
constexpr int kBRowsPerWarpTile = 4;    // rows per warp in one warp-bin tile

struct NoPrepB {
  __device__ __forceinline__ NoPayload operator()(int) const { return NoPayload{}; }
};

__device__ __forceinline__ uint8_t bclassify(const BBinTable& t, long long q, int flat) {
  if (q <= 0) return 0xFF;
  for (int b = 0; b < t.nb; ++b)
    if (q <= t.hi[b] && (t.kind[b] == 1 || t.flat[b] == flat)) return (uint8_t)b;
  return 0xFE;  // beyond the batched accumulators
}

__global__ void k_b_rowpair(int32_t count, const PairDesc* __restrict__ d, int32_t* __restrict__ row_pair) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const long long base = d[k].row_base;
    for (int i = threadIdx.x; i < d[k].A.m; i += blockDim.x) row_pair[base + i] = k;
  }
}

// Per pair: B structure valid?  rows strictly ascending?
__global__ void k_b_analyze_b(int32_t count, PairDesc* __restrict__ d, int* status) {
  __shared__ int s_unsorted, s_bad;
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    if (threadIdx.x == 0) {
      s_unsorted = 0;
      s_bad = d[k].B.m > 0 && d[k].B.rowptr[0] != 0;
    }
    __syncthreads();
    const CsrView B = d[k].B;
    int uns = 0, bad = 0;
    for (int r = threadIdx.x; r < B.m; r += blockDim.x) {
      const int bs = B.rowptr[r], be = B.rowptr[r + 1];
      if (bs < 0 || be < bs || be > B.nnz) {
        bad = 1;
        continue;
      }
      for (int q = bs; q < be; ++q) {
        const int c = B.colind[q];
        if ((unsigned)c >= (unsigned)B.n) bad = 1;
        if (q > bs && B.colind[q - 1] >= c) uns = 1;
      }
    }
    if (uns) s_unsorted = 1;
    if (bad) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
      d[k].b_sorted = s_unsorted ? 0 : 1;
      if (s_bad) set_status(status, KK_ERR_BAD_INDEX);
    }
    __syncthreads();
  }
}

// Team of 8 lanes per global row: flop bound and symbolic bin.
__global__ void k_b_analyze_a(long long R, const PairDesc* __restrict__ d, const int32_t* __restrict__ row_pair,
                              BBinTable tab, int32_t vec_min_len, long long* __restrict__ flop,
                              uint8_t* __restrict__ bin, unsigned long long* total_flop, int* status) {
  constexpr int T = 8;
  const int tl = threadIdx.x % T;
  const unsigned mask = team_mask<T>();
  const long long team0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / T;
  const long long nteams = (long long)gridDim.x * blockDim.x / T;
  const long long iters = (R + nteams - 1) / nteams;
  unsigned long long acc = 0;
  for (long long it = 0; it < iters; ++it) {
    const long long g = team0 + it * nteams;
    long long f = 0;
    int bad = 0, nza = 0;
    if (g < R) {
      const PairDesc& p = d[row_pair[g]];
      const int i = (int)(g - p.row_base);
      int pa = p.A.rowptr[i], pe = p.A.rowptr[i + 1];
      if (pa < 0 || pe < pa || pe > p.A.nnz || (i == 0 && pa != 0)) {
        bad = 1;
        pe = pa;
      }
      nza = pe - pa;
      for (int q = pa + tl; q < pe; q += T) {
        const int j = p.A.colind[q];
        if ((unsigned)j >= (unsigned)p.B.m) {
          bad = 1;
          continue;
        }
        f += p.B.rowptr[j + 1] - p.B.rowptr[j];
      }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) f += __shfl_xor_sync(mask, f, o, T);
    if (bad) set_status(status, KK_ERR_BAD_INDEX);
    if (g < R && tl == 0) {
      flop[g] = f;
      const uint8_t b = bclassify(tab, f, f < (long long)vec_min_len * nza ? 1 : 0);
      if (b == 0xFE) set_status(status, KK_ERR_CAPACITY);
      bin[g] = b == 0xFE ? (uint8_t)0xFF : b;
      acc += (unsigned long long)f;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total_flop, acc);
}

// Numeric bins from C's row counts.
__global__ void k_b_nclassify(long long R, const PairDesc* __restrict__ d, const int32_t* __restrict__ row_pair,
                              const int64_t* __restrict__ rowptr, const long long* __restrict__ flop,
                              BBinTable tab, int32_t vec_min_len, uint8_t* __restrict__ bin, int* status) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < R;
       g += (long long)gridDim.x * blockDim.x) {
    const PairDesc& p = d[row_pair[g]];
    const int i = (int)(g - p.row_base);
    const int nza = p.A.rowptr[i + 1] - p.A.rowptr[i];
    const uint8_t b = bclassify(tab, rowptr[g + 1] - rowptr[g], flop[g] < (long long)vec_min_len * nza ? 1 : 0);
    if (b == 0xFE) set_status(status, KK_ERR_CAPACITY);
    bin[g] = b == 0xFE ? (uint8_t)0xFF : b;
  }
}

// Tile prefix per bin: warp bins take kBWarps * kBRowsPerWarpTile rows per
// tile, CTA bins one row.
__global__ void k_b_tileprefix(BBinTable tab, const int32_t* __restrict__ bin_start,
                               int32_t* __restrict__ tile_prefix) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int acc = 0;
  for (int b = 0; b < tab.nb; ++b) {
    tile_prefix[b] = acc;
    const int n = bin_start[b + 1] - bin_start[b];
    const int per = tab.kind[b] == 0 ? kBWarps * kBRowsPerWarpTile : 1;
    acc += (n + per - 1) / per;
  }
  tile_prefix[tab.nb] = acc;
}

__global__ void k_b_split(int32_t count, PairDesc* __restrict__ d, float2* __restrict__ split) {
  __shared__ int s_bad;
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const CsrView B = d[k].B;
    float2* out = split + d[k].split_base;
    int bad = 0;
    for (int q = threadIdx.x; q < B.nnz; q += blockDim.x) {
      DF t;
      bad |= df_split(B.vals[q], t) ? 0 : 1;
      out[q] = make_float2(t.hi, t.lo);
    }
    if (bad) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0) d[k].range_bad = s_bad;
    __syncthreads();
  }
}

__global__ void k_b_offsets(int32_t count, const PairDesc* __restrict__ d, long long R,
                            const int64_t* __restrict__ rowptr, int64_t* __restrict__ off) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= count; k += gridDim.x * blockDim.x)
    off[k] = rowptr[k < count ? d[k].row_base : R];
}

// Decode a tile index into (bin, first row position, end position).
__device__ __forceinline__ void decode_tile(int t, int nb, const int* s_tp, const int* s_bs, const BBinTable& tab,
                                            int& b, int& start, int& end) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_tp[mid] <= t) lo = mid; else hi = mid - 1;
  }
  b = lo;
  const int per = tab.kind[b] == 0 ? kBWarps * kBRowsPerWarpTile : 1;
  start = s_bs[b] + (t - s_tp[b]) * per;
  end = min(start + per, s_bs[b + 1]);
}

// --------------------------------------------------------------------------
// Persistent symbolic kernel
// --------------------------------------------------------------------------
__device__ __forceinline__ int warp_sym_row(const PairDesc& p, int i, int* tab, int log2s, bool flat,
                                            int lane, int* status) {
  const int S = 1 << log2s;
  for (int s = lane; s < S; s += 32) tab[s] = kEmptyKey;
  __syncwarp();
  const FullRange rng{p.A.colind, p.B.rowptr};
  const int32_t* bcol = p.B.colind;
  int mine = 0;
  auto ins = [&](NoPayload, int, int q) { mine += set_insert(tab, bcol[q], log2s, status); };
  if (flat)
    visit_products<32, true, NoPayload>(p.A.rowptr[i], p.A.rowptr[i + 1], 0, 1, lane, 0xffffffffu, rng, NoPrepB{}, ins);
  else
    visit_products<32, false, NoPayload>(p.A.rowptr[i], p.A.rowptr[i + 1], 0, 1, lane, 0xffffffffu, rng, NoPrepB{}, ins);
  mine = team_sum<32>(mine, 0xffffffffu);
  __syncwarp();
  return mine;
}

__device__ __forceinline__ int cta_sym_row(const PairDesc& p, int i, int* tab, int log2s, int* red, int* status) {
  const int S = 1 << log2s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int s = threadIdx.x; s < S; s += blockDim.x) tab[s] = kEmptyKey;
  __syncthreads();
  const FullRange rng{p.A.colind, p.B.rowptr};
  const int32_t* bcol = p.B.colind;
  int mine = 0;
  visit_products<32, true, NoPayload>(p.A.rowptr[i], p.A.rowptr[i + 1], warp, kBWarps, lane, 0xffffffffu, rng,
                                      NoPrepB{}, [&](NoPayload, int, int q) {
                                        mine += set_insert(tab, bcol[q], log2s, status);
                                      });
  mine = team_sum<32>(mine, 0xffffffffu);
  if (lane == 0) red[warp] = mine;
  __syncthreads();
  int t = 0;
  for (int w = 0; w < kBWarps; ++w) t += red[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(kBBlock)
k_b_symbolic(const PairDesc* __restrict__ d, const int32_t* __restrict__ row_pair,
             const int32_t* __restrict__ rows, const int32_t* __restrict__ bin_start,
             const int32_t* __restrict__ tile_prefix, BBinTable tab, int* queue,
             int32_t* __restrict__ cnt, int* status) {
  extern __shared__ __align__(16) int smem_b[];
  __shared__ int s_tp[kMaxBBins + 1], s_bs[kMaxBBins + 1], s_tile, red[kBWarps];
  for (int b = threadIdx.x; b <= tab.nb; b += blockDim.x) {
    s_tp[b] = tile_prefix[b];
    s_bs[b] = bin_start[b];
  }
  __syncthreads();
  const int ntiles = s_tp[tab.nb];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= ntiles) break;
    int b, start, end;
    decode_tile(t, tab.nb, s_tp, s_bs, tab, b, start, end);
    if (tab.kind[b] == 0) {
      int* tabw = smem_b + warp * (kBWarpBytes / 4);
      for (int r = start + warp; r < end; r += kBWarps) {
        const int g = rows[r];
        const PairDesc& p = d[row_pair[g]];
        const int c = warp_sym_row(p, (int)(g - p.row_base), tabw, tab.log2s[b], tab.flat[b] != 0, lane, status);
        if (lane == 0) cnt[g] = c;
      }
    } else {
      const int g = rows[start];
      const PairDesc& p = d[row_pair[g]];
      const int c = cta_sym_row(p, (int)(g - p.row_base), smem_b, tab.log2s[b], red, status);
      if (threadIdx.x == 0) cnt[g] = c;
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// Persistent numeric kernel
// --------------------------------------------------------------------------
__device__ __forceinline__ void warp_num_row(const PairDesc& p, int i, long long g, const int64_t* rowptr,
                                             unsigned char* base, int log2s, bool flat, bool df_all,
                                             const float2* split, int32_t* ccol, double* cval, int lane,
                                             int* status) {
  const int S = 1 << log2s;
  const int H = S / 2;
  u64* vals = reinterpret_cast<u64*>(base);
  u64* sbuf = vals + S;
  int* keys = reinterpret_cast<int*>(sbuf + H);
  const int64_t off = rowptr[g];
  const int cnt = (int)(rowptr[g + 1] - off);
  for (int s = lane; s < S; s += 32) {
    keys[s] = kEmptyKey;
    vals[s] = 0ull;
  }
  __syncwarp();
  const int pa = p.A.rowptr[i], pe = p.A.rowptr[i + 1];
  const bool df = df_all && p.range_bad == 0 && p.b_sorted && df_row_terms_ok(pa, pe) &&
                  row_df_ok<32>(p.A.vals, pa, pe, lane, 0xffffffffu);
  const bool atomic = flat || !p.b_sorted;
  const FullRange rng{p.A.colind, p.B.rowptr};
  const int32_t* bcol = p.B.colind;
  const double* bval = p.B.vals;
  const float2* bspl = split + p.split_base;
  if (df) {
    auto f = [&](DF a, int, int q) {
      const int slot = map_slot(keys, bcol[q], log2s, status);
      if (slot >= 0) upd_df(vals, slot, a, load_b(bspl, q), atomic, status);
    };
    if (flat) visit_products<32, true, DF>(pa, pe, 0, 1, lane, 0xffffffffu, rng, PrepDF{p.A, i}, f);
    else visit_products<32, false, DF>(pa, pe, 0, 1, lane, 0xffffffffu, rng, PrepDF{p.A, i}, f);
  } else {
    auto f = [&](double a, int, int q) {
      const int slot = map_slot(keys, bcol[q], log2s, status);
      if (slot >= 0) upd_f64(vals, slot, a, bval[q], atomic);
    };
    if (flat) visit_products<32, true, double>(pa, pe, 0, 1, lane, 0xffffffffu, rng, PrepF64{p.A, i}, f);
    else visit_products<32, false, double>(pa, pe, 0, 1, lane, 0xffffffffu, rng, PrepF64{p.A, i}, f);
  }
  __syncwarp();
  int n = 0;
  for (int s0 = 0; s0 < S; s0 += 32) {
    const int s = s0 + lane;
    const int key = keys[s];
    const bool occ = key != kEmptyKey;
    const unsigned bal = __ballot_sync(0xffffffffu, occ);
    const int pos = n + __popc(bal & ((1u << lane) - 1u));
    if (occ && pos < H) sbuf[pos] = ((u64)(uint32_t)key << 32) | (u64)s;
    n += __popc(bal);
  }
  if (n != cnt && lane == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  const int nn = max(0, min(min(n, cnt), H));
  const int P = pow2ceil(nn);
  for (int t = nn + lane; t < P; t += 32) sbuf[t] = ~0ull;
  __syncwarp();
  team_bitonic<32>(sbuf, P, lane, 0xffffffffu);
  for (int t = lane; t < nn; t += 32) {
    const u64 it = sbuf[t];
    ccol[off + t] = (int32_t)(it >> 32);
    cval[off + t] = out_value(vals[(uint32_t)it], df);
  }
  __syncwarp();
}

__device__ __forceinline__ void cta_num_row(const PairDesc& p, int i, long long g, const int64_t* rowptr,
                                            unsigned char* base, int log2s, bool df_all, const float2* split,
                                            int32_t* ccol, double* cval, int* scan_scratch, int* flag,
                                            int* status) {
  const int S = 1 << log2s;
  const int H = S / 2;
  u64* vals = reinterpret_cast<u64*>(base);
  u64* sbuf = vals + S;
  int* keys = reinterpret_cast<int*>(sbuf + H);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t off = rowptr[g];
  const int cnt = (int)(rowptr[g + 1] - off);
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    keys[s] = kEmptyKey;
    vals[s] = 0ull;
  }
  const int pa = p.A.rowptr[i], pe = p.A.rowptr[i + 1];
  const bool df = df_all && p.range_bad == 0 && p.b_sorted && df_row_terms_ok(pa, pe) &&
                  block_df_ok(p.A.vals, pa, pe, flag);  // syncs
  const FullRange rng{p.A.colind, p.B.rowptr};
  const int32_t* bcol = p.B.colind;
  const double* bval = p.B.vals;
  const float2* bspl = split + p.split_base;
  if (df) {
    visit_products<32, true, DF>(pa, pe, warp, kBWarps, lane, 0xffffffffu, rng, PrepDF{p.A, i},
                                 [&](DF a, int, int q) {
                                   const int slot = map_slot(keys, bcol[q], log2s, status);
                                   if (slot >= 0) upd_df(vals, slot, a, load_b(bspl, q), true, status);
                                 });
  } else {
    visit_products<32, true, double>(pa, pe, warp, kBWarps, lane, 0xffffffffu, rng, PrepF64{p.A, i},
                                     [&](double a, int, int q) {
                                       const int slot = map_slot(keys, bcol[q], log2s, status);
                                       if (slot >= 0) upd_f64(vals, slot, a, bval[q], true);
                                     });
  }
  __syncthreads();
  int n = 0;
  for (int s0 = 0; s0 < S; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const int occ = (s < S && keys[s] != kEmptyKey) ? 1 : 0;
    int tot;
    const int pos = n + block_exclusive_scan(occ, scan_scratch, &tot);
    if (occ && pos < H) sbuf[pos] = ((u64)(uint32_t)keys[s] << 32) | (u64)s;
    n += tot;
  }
  if (n != cnt && threadIdx.x == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  const int nn = max(0, min(min(n, cnt), H));
  const int P = pow2ceil(nn);
  for (int t = nn + threadIdx.x; t < P; t += blockDim.x) sbuf[t] = ~0ull;
  __syncthreads();
  block_bitonic(sbuf, P);
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const u64 it = sbuf[t];
    ccol[off + t] = (int32_t)(it >> 32);
    cval[off + t] = out_value(vals[(uint32_t)it], df);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBBlock)
k_b_numeric(const PairDesc* __restrict__ d, const int32_t* __restrict__ row_pair,
            const int32_t* __restrict__ rows, const int32_t* __restrict__ bin_start,
            const int32_t* __restrict__ tile_prefix, BBinTable tab, int* queue, int32_t arith,
            const float2* __restrict__ split, const int64_t* __restrict__ rowptr,
            int32_t* __restrict__ ccol, double* __restrict__ cval, int* status) {
  extern __shared__ __align__(16) unsigned char smem_nb[];
  __shared__ int s_tp[kMaxBBins + 1], s_bs[kMaxBBins + 1], s_tile, scan_scratch[33], flag;
  for (int b = threadIdx.x; b <= tab.nb; b += blockDim.x) {
    s_tp[b] = tile_prefix[b];
    s_bs[b] = bin_start[b];
  }
  __syncthreads();
  const int ntiles = s_tp[tab.nb];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool df_all = arith == kArithDF32;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    const int t = s_tile;
    __syncthreads();
    if (t >= ntiles) break;
    int b, start, end;
    decode_tile(t, tab.nb, s_tp, s_bs, tab, b, start, end);
    if (tab.kind[b] == 0) {
      unsigned char* base = smem_nb + (size_t)warp * kBWarpBytes;
      for (int r = start + warp; r < end; r += kBWarps) {
        const int g = rows[r];
        const PairDesc& p = d[row_pair[g]];
        warp_num_row(p, (int)(g - p.row_base), g, rowptr, base, tab.log2s[b], tab.flat[b] != 0, df_all,
                     split, ccol, cval, lane, status);
      }
    } else {
      const int g = rows[start];
      const PairDesc& p = d[row_pair[g]];
      cta_num_row(p, (int)(g - p.row_base), g, rowptr, smem_nb, tab.log2s[b], df_all, split, ccol, cval,
                  scan_scratch, &flag, status);
    }
    __syncthreads();
  }
}

int persist_grid(int num_sms) {
  return num_sms * (228 * 1024 / (kBSmem + 4096));  // CTAs resident per SM by shared memory
}

}  // namespace

void batched_bin_tables(BBinTable& sym, BBinTable& num, int sym_load_pct, int num_load_pct) {
  sym = BBinTable{};
  num = BBinTable{};
  // symbolic, keyed by flop bound: warp tables of 2^5..2^11 keys (load <= sym_load_pct), vector
  // and flattened; numeric rows fill at most num_load_pct (<= 50) of their map
  for (int ls = 5; ls <= 11; ++ls) {
    for (int fl = 0; fl < 2; ++fl) {
      sym.kind[sym.nb] = 0;
      sym.log2s[sym.nb] = ls;
      sym.flat[sym.nb] = fl;
      sym.hi[sym.nb] = ((1ll << ls) * sym_load_pct) / 100;
      ++sym.nb;
    }
  }
  for (int ls = 12; ls <= 14; ++ls) {  // CTA tables up to 64 KB
    sym.kind[sym.nb] = 1;
    sym.log2s[sym.nb] = ls;
    sym.flat[sym.nb] = 1;
    sym.hi[sym.nb] = ((1ll << ls) * sym_load_pct) / 100;
    ++sym.nb;
  }
  // numeric, keyed by nnz(C(i,:)): warp maps 2^5..2^9 slots (16 B per slot), CTA 2^10..2^12
  for (int ls = 5; ls <= 9; ++ls) {
    for (int fl = 0; fl < 2; ++fl) {
      num.kind[num.nb] = 0;
      num.log2s[num.nb] = ls;
      num.flat[num.nb] = fl;
      num.hi[num.nb] = ((1ll << ls) * num_load_pct) / 100;
      ++num.nb;
    }
  }
  for (int ls = 10; ls <= 12; ++ls) {
    num.kind[num.nb] = 1;
    num.log2s[num.nb] = ls;
    num.flat[num.nb] = 1;
    num.hi[num.nb] = ((1ll << ls) * num_load_pct) / 100;
    ++num.nb;
  }
}

cudaError_t launch_b_prepare(cudaStream_t s, int num_sms, int32_t count, PairDesc* d, long long R,
                             int32_t* row_pair, int* status) {
  if (count <= 0) return cudaSuccess;
  const int g = count < num_sms * 8 ? count : num_sms * 8;
  k_b_rowpair<<<g, 256, 0, s>>>(count, d, row_pair);
  k_b_analyze_b<<<g, 256, 0, s>>>(count, d, status);
  return cudaGetLastError();
}

cudaError_t launch_b_analyze_a(cudaStream_t s, int num_sms, long long R, const PairDesc* d,
                               const int32_t* row_pair, const BBinTable& tab, int32_t vec_min_len,
                               long long* flop, uint8_t* bin, unsigned long long* total_flop, int* status) {
  if (R <= 0) return cudaSuccess;
  long long g = (R * 8 + 255) / 256;
  if (g > num_sms * 16) g = num_sms * 16;
  k_b_analyze_a<<<(unsigned)g, 256, 0, s>>>(R, d, row_pair, tab, vec_min_len, flop, bin, total_flop, status);
  return cudaGetLastError();
}

cudaError_t launch_b_nclassify(cudaStream_t s, int num_sms, long long R, const PairDesc* d,
                               const int32_t* row_pair, const int64_t* rowptr, const long long* flop,
                               const BBinTable& tab, int32_t vec_min_len, uint8_t* bin, int* status) {
  if (R <= 0) return cudaSuccess;
  long long g = (R + 255) / 256;
  if (g > num_sms * 8) g = num_sms * 8;
  k_b_nclassify<<<(unsigned)g, 256, 0, s>>>(R, d, row_pair, rowptr, flop, tab, vec_min_len, bin, status);
  return cudaGetLastError();
}

cudaError_t launch_b_symbolic(const LaunchCtx& ctx, const PairDesc* d, const int32_t* row_pair,
                              const int32_t* rows, const int32_t* bin_start, int32_t* tile_prefix,
                              const BBinTable& tab, int* queue, int32_t* cnt) {
  cudaError_t e = cudaFuncSetAttribute(k_b_symbolic, cudaFuncAttributeMaxDynamicSharedMemorySize, kBSmem);
  if (e != cudaSuccess) return e;
  k_b_tileprefix<<<1, 32, 0, ctx.stream>>>(tab, bin_start, tile_prefix);
  cudaMemsetAsync(queue, 0, sizeof(int), ctx.stream);
  timer_begin(ctx.timer, ctx.stream, "batched_symbolic");
  k_b_symbolic<<<persist_grid(ctx.num_sms), kBBlock, kBSmem, ctx.stream>>>(
      d, row_pair, rows, bin_start, tile_prefix, tab, queue, cnt, ctx.status);
  timer_end(ctx.timer, ctx.stream);
  return cudaGetLastError();
}

cudaError_t launch_b_numeric(const LaunchCtx& ctx, int32_t count, PairDesc* d, const int32_t* row_pair,
                             const int32_t* rows, const int32_t* bin_start, int32_t* tile_prefix,
                             const BBinTable& tab, int* queue, int32_t arith, float2* split,
                             const int64_t* rowptr, int32_t* ccol, double* cval) {
  cudaError_t e = cudaFuncSetAttribute(k_b_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize, kBSmem);
  if (e != cudaSuccess) return e;
  if (arith == kArithDF32 && count > 0) {
    const int g = count < ctx.num_sms * 8 ? count : ctx.num_sms * 8;
    timer_begin(ctx.timer, ctx.stream, "batched_split");
    k_b_split<<<g, 256, 0, ctx.stream>>>(count, d, split);
    timer_end(ctx.timer, ctx.stream);
  }
  k_b_tileprefix<<<1, 32, 0, ctx.stream>>>(tab, bin_start, tile_prefix);
  cudaMemsetAsync(queue, 0, sizeof(int), ctx.stream);
  timer_begin(ctx.timer, ctx.stream, "batched_numeric");
  k_b_numeric<<<persist_grid(ctx.num_sms), kBBlock, kBSmem, ctx.stream>>>(
      d, row_pair, rows, bin_start, tile_prefix, tab, queue, arith, split, rowptr, ccol, cval, ctx.status);
  timer_end(ctx.timer, ctx.stream);
  return cudaGetLastError();
}

cudaError_t launch_b_offsets(cudaStream_t s, int32_t count, const PairDesc* d, long long R,
                             const int64_t* rowptr, int64_t* off) {
  k_b_offsets<<<(count + 256) / 256, 256, 0, s>>>(count, d, R, rowptr, off);
  return cudaGetLastError();
}

}  // namespace kk

// --------------------------------------------------------------------------
// Packed batch: the pairs as one block-diagonal product
// --------------------------------------------------------------------------
namespace kk {
namespace {

// One CTA per pair: A_k's rows go to packed rows [R_k, R_k + A_k.m) with
// columns shifted to B_k's packed rows; B_k's rows go to [RB_k, RB_k + B_k.m)
// with their columns unchanged (C_k's columns stay local to the pair).
// vals_only: copy values only (numeric calls on the same structure).
__global__ void k_b_pack(int32_t count, const PairDesc* __restrict__ d,
                         const long long* __restrict__ base, int32_t vals_only, int32_t* pa_rp,
                         int32_t* pa_ci, double* pa_v, int32_t* pb_rp, int32_t* pb_ci, double* pb_v,
                         long long RA, long long NA, long long RB, long long NB) {
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const CsrView A = d[k].A, B = d[k].B;
    // base[4k ..]: A rows, A entries, B rows, B entries before pair k
    const long long ra = base[4 * k], na = base[4 * k + 1], rb = base[4 * k + 2], nb = base[4 * k + 3];
    if (!vals_only) {
      for (int r = threadIdx.x; r < A.m; r += blockDim.x) pa_rp[ra + r] = (int32_t)(na + A.rowptr[r]);
      for (int q = threadIdx.x; q < A.nnz; q += blockDim.x) pa_ci[na + q] = (int32_t)(rb + A.colind[q]);
      for (int r = threadIdx.x; r < B.m; r += blockDim.x) pb_rp[rb + r] = (int32_t)(nb + B.rowptr[r]);
      for (int q = threadIdx.x; q < B.nnz; q += blockDim.x) pb_ci[nb + q] = B.colind[q];
    }
    for (int q = threadIdx.x; q < A.nnz; q += blockDim.x) pa_v[na + q] = A.vals ? A.vals[q] : 0.0;
    for (int q = threadIdx.x; q < B.nnz; q += blockDim.x) pb_v[nb + q] = B.vals ? B.vals[q] : 0.0;
  }
  if (!vals_only && blockIdx.x == 0 && threadIdx.x == 0) {
    pa_rp[RA] = (int32_t)NA;
    pb_rp[RB] = (int32_t)NB;
  }
}

}  // namespace

cudaError_t launch_b_pack(cudaStream_t s, int num_sms, int32_t count, const PairDesc* d,
                          const long long* base, bool vals_only, int32_t* pa_rp, int32_t* pa_ci,
                          double* pa_v, int32_t* pb_rp, int32_t* pb_ci, double* pb_v, long long RA,
                          long long NA, long long RB, long long NB) {
  if (count <= 0) return cudaSuccess;
  const int grid = count < num_sms * 8 ? count : num_sms * 8;
  k_b_pack<<<grid, 256, 0, s>>>(count, d, base, vals_only ? 1 : 0, pa_rp, pa_ci, pa_v, pb_rp, pb_ci,
                                pb_v, RA, NA, RB, NB);
  return cudaGetLastError();
}

}  // namespace kk
