// Numeric phase of the window rows whose structure the symbolic phase kept
// (the paper's symbolic/numeric split, Sec. "SpGEMM: Sparse Matrix Matrix
// Multiply": the numeric phase of a reused structure computes values only).
#include "kk_internal.h"
#include "kk_kept.cuh"

namespace kk {
namespace {

using u64 = unsigned long long;
constexpr unsigned kFull = 0xffffffffu;
constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Numeric phase of the rows whose structure the symbolic phase kept: the
// row's words go into a small open-addressing table (slot = word mod 256,
// linear probing; at most kCacheWords words in 256 slots) instead of a W-bit
// window, so a warp needs about 4.6 KB of shared memory whatever the row's
// span and more rows are in flight per SM.  Words less than 256 apart never
// share a slot; a row whose words did collide takes the probing variant of the
// value pass.  An entry packs the word's bits (low 32), its prefix count (bits
// 32..47) and the word index (48..63).  Rows without kept structure are
// appended to `left` for k_num_window.
constexpr int kKeptWarps = 8;
struct KeptGeom {
  // table u64[kKeptSlots] | vacc u64[kWindowMaxNnz + 2] | ainfo int4[32]
  static constexpr size_t kValOff = (size_t)kKeptSlots * 8;
  static constexpr size_t kInfoOff = al16(kValOff + (size_t)(kWindowMaxNnz + 2) * 8);
  static constexpr size_t kWarpBytes = kInfoOff + 32 * 16;
};

// CHECK = false: the index arrays were verified against the symbolic call by
// their fingerprints fp[0] (symbolic) and fp[1] (this call), so products are
// not checked one by one against the kept structure.
template <bool CHECK, bool JAC>
__global__ void __launch_bounds__(kKeptWarps * 32, 6)
k_num_kept(CsrView A, CsrView B, WinCacheView cache, const int32_t* __restrict__ row_lo,
           const float2* __restrict__ bspl, const int32_t* __restrict__ b_range_bad, int32_t arith,
           const int64_t* __restrict__ c_rowptr, const int32_t* __restrict__ rows, int32_t nrows,
           int32_t* __restrict__ c_colind, double* __restrict__ c_vals, int* status,
           int32_t* __restrict__ left_rows, int32_t* __restrict__ left_count,
           const unsigned long long* __restrict__ fp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * KeptGeom::kWarpBytes;
  u64* table = reinterpret_cast<u64*>(base);
  u64* vacc = reinterpret_cast<u64*>(base + KeptGeom::kValOff);
  int4* ainfo = reinterpret_cast<int4*>(base + KeptGeom::kInfoOff);
  const bool df_all = arith == kArithDF32 && *b_range_bad == 0;
  if (!CHECK && blockIdx.x == 0 && threadIdx.x == 0 && fp[0] != fp[1])
    set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  for (int s = lane; s < kKeptSlots; s += 32) table[s] = kKeptEmpty;
  __syncwarp();
  const int nw = gridDim.x * kKeptWarps;  // rows dealt round-robin over the grid
  for (int r = blockIdx.x * kKeptWarps + warp; r < nrows; r += nw) {
    const int i = rows[r];
    const int L = cache.n[i];
    if (L < 0 || L > kCacheWords) {
      if (lane == 0) left_rows[atomicAdd(left_count, 1)] = i;
      continue;
    }
    const int lo_c = (row_lo[i] >> 5) * 32;
    const int64_t off = c_rowptr[i];
    const int cnt = (int)(c_rowptr[i + 1] - off);
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    for (int e = lane; e < cnt && e < kWindowMaxNnz; e += 32) vacc[e] = 0ull;
    __syncwarp();
    int run = 0, bad = 0, probe = 0;
    uint32_t slot0 = kKeptSlots, slot1 = kKeptSlots;  // slots this lane filled
    for (int e0 = 0; e0 < L; e0 += 32) {
      const int e = e0 + lane;
      uint32_t w = 0u, m = 0u;
      if (e < L) {
        w = cache.w[(size_t)i * kCacheWords + e];
        m = cache.m[(size_t)i * kCacheWords + e];
      }
      const int c = __popc(m);
      const int incl = team_inclusive_scan<32>(c, lane, kFull);
      int pos = run + incl - c;
      run += __shfl_sync(kFull, incl, 31);
      if (e < L) {
        const u64 entry = (u64)m | ((u64)(uint32_t)pos << 32) | ((u64)w << 48);
        uint32_t s = w & (kKeptSlots - 1);
        bool placed = false;
        for (int k = 0; k < kKeptSlots && !placed; ++k) {
          placed = atomicCAS(&table[s], kKeptEmpty, entry) == kKeptEmpty;
          if (placed) {
            if (e0 == 0) slot0 = s;
            else slot1 = s;
          } else {
            probe = 1;
            s = (s + 1) & (kKeptSlots - 1);
          }
        }
        if (!placed) bad = 1;
        while (m) {
          const int b = __ffs(m) - 1;
          m &= m - 1;
          if (pos < cnt) c_colind[off + pos] = lo_c + (int)w * 32 + b;
          ++pos;
        }
      }
    }
    if (bad || (run != cnt && lane == 0)) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    probe = __any_sync(kFull, probe);
    __syncwarp();
    // arithmetic of this row: DF32 unless a value of the row is outside its window
    int missing = 0;
    const bool df =
        probe ? kept_values<true, CHECK, JAC>(pa, pe, df_all, A, i, B.rowptr, ainfo, lo_c, table,
                                         vacc, B.colind, bspl, B.vals, lane, missing)
              : kept_values<false, CHECK, JAC>(pa, pe, df_all, A, i, B.rowptr, ainfo, lo_c,
                                          table, vacc, B.colind, bspl, B.vals, lane, missing);
    if (missing) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    const int n = min(cnt, kWindowMaxNnz);
    for (int e = lane; e < n; e += 32) {
      const u64 v = vacc[e];
      c_vals[off + e] = df ? df_to_double(df_unpack(v)) : __longlong_as_double((long long)v);
    }
    // empty the slots this row filled for the next row
    if (slot0 < kKeptSlots) table[slot0] = kKeptEmpty;
    if (slot1 < kKeptSlots) table[slot1] = kKeptEmpty;
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_num_kept(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                            const WinCacheView& cache, const float2* b_split, const int32_t* b_range_bad,
                            int32_t arith, const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                            int32_t* c_colind, double* c_vals, int32_t* left_rows, int32_t* left_count) {
  const size_t smem = (size_t)kKeptWarps * KeptGeom::kWarpBytes;
  const bool check = ctx.fingerprint == nullptr;
  const bool jac = A.jac_s != nullptr;
  auto kern = check ? (jac ? k_num_kept<true, true> : k_num_kept<true, false>)
                    : (jac ? k_num_kept<false, true> : k_num_kept<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // one resident wave: the rows in flight form one contiguous band, so the B
  // rows they share stay in L2 (a grid of several waves runs bands far apart)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kKeptWarps * 32, smem) != cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    per_sm = 1;
  }
  long long blocks = (nrows + kKeptWarps - 1) / kKeptWarps;
  const long long capb = (long long)ctx.num_sms * per_sm;
  if (blocks > capb) blocks = capb;
  if (blocks < 1) blocks = 1;
  kern<<<(int)blocks, kKeptWarps * 32, smem, ctx.stream>>>(
      A, B, cache, ctx.row_lo, b_split, b_range_bad, arith, c_rowptr, rows, nrows, c_colind, c_vals,
      ctx.status, left_rows, left_count, ctx.fingerprint);
  return cudaGetLastError();
}


}  // namespace kk
