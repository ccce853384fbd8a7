// C ABI and host orchestration of the two-phase SpGEMM (Kokkos Kernels paper,
// Sec. "Standard SpGEMM Kernel"): allocate C's row pointers, symbolic phase,
// nnz(C) to the host, then the numeric phase into caller-allocated arrays.
//
// Symbolic call sequence on the handle's stream:
//   analyze B (strictly ascending rows?, column range)  ->  analyze A (per-row
//   flop bound sum_{j in A(i,:)} nnz(B(j,:)), column range, bin id)  ->  stable
//   binning of rows  ->  [sync: bin sizes]  ->  one symbolic kernel per non-empty
//   bin  ->  exclusive scan of the counts into C's int64 row pointers, fused with
//   the numeric bin id (from nnz(C(i,:)))  ->  stable binning  ->  [sync: nnz(C),
//   bin sizes].
// Numeric call sequence: split B's values into DF32 pairs (range-checked), one
// numeric kernel per non-empty bin.  No host synchronisation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kk_internal.h"
#include "kk_device.cuh"
#include "kk_batched.h"
#include "kk_learned.h"
#include "kk_jacobi.h"
#include "kk_spadd.h"

namespace kk {

// ---------------------------------------------------------------------------
// Kernel timer
// ---------------------------------------------------------------------------
struct KernelTimer {
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<const char*> names;
  std::vector<double> total_ms;
  std::vector<long long> launches;
  cudaEvent_t take() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void collect() {
    for (auto& r : pending) {
      cudaEventSynchronize(r.b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      size_t k = 0;
      for (; k < names.size(); ++k)
        if (std::strcmp(names[k], r.name) == 0) break;
      if (k == names.size()) {
        names.push_back(r.name);
        total_ms.push_back(0.0);
        launches.push_back(0);
      }
      total_ms[k] += ms;
      launches[k] += 1;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  ~KernelTimer() {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

void timer_begin(KernelTimer* t, cudaStream_t s, const char* name) {
  if (!t) return;
  KernelTimer::Rec r{name, t->take(), t->take()};
  cudaEventRecord(r.a, s);
  t->pending.push_back(r);
}

void timer_end(KernelTimer* t, cudaStream_t s) {
  if (!t || t->pending.empty()) return;
  cudaEventRecord(t->pending.back().b, s);
}

namespace {

// ---------------------------------------------------------------------------
// Grow-only device buffer
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t need) {
    if (need <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t b = need < 256 ? 256 : need;
    b += b / 4;  // slack for growth
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = b;
    return cudaSuccess;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

constexpr int kMaxBins = 32;
constexpr uint8_t kSkipBin = 0xFF;

// Device-side classifier: first bin whose hi bound covers q and whose mode
// (0 = vector only, 1 = flattened only, 2 = either) admits the row's mode.
// Window bins (window tier) are tried first: a row qualifies for window class
// w when B's rows are sorted, its span fits kWindowBits[w], the window is not
// too wide for its flop count, and (numeric) its nnz fits the dense value slots.
struct BinTable {
  int32_t nb;
  long long hi[kMaxBins];
  int32_t mode[kMaxBins];  // 0 vector, 1 flattened, 2 either, 3 thread tier (flop capped too)
  long long thread_flop;
  int32_t nwin;
  int32_t win_bits[kMaxWindowBins];
  int32_t win_bin[kMaxWindowBins];
  long long win_q[kMaxWindowBins];      // largest binning quantity of each window bin
  long long win_qlo[kMaxWindowBins];    // binning quantity must exceed this
  long long win_ratio[kMaxWindowBins];  // window W only when W <= ratio * flop
};

__device__ __forceinline__ uint8_t classify(const BinTable& t, long long q, int flat, int span,
                                            long long flop, int sorted) {
  if (q <= 0) return kSkipBin;
  if (sorted && span > 0) {
    for (int w = 0; w < t.nwin; ++w)
      if (q > t.win_qlo[w] && q <= t.win_q[w] && span <= t.win_bits[w] &&
          (long long)t.win_bits[w] <= t.win_ratio[w] * flop)
        return (uint8_t)t.win_bin[w];
  }
  for (int b = 0; b < t.nb; ++b) {
    if (t.mode[b] == 3) {
      if (q <= t.hi[b] && flop <= t.thread_flop) return (uint8_t)b;
      continue;
    }
    if (q <= t.hi[b] && (t.mode[b] == 2 || t.mode[b] == flat)) return (uint8_t)b;
  }
  return (uint8_t)(t.nb - 1);
}

// ---------------------------------------------------------------------------
// Analysis kernels
// ---------------------------------------------------------------------------
// A rows: flop bound, column range, symbolic bin id; optional total flops.
// One team of T lanes per row.  The kernel is bound by its dependent gathers
// (A column -> B row bounds -> B's first and last column), so each lane issues
// those of U entries together and the next row's bounds are loaded while a row
// is processed; T and U follow A's mean row length.  STATS (the learned
// form): also the longest and shortest referenced B row of each row, to stat.
template <int T, int U, bool STATS>
__global__ void __launch_bounds__(256, 6)
k_analyze_a(CsrView A, const int32_t* __restrict__ brp,
                            const int32_t* __restrict__ bcol, int32_t nb_rows,
                            const int32_t* __restrict__ b_sorted, BinTable tab,
                            int32_t vec_min_len, long long* __restrict__ flop,
                            uint8_t* __restrict__ bin, int32_t* __restrict__ row_lo,
                            int32_t* __restrict__ row_span, int2* __restrict__ stat,
                            unsigned long long* total_flop, int* status) {
  const int sorted = *b_sorted;
  const int tl = threadIdx.x % T;
  const unsigned mask = team_mask<T>();
  const long long team0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / T;
  const long long nteams = (long long)gridDim.x * blockDim.x / T;
  const long long iters = (A.m + nteams - 1) / nteams;
  unsigned long long acc = 0;
  long long r = team0;
  int pa_n = 0, pe_n = 0;
  if (r < A.m) {
    pa_n = A.rowptr[r];
    pe_n = A.rowptr[r + 1];
  }
  for (long long it = 0; it < iters; ++it, r += nteams) {
    int pa = pa_n, pe = pe_n;
    if (r + nteams < A.m) {
      pa_n = A.rowptr[r + nteams];
      pe_n = A.rowptr[r + nteams + 1];
    }
    long long f = 0;
    int bad = 0;
    int lo = 0x7fffffff, hi = -1;
    int mx = 0, mn = 0x7fffffff;
    if (r < A.m) {
      if (pa < 0 || pe < pa || pe > A.nnz || (r == 0 && pa != 0)) {
        bad = 1;
        pe = pa;
      }
      for (int p0 = pa; p0 < pe; p0 += T * U) {
        int j[U], bs[U], be[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int p = p0 + u * T + tl;
          j[u] = p < pe ? A.colind[p] : -1;
          if (p < pe && (unsigned)j[u] >= (unsigned)nb_rows) {
            bad = 1;
            j[u] = -1;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          bs[u] = 0;
          be[u] = 0;
          if (j[u] >= 0) {
            bs[u] = brp[j[u]];
            be[u] = brp[j[u] + 1];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          f += be[u] - bs[u];
          if (STATS && j[u] >= 0) {
            mx = max(mx, be[u] - bs[u]);
            mn = min(mn, be[u] - bs[u]);
          }
          if (sorted && be[u] > bs[u]) {
            lo = min(lo, bcol[bs[u]]);
            hi = max(hi, bcol[be[u] - 1]);
          }
        }
      }
    }
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) {
      f += __shfl_xor_sync(mask, f, o, T);
      lo = min(lo, __shfl_xor_sync(mask, lo, o, T));
      hi = max(hi, __shfl_xor_sync(mask, hi, o, T));
      if (STATS) {
        mx = max(mx, __shfl_xor_sync(mask, mx, o, T));
        mn = min(mn, __shfl_xor_sync(mask, mn, o, T));
      }
    }
    if (bad) set_status(status, KK_ERR_BAD_INDEX);
    if (r < A.m && tl == 0) {
      flop[r] = f;
      const long long span = hi >= lo ? (long long)hi - lo + 1 : 0;
      const int sp = span > 0x7fffffff ? 0x7fffffff : (int)span;
      row_lo[r] = hi >= lo ? lo : 0;
      row_span[r] = sp;
      const int flat = (f < (long long)vec_min_len * (pe - pa)) ? 1 : 0;
      bin[r] = classify(tab, f, flat, sp, f, sorted);
      if (STATS) stat[r] = make_int2(mx, pe > pa ? mn : 0);
      acc += (unsigned long long)f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total_flop, acc);
}

// ---------------------------------------------------------------------------
// Stable binning: rows grouped by bin id, ascending row order within a bin.
// ---------------------------------------------------------------------------
constexpr int kBinBlock = 256;
constexpr int kBinPerThread = 8;
constexpr int kBinRows = kBinBlock * kBinPerThread;
constexpr int kBinScanPer = 8;  // counts per thread in the bin-offset scan

__global__ void __launch_bounds__(kBinBlock)
k_bin_count(int32_t m, const uint8_t* __restrict__ bin, int32_t nb, int32_t nblk,
            int32_t* __restrict__ blk_counts) {
  __shared__ int c[kMaxBins];
  if (threadIdx.x < kMaxBins) c[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kBinRows;
  for (int t = 0; t < kBinPerThread; ++t) {
    const long long r = base + t * kBinBlock + threadIdx.x;
    if (r < m) {
      const uint8_t b = bin[r];
      if (b != kSkipBin) atomicAdd(&c[b], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x < nb) blk_counts[(long long)threadIdx.x * nblk + blockIdx.x] = c[threadIdx.x];
}

// Single CTA: exclusive scan (bin-major) of the per-block counts in place;
// bin_start[b] = first position of bin b, bin_start[nb] = total.
__global__ void __launch_bounds__(1024)
k_bin_scan(int32_t nb, int32_t nblk, int32_t* __restrict__ blk, int32_t* __restrict__ bin_start) {
  // every thread scans kBinScanPer consecutive counts, so one pass of the
  // 1024-thread block covers 8,192 (bin, block) counts (few barriers)
  constexpr int P = kBinScanPer;
  __shared__ int warp_tot[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const long long total = (long long)nb * nblk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long c0 = 0; c0 < total; c0 += (long long)blockDim.x * P) {
    const long long i0 = c0 + (long long)threadIdx.x * P;
    int v[P];
    int sum = 0;
#pragma unroll
    for (int t = 0; t < P; ++t) {
      v[t] = i0 + t < total ? blk[i0 + t] : 0;
      sum += v[t];
    }
    const int incl = team_inclusive_scan<32>(sum, lane, 0xffffffffu);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int w = warp_tot[lane];
      const int wi = team_inclusive_scan<32>(w, lane, 0xffffffffu);
      warp_tot[lane] = wi - w;
    }
    __syncthreads();
    int run = carry + warp_tot[warp] + incl - sum;
#pragma unroll
    for (int t = 0; t < P; ++t) {
      const long long idx = i0 + t;
      if (idx < total) {
        blk[idx] = run;
        if (idx % nblk == 0) bin_start[idx / nblk] = run;
      }
      run += v[t];
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = run;
    __syncthreads();
  }
  if (threadIdx.x == 0) bin_start[nb] = carry;
}

__global__ void __launch_bounds__(kBinBlock)
k_bin_scatter(int32_t m, const uint8_t* __restrict__ bin, int32_t nb, int32_t nblk,
              const int32_t* __restrict__ blk_off, int32_t* __restrict__ rows_out) {
  constexpr int NW = kBinBlock / 32;
  __shared__ int wcount[NW][kMaxBins];
  __shared__ int running[kMaxBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < NW * kMaxBins; t += blockDim.x) (&wcount[0][0])[t] = 0;
  if (threadIdx.x < nb) running[threadIdx.x] = blk_off[(long long)threadIdx.x * nblk + blockIdx.x];
  __syncthreads();
  const long long base = (long long)blockIdx.x * kBinRows;
  const unsigned lt = (1u << lane) - 1u;
  for (int t = 0; t < kBinPerThread; ++t) {
    const long long r = base + t * kBinBlock + threadIdx.x;
    const int b = r < m ? (int)bin[r] : (int)kSkipBin;
    const unsigned same = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(same & lt);
    if (b != kSkipBin && rank == 0) wcount[warp][b] = __popc(same);
    __syncthreads();
    if (b != kSkipBin) {
      int pre = running[b];
      for (int w = 0; w < warp; ++w) pre += wcount[w][b];
      rows_out[pre + rank] = (int32_t)r;
    }
    __syncthreads();
    if (threadIdx.x < nb) {
      int s = 0;
      for (int w = 0; w < NW; ++w) s += wcount[w][threadIdx.x];
      running[threadIdx.x] += s;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NW * kMaxBins; q += blockDim.x) (&wcount[0][0])[q] = 0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Scan of row counts into int64 row pointers, fused with numeric bin ids.
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 256;
constexpr int kScanPer = 8;
constexpr int kScanRows = kScanBlock * kScanPer;

__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long* scratch,
                                                        long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < nw ? scratch[lane] : 0;
    long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < nw) scratch[lane] = wi - w;
    if (lane == 31) scratch[32] = wi;
  }
  __syncthreads();
  const long long r = scratch[warp] + incl - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanBlock)
k_scan_partial(int32_t m, const int32_t* __restrict__ cnt, long long* __restrict__ blk_sum) {
  __shared__ long long scratch[33];
  const long long base = (long long)blockIdx.x * kScanRows + (long long)threadIdx.x * kScanPer;
  long long s = 0;
  for (int t = 0; t < kScanPer; ++t)
    if (base + t < m) s += cnt[base + t];
  long long tot;
  block_excl_scan_ll(s, scratch, &tot);
  if (threadIdx.x == 0) blk_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024)
k_scan_top(int32_t nblk, long long* __restrict__ blk_sum, long long* __restrict__ grand) {
  __shared__ long long scratch[33];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nblk; c0 += blockDim.x) {
    const int idx = c0 + threadIdx.x;
    const long long v = idx < nblk ? blk_sum[idx] : 0;
    long long tot;
    const long long ex = block_excl_scan_ll(v, scratch, &tot);
    if (idx < nblk) blk_sum[idx] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void __launch_bounds__(kScanBlock)
k_scan_final(int32_t m, const int32_t* __restrict__ cnt, const long long* __restrict__ blk_off,
             const long long* __restrict__ flop, const int32_t* __restrict__ arp,
             const int32_t* __restrict__ row_span, const int32_t* __restrict__ b_sorted,
             int32_t vec_min_len, BinTable ntab, int64_t* __restrict__ rowptr,
             uint8_t* __restrict__ nbin) {
  const int sorted = *b_sorted;
  __shared__ long long scratch[33];
  const long long base = (long long)blockIdx.x * kScanRows + (long long)threadIdx.x * kScanPer;
  int v[kScanPer];
  long long s = 0;
  for (int t = 0; t < kScanPer; ++t) {
    v[t] = base + t < m ? cnt[base + t] : 0;
    s += v[t];
  }
  long long tot;
  long long run = blk_off[blockIdx.x] + block_excl_scan_ll(s, scratch, &tot);
  for (int t = 0; t < kScanPer; ++t) {
    const long long r = base + t;
    if (r < m) {
      rowptr[r] = run;
      if (nbin) {
        const int nza = arp[r + 1] - arp[r];
        const int flat = (flop[r] < (long long)vec_min_len * nza) ? 1 : 0;
        nbin[r] = classify(ntab, v[t], flat, row_span[r], flop[r], sorted);
      }
      if (r == m - 1) rowptr[m] = run + v[t];
    }
    run += v[t];
  }
}

// Symbolic bin of every row from its flop bound and span (learned form: the
// rows left to the plain path are picked from these afterwards).
// Per numeric tier: C entries and A entries of the rows binned to it (for the
// per-kernel roofline accounting).
struct TierOfBin {
  int32_t nb;
  int8_t tier[kMaxBins];
};

__global__ void k_tier_sums(int32_t m, const uint8_t* __restrict__ nbin, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ arp, const long long* __restrict__ flop, TierOfBin tb,
                            unsigned long long* tier_c, unsigned long long* tier_a,
                            unsigned long long* tier_f) {
  unsigned long long c[4] = {0, 0, 0, 0}, a[4] = {0, 0, 0, 0}, f[4] = {0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const uint8_t b = nbin[i];
    if (b == kSkipBin || b >= tb.nb) continue;
    const int t = tb.tier[b];
    c[t] += (unsigned long long)(rowptr[i + 1] - rowptr[i]);
    a[t] += (unsigned long long)(arp[i + 1] - arp[i]);
    f[t] += (unsigned long long)flop[i];
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c[t] += __shfl_xor_sync(0xffffffffu, c[t], o);
      a[t] += __shfl_xor_sync(0xffffffffu, a[t], o);
      f[t] += __shfl_xor_sync(0xffffffffu, f[t], o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (c[t]) atomicAdd(&tier_c[t], c[t]);
      if (a[t]) atomicAdd(&tier_a[t], a[t]);
      if (f[t]) atomicAdd(&tier_f[t], f[t]);
    }
  }
}

TierOfBin tier_of_bins(const std::vector<BinSpec>& bins) {
  TierOfBin t{};
  t.nb = (int32_t)bins.size();
  for (size_t b = 0; b < bins.size() && b < (size_t)kMaxBins; ++b) t.tier[b] = (int8_t)stat_tier(bins[b].tier);
  return t;
}

// ---------------------------------------------------------------------------
// Structure fingerprint: a 64-bit sum over the elements of the index arrays
// (A's and B's row pointers and columns) of a term of (value, position, array),
// order-independent so blocks add their parts atomically.  The symbolic call
// that keeps window structure records it; a numeric call that uses that
// structure recomputes it, and a difference (index arrays changed in place
// behind the same pointers) is reported as a structure mismatch.
// ---------------------------------------------------------------------------
struct FpArrays {
  const int32_t* p[4];
  long long n[4];
};

// The term of element x at position i of array a: x XORed with a value of
// (i, a), times an odd constant.  For a fixed position it is a bijection of x,
// and the terms are summed as 32-bit values into 64 bits (no wrap below 2^32
// elements), so changing any one element always changes the sum; three
// integer operations per element keep the pass at memory speed.
__device__ __forceinline__ unsigned long long fp_mix(uint32_t x, uint32_t i, uint32_t a) {
  return (unsigned long long)((x ^ (i * 0x9E3779B1u + a * 0x7F4A7C15u)) * 0x85EBCA6Bu);
}

// blockIdx.y = the array.  The aligned middle of the array is read as int4 with
// kFpUnroll loads in flight per thread (the pass is bound by HBM latency and
// bandwidth); block 0 takes the few elements before the first and after the
// last 16-byte boundary.  One atomic per block.
constexpr int kFpUnroll = 4;
constexpr int kFpThreads = 256;
__global__ void __launch_bounds__(kFpThreads) k_fingerprint(FpArrays arr, unsigned long long* out) {
  const int a = blockIdx.y;
  // selects instead of indexing the parameter arrays (which would go through
  // local memory)
  const int32_t* __restrict__ x = a == 0 ? arr.p[0] : a == 1 ? arr.p[1] : a == 2 ? arr.p[2] : arr.p[3];
  const long long n = a == 0 ? arr.n[0] : a == 1 ? arr.n[1] : a == 2 ? arr.n[2] : arr.n[3];
  long long head = (long long)(((16u - (unsigned)((uintptr_t)x & 15u)) & 15u) / 4u);
  if (head > n) head = n;
  const long long nv = (n - head) / 4;
  const int4* __restrict__ xv = reinterpret_cast<const int4*>(x + head);
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  for (long long v0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; v0 < nv; v0 += kFpUnroll * stride) {
    int4 w[kFpUnroll];
#pragma unroll
    for (int u = 0; u < kFpUnroll; ++u)
      w[u] = v0 + u * stride < nv ? xv[v0 + u * stride] : make_int4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < kFpUnroll; ++u) {
      if (v0 + u * stride < nv) {
        const uint32_t i = (uint32_t)(head + (v0 + u * stride) * 4);
        acc += fp_mix((uint32_t)w[u].x, i, a) + fp_mix((uint32_t)w[u].y, i + 1, a) +
               fp_mix((uint32_t)w[u].z, i + 2, a) + fp_mix((uint32_t)w[u].w, i + 3, a);
      }
    }
  }
  if (blockIdx.x == 0) {
    for (long long q = threadIdx.x; q < head; q += blockDim.x) acc += fp_mix((uint32_t)x[q], (uint32_t)q, a);
    for (long long q = head + nv * 4 + threadIdx.x; q < n; q += blockDim.x)
      acc += fp_mix((uint32_t)x[q], (uint32_t)q, a);
  }
  __shared__ unsigned long long part[kFpThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < kFpThreads / 32; ++k) t += part[k];
    if (t) atomicAdd(out, t);
  }
}

// ---------------------------------------------------------------------------
// Jacobi-fused numeric phase: the values of A' with C = A' B = (I - omega D^-1 A) B,
// i.e. a'_ij = s_i a_ij and a'_ii = 1 + s_i a_ii at the row's first stored
// diagonal entry, s_i = -omega / D(i), D(i) = the sum of the row's stored
// diagonal entries.  One team of kJacTeam lanes per row.
// ---------------------------------------------------------------------------
// The row scaling of the Jacobi-fused product (paper Sec. "Jacobi-Fused SpGEMM
// Kernel", C = (I - omega D^-1 A) B): per row i, D(i) = the sum of the row's
// stored diagonal entries, s_i = -omega / D(i) and the position of the row's
// first diagonal entry.  The numeric kernels then take A(i,j) as s_i * a_ij,
// plus 1 at that entry (so B(i,:) is added once per row), as they load it: A
// is not rewritten.  The thread tier, whose rows are short, finds s_i itself;
// this kernel serves the rows of the other tiers, the rows[0..nrows) of one
// numeric bin.  T lanes per row, the column loads of U entries per lane in
// flight (a value is loaded only for a diagonal entry); the next row's bounds
// are loaded while a row is processed.  A row without a stored diagonal, or
// whose diagonal sums to 0, is reported (KK_ERR_INVALID_ARG).
template <int T, int U>
__global__ void __launch_bounds__(256) k_jacobi_rows(CsrView A, const int32_t* __restrict__ rows, int32_t nrows,
                                                     double omega, double* __restrict__ out_s,
                                                     int32_t* __restrict__ out_p, int* status) {
  const int tl = threadIdx.x % T;
  const unsigned mask = team_mask<T>();
  const long long team0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / T;
  const long long nteams = (long long)gridDim.x * blockDim.x / T;
  int bad = 0;
  long long t = team0;
  int pa_n = 0, pe_n = 0, r_n = 0;
  if (t < nrows) {
    r_n = rows[t];
    pa_n = A.rowptr[r_n];
    pe_n = A.rowptr[r_n + 1];
  }
  for (; t < nrows; t += nteams) {
    const int pa = pa_n, pe = pe_n, r = r_n;
    if (t + nteams < nrows) {
      r_n = rows[t + nteams];
      pa_n = A.rowptr[r_n];
      pe_n = A.rowptr[r_n + 1];
    }
    // the diagonal value is picked by selects; repeats of it are added on a
    // branch taken only when a row has them
    double d = 0.0, dx = 0.0;
    int first = 0x7fffffff, nd = 0;
    for (int p0 = pa; p0 < pe; p0 += T * U) {
      int c[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * T + tl;
        c[u] = p < pe ? A.colind[p] : -1;
      }
      const int nd0 = nd;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool on = c[u] == r;
        const double v = on ? A.vals[p0 + u * T + tl] : 0.0;
        d = (on && nd == 0) ? v : d;
        nd += on ? 1 : 0;
        first = on ? min(first, p0 + u * T + tl) : first;
      }
      if (nd - nd0 > (nd0 == 0 ? 1 : 0)) {
        // repeated diagonal entries: all but the lane's first one go to dx
        int k = nd0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (c[u] == r) {
            if (k > 0) dx += A.vals[p0 + u * T + tl];
            ++k;
          }
        }
      }
    }
    d += dx;
    if (T > 1) {
#pragma unroll
      for (int o = T / 2; o > 0; o >>= 1) {
        d += __shfl_xor_sync(mask, d, o, T);
        nd += __shfl_xor_sync(mask, nd, o, T);
        first = min(first, __shfl_xor_sync(mask, first, o, T));
      }
    }
    double sc = 0.0;
    int fp = -1;
    if (nd == 0 || (__double_as_longlong(d) << 1) == 0) {
      bad = 1;
    } else {
      sc = -omega * jacobi_recip(d);
      fp = first;
    }
    if (tl == 0) {
      out_s[r] = sc;
      out_p[r] = fp;
    }
  }
  if (bad) set_status(status, KK_ERR_INVALID_ARG);
}

// ---------------------------------------------------------------------------
// DF32 split of B's values, with the window check.
// ---------------------------------------------------------------------------
// HBM-bound: each thread keeps kSplitUnroll coalesced loads in flight.
constexpr int kSplitUnroll = 4;
__global__ void k_split_values(long long n, const double* __restrict__ v, float2* __restrict__ out,
                               int32_t* range_bad) {
  int bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; q0 < n;
       q0 += stride * kSplitUnroll) {
    double x[kSplitUnroll];
#pragma unroll
    for (int u = 0; u < kSplitUnroll; ++u) {
      const long long q = q0 + u * stride;
      x[u] = q < n ? v[q] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kSplitUnroll; ++u) {
      const long long q = q0 + u * stride;
      DF d;
      bad |= df_split(x[u], d) ? 0 : 1;
      if (q < n) out[q] = make_float2(d.hi, d.lo);
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  if (bad && (threadIdx.x & 31) == 0) atomicOr(range_bad, 1);
}

// One CTA copies n words from device memory to the page-locked staging buffer
// through its device mapping (the read-backs of the status block and bin starts).
__global__ void k_readback(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace
}  // namespace kk

using namespace kk;

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct kk_spgemm_handle_s {
  cudaStream_t stream = nullptr;
  kk_spgemm_options opt{};
  int device = 0;
  int num_sms = 0;
  int max_smem = 0;
  KernelTimer* timer = nullptr;
  std::string last_error;
  // scratch
  DevBuf d_misc;       // status int, sorted flag, range flag, total flop (u64), grand total (ll)
  DevBuf d_flop;       // long long[m]
  DevBuf d_sbin;       // uint8[m]
  DevBuf d_nbin;       // uint8[m]
  DevBuf d_srows;      // int32[m]
  DevBuf d_nrows;      // int32[m]
  DevBuf d_cnt;        // int32[m]
  DevBuf d_rowlo;      // int32[m]  first column of each row's span
  DevBuf d_span;       // int32[m]  span width (0 for rows without products)
  DevBuf d_blk;        // int32[kMaxBins * nblk]
  DevBuf d_binstart;   // int32[2 * (kMaxBins + 1)]
  DevBuf d_scan;       // long long[nblk]
  DevBuf d_bsplit;     // float2[nnzB]
  DevBuf d_jvals;      // float64[m]: row scales s_i of the Jacobi-fused numeric phase
  DevBuf d_jpos;       // int32[m]: position of each row's first diagonal entry (Jacobi)
  DevBuf d_apos, d_bpos;  // SpAdd: slot in C's row of every entry of A and of B (int32)
  DevBuf d_acnt;          // SpAdd: nnz(C(i,:)) (int32[m])
  DevBuf d_along;         // SpAdd: [0] long-row count, [1..] long rows (int32[m + 1])
  // learned form
  DevBuf d_params;     // float[KK_MLP_NUM_PARAMS]
  bool have_pred = false;
  float quantile = 0.95f;
  DevBuf d_lbin;       // uint8[m]  learned bin (one-pass class / heavy / none)
  DevBuf d_plain;      // uint8[m]  1 = row takes the plain path
  DevBuf d_cap;        // int32[m]  staging capacity
  DevBuf d_lstat;      // int2[m]   learned form: longest / shortest referenced B row
  DevBuf d_soff;       // int64[m+1] staging offsets
  DevBuf d_scol;       // int32[staging]
  DevBuf d_sval;       // double[staging]
  DevBuf d_sball;      // uint8[m]  symbolic bins of all rows
  DevBuf d_nbin2;      // uint8[m]  numeric bins of plain-path rows
  DevBuf d_lrows;      // int32[m]  learned bins' row lists
  DevBuf d_lrows2;     // int32[m]  plain-path numeric bins' row lists
  DevBuf d_mm;         // int2[n]   B row min/max columns (features)
  bool learned_valid = false;
  bool p_learned = false;  // the packed batch ran the learned form; its numeric call is due
  // SpAdd: the arrays, sizes and result of the last symbolic call
  bool add_valid = false;
  const void* add_key[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t add_m = 0, add_n = 0, add_nnza = 0, add_nnzb = 0;
  int64_t add_nnzc = 0;
  std::vector<int32_t> lnum_start;
  // batched form
  DevBuf d_bdesc, d_rowpair, d_bflop, d_bsbin, d_bnbin, d_bsrows, d_bnrows, d_bcnt, d_btiles, d_bstart,
      d_bqueue, d_bsplit2, d_boff;
  void* h_bdesc = nullptr;   // pinned PairDesc[count] (symbolic upload)
  void* h_bdesc2 = nullptr;  // pinned PairDesc[count] (numeric upload, device flags included)
  void* h_boff = nullptr;    // pinned int64[count + 1]
  size_t h_bcap = 0;         // pairs the pinned buffers hold
  int32_t b_count = 0;
  long long b_R = 0, b_total = 0, b_nnzb = 0;
  bool b_valid = false;
  BBinTable b_sym{}, b_num{};
  cudaGraphExec_t g_sym = nullptr, g_num = nullptr;
  unsigned long long g_sym_key = 0, g_num_key = 0;
  void* h_pinned = nullptr;  // host staging for readbacks
  void* d_pinned_map = nullptr;  // its device mapping (null: none)
  // symbolic state
  bool have_symbolic = false;
  bool small = false;  // the last symbolic call took the small-product path (kk_small.cu)
  int32_t am = 0, an = 0, bn = 0, annz = 0, bnnz = 0;
  int64_t nnz_c = 0;
  int32_t b_sorted = 1;
  std::vector<BinSpec> sym_bins, num_bins;
  std::vector<int32_t> num_start;  // nb + 1
  int64_t stats[32] = {0};
  int32_t last_arith = kArithDF32;
  // compressed B (window tier) and the arrays it was built from
  DevBuf d_bc;         // int2[nnzB + 2] (the padding lets 16-byte loads of pairs end past the last row)
  DevBuf d_bclen;      // int32[B.m]
  bool bc_valid = false;
  const void* bc_key[2] = {nullptr, nullptr};
  int32_t bc_m = 0, bc_nnz = 0;
  // structure kept by the symbolic window kernel, and the arrays it is for
  DevBuf d_cw;         // uint16[m * kCacheWords]
  DevBuf d_cm;         // uint32[m * kCacheWords]
  DevBuf d_cn;         // int32[m]
  DevBuf d_left;       // int32[1 + m]: count, then rows left to the window kernel
  bool cache_valid = false;
  // wide-tier bit vectors kept by the symbolic phase
  DevBuf d_wbits, d_wslot, d_wnext;
  bool b_overflow = false;             // the persistent batched form handed a batch to the packed form
  unsigned long long b_overflow_key = 0;  // ... the batch's key (pairs, output pointer, count)
  bool keep_valid = false;
  const void* keep_key[4] = {nullptr, nullptr, nullptr, nullptr};
  WideKeep keep{nullptr, nullptr, nullptr, 0, 0};  // what the next launches use
  size_t dev_total = 0;
  // packed batch: block-diagonal A and B of the last batched symbolic call
  DevBuf d_pa_rp, d_pa_ci, d_pa_v, d_pb_rp, d_pb_ci, d_pb_v, d_pbase;
  long long p_RA = 0, p_NA = 0, p_RB = 0, p_NB = 0;
  int32_t p_kmax = 0;
  bool p_valid = false;
  const void* cache_key[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

struct Misc {
  int status;
  int32_t sorted;
  int32_t range_bad;
  int32_t pad;
  unsigned long long total_flop;
  long long grand;
  long long grand2;
  unsigned long long tier_c[4];  // numeric tiers: C entries of their rows
  unsigned long long tier_a[4];  // numeric tiers: A entries of their rows
  unsigned long long tier_f[4];  // numeric tiers: multiply-adds of their rows
  unsigned long long kept;       // window rows whose structure was kept
  unsigned long long bc_pairs;   // pairs of the compressed B
  unsigned long long fp[2];      // structure fingerprints: symbolic call, numeric call
  int32_t small_flags[4];        // small-product path: row beyond it, bad index, CTA ticket
};

kk_status fail(kk_spgemm_handle h, kk_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

kk_status cuda_fail(kk_spgemm_handle h, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(h, KK_ERR_OOM, std::string(where) + ": " + cudaGetErrorString(e));
  }
  return fail(h, KK_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define KK_CUDA(h, call, where)                       \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

#define KK_TRY(expr)                   \
  do {                                 \
    const kk_status kk_try_ = (expr);  \
    if (kk_try_ != KK_OK) return kk_try_; \
  } while (0)


// A small device-to-host read into the handle's page-locked staging buffer
// (the status block, bin starts), by a one-CTA kernel writing the buffer
// through its device mapping: no copy engine is involved, so the read does
// not wait behind a large transfer queued on one (another stream's download
// of C in a serving loop).  Without the mapping, cudaMemcpyAsync.  Enqueued on
// s; the caller synchronises before reading.
kk_status readback(kk_spgemm_handle h, void* host_dst, const void* dev_src, size_t bytes, cudaStream_t s) {
  const char* base = static_cast<const char*>(h->h_pinned);
  const char* dst = static_cast<const char*>(host_dst);
  if (h->d_pinned_map && dst >= base && dst + bytes <= base + 4096 && bytes % 4 == 0 &&
      ((uintptr_t)dev_src & 3) == 0 && ((uintptr_t)host_dst & 3) == 0) {
    uint32_t* dmap = reinterpret_cast<uint32_t*>(static_cast<char*>(h->d_pinned_map) + (dst - base));
    k_readback<<<1, 256, 0, s>>>(static_cast<const uint32_t*>(dev_src), dmap, (int)(bytes / 4));
    KK_CUDA(h, cudaGetLastError(), "readback launch");
    return KK_OK;
  }
  KK_CUDA(h, cudaMemcpyAsync(host_dst, dev_src, bytes, cudaMemcpyDeviceToHost, s), "readback");
  return KK_OK;
}

kk_status check_csr(kk_spgemm_handle h, const kk_csr* M, const char* name, bool need_vals) {
  if (!M) return fail(h, KK_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (M->m < 0 || M->n < 0 || M->nnz < 0)
    return fail(h, KK_ERR_INVALID_ARG, std::string(name) + ": negative size");
  if (!M->rowptr) return fail(h, KK_ERR_INVALID_ARG, std::string(name) + ".rowptr is NULL");
  if (M->nnz > 0 && !M->colind) return fail(h, KK_ERR_INVALID_ARG, std::string(name) + ".colind is NULL");
  if (need_vals && M->nnz > 0 && !M->vals)
    return fail(h, KK_ERR_INVALID_ARG, std::string(name) + ".vals is NULL");
  return KK_OK;
}

CsrView view(const kk_csr* M) {
  return CsrView{M->m, M->n, M->nnz, M->rowptr, M->colind, M->vals};
}

// Bin tables from the options.  Symbolic bins are keyed by the flop bound,
// numeric bins by nnz(C(i,:)).  Team bins come in a vector and a flattened
// flavour; the CTA and dense tiers always flatten.
void build_bins(const kk_spgemm_options& o, bool numeric, std::vector<BinSpec>& out) {
  out.clear();
  const int force = o.force_tier;
  // thread tier first (automatic tier choice only)
  if (force == -1)
    out.push_back(BinSpec{kTierThread, 1, 0, 0, 0, numeric ? kThreadNumMax : kThreadSymMax});
  if (!numeric) {
    if (force < 1) {
      for (int ls = 5; ls <= 12; ++ls) {
        const long long S = 1ll << ls;
        const long long hi = (S * o.sym_load_pct) / 100;
        if (hi > o.sym_team_max_flop && ls > 5) break;
        out.push_back(BinSpec{kTierTeam, 32, (int)S, 0, 0, hi});
        out.push_back(BinSpec{kTierTeam, S <= 64 ? 8 : 32, (int)S, 1, 0, hi});
      }
    }
    if (force < 2) {
      for (int ls = 13; ls <= 15; ++ls) {
        const long long S = 1ll << ls;
        const long long hi = (S * o.sym_load_pct) / 100;
        if (hi > o.sym_cta_max_flop && ls > 13) break;
        out.push_back(BinSpec{kTierCta, 512, (int)S, 1, 0, hi});
      }
    }
    out.push_back(BinSpec{kTierDense, 512, 1 << 20, 1, 0, (long long)9e18});
  } else {
    if (force < 1) {
      for (int ls = 5; ls <= 11; ++ls) {
        const long long S = 1ll << ls;
        const long long hi = (S * o.num_load_pct) / 100;
        if (hi > o.num_team_max_nnz && ls > 5) break;
        out.push_back(BinSpec{kTierTeam, 32, (int)S, 0, 0, hi});
        out.push_back(BinSpec{kTierTeam, S <= 64 ? 8 : 32, (int)S, 1, 0, hi});
      }
    }
    if (force < 2) {
      for (int ls = 12; ls <= 13; ++ls) {
        const long long S = 1ll << ls;
        const long long hi = (S * o.num_load_pct) / 100;
        if (hi > o.num_cta_max_nnz && ls > 12) break;
        out.push_back(BinSpec{kTierCta, 512, (int)S, 1, 0, hi});
      }
    }
    out.push_back(BinSpec{kTierDense, 512, 16384, 1, 0, (long long)9e18});
  }
  for (size_t b = 0; b < out.size(); ++b) out[b].lo = b == 0 ? 1 : out[b - 1].hi + 1;
  // window bins last (looked up through the table's window classes)
  if (o.use_window && (force == -1 || force == 3)) {
    for (int w = 0; w < kNumWindowClasses; ++w)
      out.push_back(BinSpec{kTierWindow, 128, kWindowBits[w], 0, 0,
                            numeric ? kWindowMaxNnz : (long long)9e18});
    // numeric rows of up to kWindowMaxNnzWide columns: large value arrays
    if (numeric)
      for (const int32_t vmax : {kWindowMidNnz, kWindowMaxNnzWide})
        for (int w = 0; w < kNumWideWindowClasses; ++w)
          out.push_back(BinSpec{kTierWindow, 128, kWideWindowBits[w], 0, 0, vmax});
  }
}

BinTable to_table(const std::vector<BinSpec>& bins) {
  BinTable t{};
  t.nb = 0;
  t.nwin = 0;
  for (size_t b = 0; b < bins.size(); ++b) {
    if (bins[b].tier == kTierWindow) {
      t.win_bits[t.nwin] = bins[b].slots;
      t.win_bin[t.nwin] = (int32_t)b;
      t.win_q[t.nwin] = bins[b].hi;
      // large-value numeric bins take only rows of more than kWindowMaxNnz
      // columns (sparser rows than the ratio of the others admits: their cost
      // follows the touched words rather than W); rows of fewer columns that
      // miss the other window bins go to the hash tiers
      const bool large = bins[b].hi > kWindowMaxNnz && bins[b].hi <= kWindowMaxNnzWide;
      t.win_ratio[t.nwin] = large ? kWindowFlopRatioNum : kWindowFlopRatio;
      t.win_qlo[t.nwin] = large ? kWindowMaxNnz : 0;
      ++t.nwin;
    } else {
      t.nb = (int32_t)b + 1;
    }
  }
  t.thread_flop = kThreadNumMaxFlop;
  for (int b = 0; b < t.nb; ++b) {
    t.hi[b] = bins[b].hi;
    t.mode[b] = bins[b].tier == kTierThread ? 3 : bins[b].tier == kTierTeam ? bins[b].flat : 2;
  }
  return t;
}

LaunchCtx ctx_of(kk_spgemm_handle h) {
  return LaunchCtx{h->stream, h->timer, &h->d_misc.as<Misc>()->status, h->num_sms, h->max_smem,
                   h->d_rowlo.as<int32_t>(), h->d_flop.as<long long>(), h->keep, h->opt.debug_checks,
                   h->opt.stage_long_rows, nullptr, h->opt.arith == KK_ARITH_AUTO ? 1 : 0};
}

// Analysis of B at the start of a symbolic call; with the window tier on, the
// same pass writes the compressed B (valid once B is known to be sorted, see
// accept_bcomp).
kk_status analyze_b(kk_spgemm_handle h, const CsrView& bv) {
  h->bc_valid = false;
  if (bv.m <= 0) return KK_OK;
  int2* bc = nullptr;
  int32_t* len = nullptr;
  if (h->opt.use_window) {
    KK_CUDA(h, h->d_bc.ensure(sizeof(int2) * ((size_t)bv.nnz + 2)), "alloc compressed B");
    KK_CUDA(h, h->d_bclen.ensure(sizeof(int32_t) * (size_t)bv.m), "alloc compressed B");
    bc = h->d_bc.as<int2>();
    len = h->d_bclen.as<int32_t>();
  }
  Misc* dm = h->d_misc.as<Misc>();
  KK_CUDA(h, launch_analyze_b(ctx_of(h), bv, &dm->sorted, bc, len, &dm->bc_pairs), "analyze launch");
  return KK_OK;
}

// After the symbolic call's readback: the compressed B written by analyze_b
// belongs to these arrays if B is sorted.
void accept_bcomp(kk_spgemm_handle h, const CsrView& bv, bool analyzed) {
  h->bc_valid = analyzed && h->opt.use_window && h->b_sorted && bv.m > 0;
  h->bc_key[0] = bv.rowptr;
  h->bc_key[1] = bv.colind;
  h->bc_m = bv.m;
  h->bc_nnz = bv.nnz;
}

// Compressed B for a window launch (sorted B only): the one of the last
// symbolic call, rebuilt when B's index arrays are not the ones it was built
// from.  *built = 1 when a kernel was launched.
kk_status ensure_bcomp(kk_spgemm_handle h, const CsrView& bv, BComp* out, int* built) {
  out->bc = nullptr;
  out->len = nullptr;
  *built = 0;
  if (!h->opt.use_window || !h->b_sorted || bv.m <= 0) return KK_OK;
  const bool same = h->bc_valid && h->bc_key[0] == bv.rowptr && h->bc_key[1] == bv.colind &&
                    h->bc_m == bv.m && h->bc_nnz == bv.nnz;
  if (!same) {
    h->bc_valid = false;
    KK_CUDA(h, h->d_bc.ensure(sizeof(int2) * ((size_t)bv.nnz + 2)), "alloc compressed B");
    KK_CUDA(h, h->d_bclen.ensure(sizeof(int32_t) * (size_t)bv.m), "alloc compressed B");
    // sortedness is not re-decided here: the flag goes to a scratch word
    KK_CUDA(h, launch_analyze_b(ctx_of(h), bv, &h->d_misc.as<Misc>()->pad, h->d_bc.as<int2>(),
                                h->d_bclen.as<int32_t>(), nullptr),
            "compress launch");
    accept_bcomp(h, bv, true);
    *built = 1;
  }
  out->bc = h->d_bc.as<int2>();
  out->len = h->d_bclen.as<int32_t>();
  return KK_OK;
}

int grid_for(long long work, int per_block, int cap);

// Fingerprint of A's and B's index arrays into *out (device; B's arrays are
// skipped when they are A's).
kk_status fingerprint(kk_spgemm_handle h, const CsrView& av, const CsrView& bv,
                      unsigned long long* out) {
  FpArrays arr{};
  int na = 0;
  long long maxn = 0;
  auto add = [&](const int32_t* p, long long n) {
    if (!p || n <= 0) return;
    arr.p[na] = p;
    arr.n[na] = n;
    maxn = n > maxn ? n : maxn;
    ++na;
  };
  add(av.rowptr, (long long)av.m + 1);
  add(av.colind, av.nnz);
  if (bv.rowptr != av.rowptr) add(bv.rowptr, (long long)bv.m + 1);
  if (bv.colind != av.colind) add(bv.colind, bv.nnz);
  KK_CUDA(h, cudaMemsetAsync(out, 0, sizeof(unsigned long long), h->stream), "memset");
  if (na == 0) return KK_OK;
  timer_begin(h->timer, h->stream, "fingerprint");
  const dim3 grid(grid_for((maxn + 4 * kFpUnroll - 1) / (4 * kFpUnroll), kFpThreads, h->num_sms * 4), na);
  k_fingerprint<<<grid, kFpThreads, 0, h->stream>>>(arr, out);
  timer_end(h->timer, h->stream);
  KK_CUDA(h, cudaGetLastError(), "fingerprint launch");
  return KK_OK;
}

// Structure cache for the symbolic window kernel: every row starts without
// kept structure (n = -1); null pointers when the option is off or no row of
// the call takes the window tier.  The index arrays' fingerprint is recorded
// with it.
kk_status cache_for_symbolic(kk_spgemm_handle h, int32_t m, bool any_window, const CsrView& av,
                             const CsrView& bv, WinCache* out) {
  *out = WinCache{nullptr, nullptr, nullptr, nullptr};
  h->cache_valid = false;
  if (!h->opt.structure_cache || !any_window || m <= 0) return KK_OK;
  KK_CUDA(h, h->d_cw.ensure(sizeof(uint16_t) * (size_t)m * kCacheWords), "alloc structure cache");
  KK_CUDA(h, h->d_cm.ensure(sizeof(uint32_t) * (size_t)m * kCacheWords), "alloc structure cache");
  KK_CUDA(h, h->d_cn.ensure(sizeof(int32_t) * (size_t)m), "alloc structure cache");
  KK_CUDA(h, cudaMemsetAsync(h->d_cn.p, 0xFF, sizeof(int32_t) * (size_t)m, h->stream), "memset cache");
  *out = WinCache{h->d_cw.as<uint16_t>(), h->d_cm.as<uint32_t>(), h->d_cn.as<int32_t>(),
                  &h->d_misc.as<Misc>()->kept};
  kk_status st = fingerprint(h, av, bv, &h->d_misc.as<Misc>()->fp[0]);
  if (st != KK_OK) return st;
  h->cache_valid = true;
  h->cache_key[0] = av.rowptr;
  h->cache_key[1] = av.colind;
  h->cache_key[2] = bv.rowptr;
  h->cache_key[3] = bv.colind;
  return KK_OK;
}

// Slots for the wide tier's kept bit vectors of this symbolic call (none when
// the option is off, no row takes the wide tier or the budget is zero).
kk_status keep_for_symbolic(kk_spgemm_handle h, int32_t m, int64_t wide_rows, const CsrView& av,
                            const CsrView& bv) {
  h->keep = WideKeep{nullptr, nullptr, nullptr, 0, 0};
  h->keep_valid = false;
  if (!h->opt.structure_cache || h->opt.wide_cache_mb < 0 || wide_rows <= 0 || m <= 0) return KK_OK;
  const LaunchCtx probe = ctx_of(h);
  if (!wide_symbolic_fits(probe, bv.n) || !wide_numeric_fits(probe, bv.n)) return KK_OK;
  const size_t words = (size_t)wide_word_count(bv.n);
  const size_t budget = h->opt.wide_cache_mb > 0 ? ((size_t)h->opt.wide_cache_mb << 20) : h->dev_total / 8;
  long long slots = (long long)(budget / (words * 4));
  if (slots > wide_rows) slots = wide_rows;
  if (slots > 0x7fffffff) slots = 0x7fffffff;
  if (slots <= 0) return KK_OK;
  KK_CUDA(h, h->d_wbits.ensure(words * 4 * (size_t)slots), "alloc wide cache");
  KK_CUDA(h, h->d_wslot.ensure(sizeof(int32_t) * (size_t)m), "alloc wide cache");
  KK_CUDA(h, h->d_wnext.ensure(sizeof(int32_t)), "alloc wide cache");
  KK_CUDA(h, cudaMemsetAsync(h->d_wslot.p, 0xFF, sizeof(int32_t) * (size_t)m, h->stream), "memset");
  KK_CUDA(h, cudaMemsetAsync(h->d_wnext.p, 0, sizeof(int32_t), h->stream), "memset");
  h->keep = WideKeep{h->d_wbits.as<uint32_t>(), h->d_wslot.as<int32_t>(), h->d_wnext.as<int32_t>(),
                     (int32_t)slots, wide_keep_min_cnt(probe, bv.n)};
  h->keep_valid = true;
  h->keep_key[0] = av.rowptr;
  h->keep_key[1] = av.colind;
  h->keep_key[2] = bv.rowptr;
  h->keep_key[3] = bv.colind;
  return KK_OK;
}

// The kept wide bit vectors for a numeric call, if they belong to its arrays.
void keep_for_numeric(kk_spgemm_handle h, const CsrView& av, const CsrView& bv) {
  if (h->keep_valid && h->keep_key[0] == av.rowptr && h->keep_key[1] == av.colind &&
      h->keep_key[2] == bv.rowptr && h->keep_key[3] == bv.colind) {
    h->keep.next = nullptr;  // the numeric phase only reads
  } else {
    h->keep = WideKeep{nullptr, nullptr, nullptr, 0, 0};
  }
}

// The kept structure, if it belongs to these index arrays, and the scratch
// its numeric launches need.  Unless options.debug_checks asks for a check of
// every product, the arrays' fingerprint is taken again and ctx->fingerprint
// points the numeric kernels at both fingerprints.
kk_status cache_view(kk_spgemm_handle h, const CsrView& av, const CsrView& bv, WinCacheView* view,
                     WinScratch* scratch, LaunchCtx* ctx) {
  *view = WinCacheView{nullptr, nullptr, nullptr};
  *scratch = WinScratch{nullptr, nullptr};
  if (!h->cache_valid || h->cache_key[0] != av.rowptr || h->cache_key[1] != av.colind ||
      h->cache_key[2] != bv.rowptr || h->cache_key[3] != bv.colind)
    return KK_OK;
  KK_CUDA(h, h->d_left.ensure(sizeof(int32_t) * ((size_t)av.m + 1)), "alloc window scratch");
  *view = WinCacheView{h->d_cw.as<uint16_t>(), h->d_cm.as<uint32_t>(), h->d_cn.as<int32_t>()};
  *scratch = WinScratch{h->d_left.as<int32_t>() + 1, h->d_left.as<int32_t>()};
  if (!h->opt.debug_checks) {
    Misc* dm = h->d_misc.as<Misc>();
    kk_status st = fingerprint(h, av, bv, &dm->fp[1]);
    if (st != KK_OK) return st;
    ctx->fingerprint = dm->fp;
  }
  return KK_OK;
}

int grid_for(long long work, int per_block, int cap) {
  long long g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Stable binning of m rows by `bin` into rows_out; writes bin_start (device,
// nb+1 entries).
kk_status run_binning(kk_spgemm_handle h, int32_t m, const uint8_t* bin, int nb, int32_t* rows_out,
                      int32_t* bin_start) {
  const int nblk = (int)((m + kBinRows - 1) / kBinRows);
  if (nblk == 0) {
    KK_CUDA(h, cudaMemsetAsync(bin_start, 0, sizeof(int32_t) * (nb + 1), h->stream), "memset");
    return KK_OK;
  }
  KK_CUDA(h, h->d_blk.ensure(sizeof(int32_t) * (size_t)nb * nblk), "alloc bins");
  int32_t* blk = h->d_blk.as<int32_t>();
  timer_begin(h->timer, h->stream, "binning");
  k_bin_count<<<nblk, kBinBlock, 0, h->stream>>>(m, bin, nb, nblk, blk);
  k_bin_scan<<<1, 1024, 0, h->stream>>>(nb, nblk, blk, bin_start);
  k_bin_scatter<<<nblk, kBinBlock, 0, h->stream>>>(m, bin, nb, nblk, blk, rows_out);
  timer_end(h->timer, h->stream);
  KK_CUDA(h, cudaGetLastError(), "binning launch");
  return KK_OK;
}

kk_status check_device_status(kk_spgemm_handle h, int status) {
  if (status == 0) return KK_OK;
  const char* what = "device error";
  switch (status) {
    case KK_ERR_BAD_INDEX: what = "a column index lies outside its range"; break;
    case KK_ERR_INVALID_ARG: what = "a row of A has no nonzero stored diagonal (Jacobi)"; break;
    case KK_ERR_CAPACITY: what = "an accumulator overflowed"; break;
    case KK_ERR_STRUCTURE_MISMATCH: what = "the structure differs from the symbolic phase"; break;
    case KK_ERR_TIMEOUT: what = "a bounded device wait ran out"; break;
    default: break;
  }
  return fail(h, (kk_status)status, what);
}

}  // namespace

// Jacobi row scaling of rows[0..nrows) with teams of T lanes, one resident
// wave of blocks.
template <int T, int U>
static void launch_jacobi_rows_t(kk_spgemm_handle h, const CsrView& av, const int32_t* rows, int32_t nrows) {
  static int per_sm = 0;
  if (per_sm == 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_rows<T, U>, 256, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = 4;
  }
  k_jacobi_rows<T, U><<<grid_for((long long)nrows * T, 256, h->num_sms * (per_sm > 0 ? per_sm : 1)), 256, 0,
                        h->stream>>>(av, rows, nrows, av.jac_omega, const_cast<double*>(av.jac_s),
                                     const_cast<int32_t*>(av.jac_p), &h->d_misc.as<Misc>()->status);
}

// Team width by the mean row length of A: one lane per row for short rows (AMG
// operators), a warp for long ones.
static cudaError_t launch_jacobi_rows(kk_spgemm_handle h, const CsrView& av, const int32_t* rows,
                                      int32_t nrows) {
  timer_begin(h->timer, h->stream, "jacobi_rows");
  const long long avg = av.m > 0 ? (long long)av.nnz / av.m : 0;
  if (avg <= 8)
    launch_jacobi_rows_t<1, 8>(h, av, rows, nrows);
  else if (avg <= 32)
    launch_jacobi_rows_t<4, 8>(h, av, rows, nrows);
  else
    launch_jacobi_rows_t<32, 4>(h, av, rows, nrows);
  timer_end(h->timer, h->stream);
  return cudaGetLastError();
}

// Analysis of A with teams of T lanes, one resident wave of blocks (the kernel
// strides over rows).
// bin receives the symbolic bin ids; with STATS, stat the learned form's row
// statistics.
template <int T, int U, bool STATS = false>
static void launch_analyze_a(kk_spgemm_handle h, const CsrView& av, const CsrView& bv, Misc* dm,
                             cudaStream_t s, uint8_t* bin, int2* stat = nullptr) {
  static int per_sm = 0;
  if (per_sm == 0 &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_analyze_a<T, U, STATS>, 256, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    per_sm = 4;
  }
  const int64_t m = av.m;
  k_analyze_a<T, U, STATS><<<grid_for(m * T, 256, h->num_sms * (per_sm > 0 ? per_sm : 1)), 256, 0, s>>>(
      av, bv.rowptr, bv.colind, bv.m, &dm->sorted, to_table(h->sym_bins), h->opt.team_vec_min_len,
      h->d_flop.as<long long>(), bin, h->d_rowlo.as<int32_t>(), h->d_span.as<int32_t>(), stat,
      &dm->total_flop, &dm->status);
}

extern "C" {

const char* kk_status_string(kk_status s) {
  switch (s) {
    case KK_OK: return "KK_OK";
    case KK_ERR_INVALID_ARG: return "KK_ERR_INVALID_ARG";
    case KK_ERR_CUDA: return "KK_ERR_CUDA";
    case KK_ERR_OOM: return "KK_ERR_OOM";
    case KK_ERR_STRUCTURE_MISMATCH: return "KK_ERR_STRUCTURE_MISMATCH";
    case KK_ERR_CAPACITY: return "KK_ERR_CAPACITY";
    case KK_ERR_TIMEOUT: return "KK_ERR_TIMEOUT";
    case KK_ERR_NOT_SYMBOLIC: return "KK_ERR_NOT_SYMBOLIC";
    case KK_ERR_BAD_INDEX: return "KK_ERR_BAD_INDEX";
  }
  return "KK_ERR_UNKNOWN";
}

kk_status kk_spgemm_options_default(kk_spgemm_options* opt) {
  if (!opt) return KK_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->arith = KK_ARITH_AUTO;
  opt->debug_checks = 0;
  opt->batched_learned = 0;
  opt->timing = 0;
  opt->force_tier = -1;
  opt->team_vec_min_len = 12;
  opt->sym_team_max_flop = 3072;
  opt->sym_cta_max_flop = 24576;
  opt->num_team_max_nnz = 1024;
  opt->num_cta_max_nnz = 4096;
  opt->use_window = 1;
  opt->batched_graph = 1;
  opt->sym_load_pct = 75;
  opt->num_load_pct = 50;
  opt->structure_cache = 1;
  opt->wide_cache_mb = 0;
  opt->batched_mode = 0;
  opt->stage_long_rows = 0;
  opt->small_max_rows = 4096;
  return KK_OK;
}

kk_status kk_spgemm_handle_create(kk_spgemm_handle* out, const kk_spgemm_options* opt,
                                  void* cuda_stream) {
  if (!out) return KK_ERR_INVALID_ARG;
  *out = nullptr;
  kk_spgemm_handle h = new (std::nothrow) kk_spgemm_handle_s();
  if (!h) return KK_ERR_OOM;
  if (opt) h->opt = *opt; else kk_spgemm_options_default(&h->opt);
  if (h->opt.arith < 0 || h->opt.arith > 2 || h->opt.force_tier < -1 || h->opt.force_tier > 3 ||
      h->opt.sym_load_pct < 10 || h->opt.sym_load_pct > 100 || h->opt.num_load_pct < 10 ||
      h->opt.num_load_pct > 50 || h->opt.structure_cache < 0 || h->opt.structure_cache > 1 || h->opt.wide_cache_mb < -1 || h->opt.batched_mode < 0 ||
      h->opt.batched_mode > 2 || h->opt.stage_long_rows < 0 || h->opt.stage_long_rows > 1 ||
      h->opt.small_max_rows < 0 || h->opt.small_max_rows > kSmallMaxRowsCap ||
      h->opt.team_vec_min_len < 0) {
    delete h;
    return KK_ERR_INVALID_ARG;
  }
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e == cudaSuccess) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    h->dev_total = tot;
  }
  if (e == cudaSuccess) e = h->d_misc.ensure(sizeof(Misc));
  if (e == cudaSuccess) e = h->d_binstart.ensure(sizeof(int32_t) * 2 * (kMaxBins + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_pinned, 4096);
  if (e == cudaSuccess && cudaHostGetDevicePointer(&h->d_pinned_map, h->h_pinned, 0) != cudaSuccess) {
    (void)cudaGetLastError();  // no device mapping: read-backs take cudaMemcpyAsync
    h->d_pinned_map = nullptr;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_misc.p, 0, sizeof(Misc), h->stream);
  if (e != cudaSuccess) {
    h->d_misc.release();
    h->d_binstart.release();
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    delete h;
    return e == cudaErrorMemoryAllocation ? KK_ERR_OOM : KK_ERR_CUDA;
  }
  if (h->opt.timing) h->timer = new (std::nothrow) KernelTimer();
  *out = h;
  return KK_OK;
}

kk_status kk_spgemm_set_stream(kk_spgemm_handle h, void* cuda_stream) {
  if (!h) return KK_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return KK_OK;
}

const char* kk_spgemm_last_error(kk_spgemm_handle h) { return h ? h->last_error.c_str() : ""; }

int32_t kk_spgemm_last_arith(kk_spgemm_handle h) { return h ? h->last_arith : 0; }

kk_status kk_spgemm_stats(kk_spgemm_handle h, int64_t stats[32]) {
  if (!h || !stats) return KK_ERR_INVALID_ARG;
  for (int i = 0; i < 32; ++i) stats[i] = h->stats[i];
  return KK_OK;
}

kk_status kk_spgemm_symbolic(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                             int64_t* c_rowptr, int64_t* nnz_c) {
  if (!h) return KK_ERR_INVALID_ARG;
  kk_status st;
  if ((st = check_csr(h, A, "A", false)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", false)) != KK_OK) return st;
  if (A->n != B->m) return fail(h, KK_ERR_INVALID_ARG, "A.n != B.m");
  if (!c_rowptr || !nnz_c) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr / nnz_c is NULL");
  h->have_symbolic = false;
  const int32_t m = A->m;
  const CsrView av = view(A), bv = view(B);
  cudaStream_t s = h->stream;
  Misc* dm = h->d_misc.as<Misc>();
  Misc* hm = static_cast<Misc*>(h->h_pinned);
  int32_t* h_start = reinterpret_cast<int32_t*>(static_cast<char*>(h->h_pinned) + 256);

  build_bins(h->opt, false, h->sym_bins);
  build_bins(h->opt, true, h->num_bins);
  const int nbs = (int)h->sym_bins.size(), nbn = (int)h->num_bins.size();

  KK_CUDA(h, h->d_flop.ensure(sizeof(long long) * (size_t)(m > 0 ? m : 1)), "alloc flop");
  KK_CUDA(h, h->d_sbin.ensure((size_t)(m > 0 ? m : 1)), "alloc bins");
  KK_CUDA(h, h->d_nbin.ensure((size_t)(m > 0 ? m : 1)), "alloc bins");
  KK_CUDA(h, h->d_srows.ensure(sizeof(int32_t) * (size_t)(m > 0 ? m : 1)), "alloc rows");
  KK_CUDA(h, h->d_nrows.ensure(sizeof(int32_t) * (size_t)(m > 0 ? m : 1)), "alloc rows");
  KK_CUDA(h, h->d_cnt.ensure(sizeof(int32_t) * (size_t)(m > 0 ? m : 1)), "alloc counts");
  KK_CUDA(h, h->d_rowlo.ensure(sizeof(int32_t) * (size_t)(m > 0 ? m : 1)), "alloc spans");
  KK_CUDA(h, h->d_span.ensure(sizeof(int32_t) * (size_t)(m > 0 ? m : 1)), "alloc spans");
  const int nblk_scan = (int)((m + kScanRows - 1) / kScanRows);
  KK_CUDA(h, h->d_scan.ensure(sizeof(long long) * (size_t)(nblk_scan > 0 ? nblk_scan : 1)), "alloc scan");

  Misc init{};
  init.sorted = 1;
  KK_CUDA(h, cudaMemcpyAsync(dm, &init, sizeof(Misc), cudaMemcpyHostToDevice, s), "init");
  // NOTE: &init is pageable; cudaMemcpyAsync from pageable memory is staged
  // synchronously with respect to the host, so the stack copy is safe.

  // Small products: one launch counts every row and scans the counts
  // (small_flags: a row beyond the path, a bad index; grand / grand2: nnz(C)
  // and the multiply-adds); a row beyond the path sends the call on to the
  // tiered path below.
  h->small = false;
  if (m > 0 && m <= h->opt.small_max_rows && h->opt.force_tier == -1 &&
      (long long)av.nnz * (long long)bv.nnz <=
          (long long)kSmallMaxMeanFlop * (long long)m * (long long)(bv.m > 0 ? bv.m : 1)) {
    timer_begin(h->timer, s, "small_symbolic");
    cudaError_t e = launch_small_symbolic(ctx_of(h), av, bv, c_rowptr, h->d_cnt.as<int32_t>(), dm->small_flags,
                                          &dm->grand);
    timer_end(h->timer, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "small symbolic launch");
    KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
    KK_CUDA(h, cudaStreamSynchronize(s), "sync");
    if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
    if (hm->small_flags[1]) return fail(h, KK_ERR_BAD_INDEX, "a row pointer or column index of A or B is out of range");
    if (!hm->small_flags[0]) {
      for (int k = 0; k < 32; ++k) h->stats[k] = 0;
      h->stats[6] = (int64_t)hm->grand2;
      h->stats[8] = 1;
      h->stats[30] = m;
      h->small = true;
      h->cache_valid = false;
      h->keep = WideKeep{nullptr, nullptr, nullptr, 0, 0};
      h->keep_valid = false;
      h->learned_valid = false;
      h->nnz_c = hm->grand;
      h->am = m;
      h->an = A->n;
      h->bn = B->n;
      h->annz = A->nnz;
      h->bnnz = B->nnz;
      h->have_symbolic = true;
      *nnz_c = h->nnz_c;
      return KK_OK;
    }
    KK_CUDA(h, cudaMemcpyAsync(dm, &init, sizeof(Misc), cudaMemcpyHostToDevice, s), "init");
  }

  int32_t* sym_start = h->d_binstart.as<int32_t>();
  int32_t* num_start = sym_start + (kMaxBins + 1);
  if (m > 0) {
    timer_begin(h->timer, s, "analyze");
    if ((st = analyze_b(h, bv)) != KK_OK) return st;
    // smallest team whose U = 8 gathers per lane cover a typical row in one
    // round (more rows in flight per SM; measured against teams of 4 and 8)
    const long long avg = m > 0 ? (long long)av.nnz / m : 0;
    if (avg <= 8)
      launch_analyze_a<1, 8>(h, av, bv, dm, s, h->d_sbin.as<uint8_t>());
    else
      launch_analyze_a<4, 8>(h, av, bv, dm, s, h->d_sbin.as<uint8_t>());
    timer_end(h->timer, s);
    KK_CUDA(h, cudaGetLastError(), "analyze launch");
    if ((st = run_binning(h, m, h->d_sbin.as<uint8_t>(), nbs, h->d_srows.as<int32_t>(), sym_start)) != KK_OK)
      return st;
  } else {
    KK_CUDA(h, cudaMemsetAsync(sym_start, 0, sizeof(int32_t) * (nbs + 1), s), "memset");
  }
  KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
  KK_TRY(readback(h, h_start, sym_start, sizeof(int32_t) * (nbs + 1), s));
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
  h->b_sorted = hm->sorted;
  h->stats[6] = (int64_t)hm->total_flop;
  h->stats[7] = hm->sorted;
  accept_bcomp(h, bv, m > 0);

  // symbolic kernels per bin
  if (m > 0) {
    KK_CUDA(h, cudaMemsetAsync(h->d_cnt.p, 0, sizeof(int32_t) * (size_t)m, s), "memset counts");
    int64_t wide_rows = 0;
    for (int b = 0; b < nbs; ++b)
      if (h->sym_bins[b].tier == kTierCta || h->sym_bins[b].tier == kTierDense)
        wide_rows += h_start[b + 1] - h_start[b];
    if ((st = keep_for_symbolic(h, m, wide_rows, av, bv)) != KK_OK) return st;
    LaunchCtx ctx = ctx_of(h);
    bool any_win = false;
    for (int b = 0; b < nbs; ++b)
      if (h->sym_bins[b].tier == kTierWindow && h_start[b + 1] > h_start[b]) any_win = true;
    BComp bcomp;
    int bc_built = 0;
    if ((st = ensure_bcomp(h, bv, &bcomp, &bc_built)) != KK_OK) return st;
    WinCache wcache;
    if ((st = cache_for_symbolic(h, m, any_win, av, bv, &wcache)) != KK_OK) return st;
    int64_t tier_rows[4] = {0, 0, 0, 0};
    for (int b = 0; b < nbs; ++b) {
      const int cnt = h_start[b + 1] - h_start[b];
      if (cnt <= 0) continue;
      tier_rows[stat_tier(h->sym_bins[b].tier)] += cnt;
      const int32_t* rows = h->d_srows.as<int32_t>() + h_start[b];
      cudaError_t e = h->sym_bins[b].tier == kTierWindow
                          ? launch_symbolic_window(ctx, h->sym_bins[b], av, bv, bcomp, rows, cnt,
                                                   h->d_cnt.as<int32_t>(), wcache)
                          : launch_symbolic_bin(ctx, h->sym_bins[b], av, bv, h->b_sorted, rows, cnt,
                                                h->d_cnt.as<int32_t>());
      if (e != cudaSuccess) return cuda_fail(h, e, "symbolic launch");
    }
    for (int t = 0; t < 3; ++t) h->stats[t] = tier_rows[t];
    h->stats[10] = tier_rows[kTierWindow];
    int64_t nb_launched = 0;
    for (int b = 0; b < nbs; ++b) nb_launched += (h_start[b + 1] - h_start[b]) > 0 ? 1 : 0;
    // analyze (2) + binning (3) + symbolic bins + scan (3) + numeric binning (3)
    h->stats[8] = (bv.m > 0 ? 1 : 0) + 1 + 3 + nb_launched + 3 + 3 + (h->opt.timing ? 1 : 0);
    // scan + numeric bins
    timer_begin(h->timer, s, "scan");
    k_scan_partial<<<nblk_scan, kScanBlock, 0, s>>>(m, h->d_cnt.as<int32_t>(), h->d_scan.as<long long>());
    k_scan_top<<<1, 1024, 0, s>>>(nblk_scan, h->d_scan.as<long long>(), &dm->grand);
    k_scan_final<<<nblk_scan, kScanBlock, 0, s>>>(
        m, h->d_cnt.as<int32_t>(), h->d_scan.as<long long>(), h->d_flop.as<long long>(), av.rowptr,
        h->d_span.as<int32_t>(), &dm->sorted, h->opt.team_vec_min_len, to_table(h->num_bins),
        c_rowptr, h->d_nbin.as<uint8_t>());
    timer_end(h->timer, s);
    KK_CUDA(h, cudaGetLastError(), "scan launch");
    if ((st = run_binning(h, m, h->d_nbin.as<uint8_t>(), nbn, h->d_nrows.as<int32_t>(), num_start)) != KK_OK)
      return st;
    // per-tier C entries, A entries and multiply-adds (statistics for
    // per-kernel accounting): only on a handle that times its kernels
    if (h->opt.timing)
      k_tier_sums<<<grid_for(m, 256, h->num_sms * 8), 256, 0, s>>>(
          m, h->d_nbin.as<uint8_t>(), c_rowptr, av.rowptr, h->d_flop.as<long long>(), tier_of_bins(h->num_bins),
          dm->tier_c, dm->tier_a, dm->tier_f);
  } else {
    KK_CUDA(h, cudaMemsetAsync(c_rowptr, 0, sizeof(int64_t), s), "memset rowptr");
    KK_CUDA(h, cudaMemsetAsync(num_start, 0, sizeof(int32_t) * (nbn + 1), s), "memset");
  }
  KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
  KK_TRY(readback(h, h_start, num_start, sizeof(int32_t) * (nbn + 1), s));
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
  h->nnz_c = m > 0 ? hm->grand : 0;
  h->num_start.assign(h_start, h_start + nbn + 1);
  int64_t ntier[4] = {0, 0, 0, 0};
  for (int b = 0; b < nbn; ++b) ntier[stat_tier(h->num_bins[b].tier)] += h_start[b + 1] - h_start[b];
  for (int t = 0; t < 3; ++t) h->stats[3 + t] = ntier[t];
  h->stats[11] = ntier[kTierWindow];
  for (int t = 0; t < 4; ++t) {
    h->stats[16 + t] = (int64_t)hm->tier_c[t];
    h->stats[20 + t] = (int64_t)hm->tier_a[t];
    h->stats[26 + t] = (int64_t)hm->tier_f[t];
  }
  h->stats[24] = (int64_t)hm->kept;
  h->stats[25] = (int64_t)hm->bc_pairs;
  h->am = m;
  h->an = A->n;
  h->bn = B->n;
  h->annz = A->nnz;
  h->bnnz = B->nnz;
  h->have_symbolic = true;
  *nnz_c = h->nnz_c;
  return KK_OK;
}

// The numeric phase; jac makes it the Jacobi-fused phase (see CsrView) with
// weight omega, in float64.
static kk_status numeric_impl(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B, const int64_t* c_rowptr,
                              int32_t* c_colind, double* c_vals, bool jac, double omega) {
  if (!h) return KK_ERR_INVALID_ARG;
  if (!h->have_symbolic) return fail(h, KK_ERR_NOT_SYMBOLIC, "numeric before symbolic");
  kk_status st;
  if ((st = check_csr(h, A, "A", true)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", true)) != KK_OK) return st;
  if (A->m != h->am || A->n != h->an || B->n != h->bn || A->nnz != h->annz || B->nnz != h->bnnz)
    return fail(h, KK_ERR_STRUCTURE_MISMATCH, "A/B dims or nnz differ from the symbolic call");
  if (!c_rowptr) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr is NULL");
  if (h->nnz_c > 0 && (!c_colind || !c_vals)) return fail(h, KK_ERR_INVALID_ARG, "C arrays are NULL");
  CsrView av = view(A);
  if (jac && h->am > 0) {
    KK_CUDA(h, h->d_jvals.ensure(sizeof(double) * (size_t)h->am), "alloc Jacobi row scales");
    KK_CUDA(h, h->d_jpos.ensure(sizeof(int32_t) * (size_t)h->am), "alloc Jacobi row scales");
    av.jac_s = h->d_jvals.as<double>();
    av.jac_p = h->d_jpos.as<int32_t>();
    av.jac_omega = omega;
  }
  const CsrView bv = view(B);
  cudaStream_t s = h->stream;
  Misc* dm = h->d_misc.as<Misc>();
  if (h->small) {  // after a small-path symbolic call: one launch, float64
    h->last_arith = kArithF64;
    if (h->am == 0 || h->nnz_c == 0) return KK_OK;
    timer_begin(h->timer, s, "small_numeric");
    cudaError_t e = launch_small_numeric(ctx_of(h), av, bv, c_rowptr, c_colind, c_vals);
    timer_end(h->timer, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "small numeric launch");
    h->stats[9] = 1;
    return KK_OK;
  }
  // DF32 needs B's rows strictly ascending (its error bound counts at most
  // nnz(A(i,:)) contributions per entry); otherwise the product runs in float64,
  // as does the Jacobi-fused product (its scaled values are formed in float64)
  const int32_t arith =
      (h->opt.arith == KK_ARITH_FP64 || !h->b_sorted || jac) ? kArithF64 : kArithDF32;
  h->last_arith = arith;
  if (h->am == 0 || h->nnz_c == 0) return KK_OK;
  const float2* bsplit = nullptr;
  keep_for_numeric(h, av, bv);
  if (arith == kArithDF32) {
    KK_CUDA(h, h->d_bsplit.ensure(sizeof(float2) * (size_t)(bv.nnz > 0 ? bv.nnz : 1)), "alloc split");
    KK_CUDA(h, cudaMemsetAsync(&dm->range_bad, 0, sizeof(int32_t), s), "memset");
    if (bv.nnz > 0) {
      timer_begin(h->timer, s, "split_b");
      k_split_values<<<grid_for(bv.nnz, 256, h->num_sms * 8), 256, 0, s>>>(
          bv.nnz, bv.vals, h->d_bsplit.as<float2>(), &dm->range_bad);
      timer_end(h->timer, s);
      KK_CUDA(h, cudaGetLastError(), "split launch");
    }
    bsplit = h->d_bsplit.as<float2>();
  }
  LaunchCtx ctx = ctx_of(h);
  const int nbn = (int)h->num_bins.size();
  h->stats[9] = (arith == kArithDF32 && bv.nnz > 0) ? 1 : 0;
  bool any_win = false;
  for (int b = 0; b < nbn; ++b)
    if (h->num_bins[b].tier == kTierWindow && h->num_start[b + 1] > h->num_start[b]) any_win = true;
  BComp bcomp{nullptr, nullptr};
  if (any_win) {
    int built = 0;
    if ((st = ensure_bcomp(h, bv, &bcomp, &built)) != KK_OK) return st;
    h->stats[9] += built;
  }
  WinCacheView wview;
  WinScratch wscratch;
  if ((st = cache_view(h, av, bv, &wview, &wscratch, &ctx)) != KK_OK) return st;
  for (int b = 0; b < nbn; ++b) {
    const int cnt = h->num_start[b + 1] - h->num_start[b];
    if (cnt <= 0) continue;
    h->stats[9] += 1;
    const int32_t* rows = h->d_nrows.as<int32_t>() + h->num_start[b];
    if (jac && h->num_bins[b].tier != kTierThread) {
      // the row scales of this bin's rows (the thread tier forms its own)
      cudaError_t e = launch_jacobi_rows(h, av, rows, cnt);
      if (e != cudaSuccess) return cuda_fail(h, e, "Jacobi launch");
      h->stats[9] += 1;
    }
    cudaError_t e = h->num_bins[b].tier == kTierWindow
                        ? launch_numeric_window(ctx, h->num_bins[b], av, bv, bcomp, wview, wscratch, bsplit,
                                                &dm->range_bad, arith, c_rowptr, rows, cnt, c_colind,
                                                c_vals)
                        : launch_numeric_bin(ctx, h->num_bins[b], av, bv, h->b_sorted, bsplit,
                                             &dm->range_bad, arith, c_rowptr, rows, cnt, c_colind,
                                             c_vals, h->opt.debug_checks);
    if (e != cudaSuccess) return cuda_fail(h, e, "numeric launch");
  }
  return KK_OK;
}

// ---------------------------------------------------------------------------
// Jacobi-fused numeric phase (kk_jacobi.h)
// ---------------------------------------------------------------------------

kk_status kk_spgemm_numeric(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                            const int64_t* c_rowptr, int32_t* c_colind, double* c_vals) {
  return numeric_impl(h, A, B, c_rowptr, c_colind, c_vals, false, 0.0);
}

kk_status kk_spgemm_jacobi_numeric(kk_spgemm_handle h, double omega, const kk_csr* A,
                                   const kk_csr* B, const int64_t* c_rowptr, int32_t* c_colind,
                                   double* c_vals) {
  if (!h) return KK_ERR_INVALID_ARG;
  kk_status st;
  if ((st = check_csr(h, A, "A", true)) != KK_OK) return st;
  if (A->m != A->n) return fail(h, KK_ERR_INVALID_ARG, "Jacobi needs a square A");
  if (!std::isfinite(omega)) return fail(h, KK_ERR_INVALID_ARG, "omega is not finite");
  // the numeric tiers scale A's values by row as they load them
  return numeric_impl(h, A, B, c_rowptr, c_colind, c_vals, true, omega);
}

// ---------------------------------------------------------------------------
// Learned form (kk_learned.h)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// Exclusive scan of int32 counts into int64 offsets out[0..m] (out[m] = total,
// also written to *grand); nbin (nullable) receives numeric bin ids.
kk_status run_scan(kk_spgemm_handle h, int32_t m, const int32_t* cnt, int64_t* out, long long* grand,
                   const CsrView& av, uint8_t* nbin) {
  cudaStream_t s = h->stream;
  const int nblk = (int)((m + kScanRows - 1) / kScanRows);
  if (m == 0) return KK_OK;
  KK_CUDA(h, h->d_scan.ensure(sizeof(long long) * (size_t)nblk), "alloc scan");
  Misc* dm = h->d_misc.as<Misc>();
  k_scan_partial<<<nblk, kScanBlock, 0, s>>>(m, cnt, h->d_scan.as<long long>());
  k_scan_top<<<1, 1024, 0, s>>>(nblk, h->d_scan.as<long long>(), grand);
  k_scan_final<<<nblk, kScanBlock, 0, s>>>(m, cnt, h->d_scan.as<long long>(), h->d_flop.as<long long>(),
                                           av.rowptr, h->d_span.as<int32_t>(), &dm->sorted,
                                           h->opt.team_vec_min_len, to_table(h->num_bins), out, nbin);
  KK_CUDA(h, cudaGetLastError(), "scan launch");
  return KK_OK;
}

}  // namespace

extern "C" {

// ---------------------------------------------------------------------------
// Sparse matrix addition (kk_spadd.h)
// ---------------------------------------------------------------------------
kk_status kk_spadd_symbolic(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B, int64_t* c_rowptr,
                            int64_t* nnz_c) {
  if (!h) return KK_ERR_INVALID_ARG;
  kk_status st;
  if ((st = check_csr(h, A, "A", false)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", false)) != KK_OK) return st;
  if (A->m != B->m || A->n != B->n) return fail(h, KK_ERR_INVALID_ARG, "A and B have different shapes");
  if (!c_rowptr || !nnz_c) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr / nnz_c is NULL");
  h->add_valid = false;
  const int32_t m = A->m;
  cudaStream_t s = h->stream;
  Misc* dm = h->d_misc.as<Misc>();
  Misc* hm = static_cast<Misc*>(h->h_pinned);
  KK_CUDA(h, h->d_apos.ensure(sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1)), "alloc SpAdd");
  KK_CUDA(h, h->d_bpos.ensure(sizeof(int32_t) * (size_t)(B->nnz > 0 ? B->nnz : 1)), "alloc SpAdd");
  KK_CUDA(h, h->d_acnt.ensure(sizeof(int32_t) * (size_t)(m > 0 ? m : 1)), "alloc SpAdd");
  KK_CUDA(h, h->d_along.ensure(sizeof(int32_t) * ((size_t)m + 1)), "alloc SpAdd");
  // only the status word is reset: the rest of the device record belongs to
  // the SpGEMM state of this handle (fingerprints, flags), which SpAdd leaves alone
  KK_CUDA(h, cudaMemsetAsync(&dm->status, 0, sizeof(int), s), "memset");
  KK_CUDA(h, cudaMemsetAsync(h->d_along.p, 0, sizeof(int32_t), s), "memset");
  int64_t nnz = 0;
  if (m > 0) {
    LaunchCtx ctx = ctx_of(h);
    timer_begin(h->timer, s, "spadd_symbolic");
    cudaError_t e = launch_spadd_symbolic(ctx, view(A), view(B), h->d_acnt.as<int32_t>(),
                                          h->d_apos.as<int32_t>(), h->d_bpos.as<int32_t>(),
                                          h->d_along.as<int32_t>() + 1, h->d_along.as<int32_t>());
    timer_end(h->timer, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "SpAdd symbolic launch");
    timer_begin(h->timer, s, "scan");
    if ((st = run_scan(h, m, h->d_acnt.as<int32_t>(), c_rowptr, &dm->grand, view(A), nullptr)) != KK_OK)
      return st;
    timer_end(h->timer, s);
  } else {
    KK_CUDA(h, cudaMemsetAsync(c_rowptr, 0, sizeof(int64_t), s), "memset");
  }
  KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
  if (m > 0) nnz = hm->grand;
  h->add_valid = true;
  h->add_key[0] = A->rowptr;
  h->add_key[1] = A->colind;
  h->add_key[2] = B->rowptr;
  h->add_key[3] = B->colind;
  h->add_m = A->m;
  h->add_n = A->n;
  h->add_nnza = A->nnz;
  h->add_nnzb = B->nnz;
  h->add_nnzc = nnz;
  *nnz_c = nnz;
  return KK_OK;
}

kk_status kk_spadd_numeric(kk_spgemm_handle h, double alpha, const kk_csr* A, double beta,
                           const kk_csr* B, const int64_t* c_rowptr, int32_t* c_colind, double* c_vals) {
  if (!h) return KK_ERR_INVALID_ARG;
  if (!h->add_valid) return fail(h, KK_ERR_NOT_SYMBOLIC, "SpAdd numeric before SpAdd symbolic");
  kk_status st;
  if ((st = check_csr(h, A, "A", true)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", true)) != KK_OK) return st;
  if (A->m != h->add_m || A->n != h->add_n || B->m != h->add_m || B->n != h->add_n ||
      A->nnz != h->add_nnza || B->nnz != h->add_nnzb || A->rowptr != h->add_key[0] ||
      A->colind != h->add_key[1] || B->rowptr != h->add_key[2] || B->colind != h->add_key[3])
    return fail(h, KK_ERR_STRUCTURE_MISMATCH,
                "SpAdd numeric needs the index arrays of the SpAdd symbolic call");
  if (!c_rowptr) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr is NULL");
  if (h->add_nnzc == 0) return KK_OK;
  if (!c_colind || !c_vals) return fail(h, KK_ERR_INVALID_ARG, "C arrays are NULL");
  cudaStream_t s = h->stream;
  timer_begin(h->timer, s, "spadd_numeric");
  KK_CUDA(h, cudaMemsetAsync(c_vals, 0, sizeof(double) * (size_t)h->add_nnzc, s), "memset");
  cudaError_t e = launch_spadd_numeric(ctx_of(h), view(A), view(B), alpha, beta, c_rowptr,
                                       h->d_apos.as<int32_t>(), h->d_bpos.as<int32_t>(), c_colind, c_vals);
  timer_end(h->timer, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "SpAdd numeric launch");
  return KK_OK;
}


kk_status kk_spgemm_row_features(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B, float* features) {
  if (!h) return KK_ERR_INVALID_ARG;
  kk_status st;
  if ((st = check_csr(h, A, "A", false)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", false)) != KK_OK) return st;
  if (A->n != B->m) return fail(h, KK_ERR_INVALID_ARG, "A.n != B.m");
  if (A->m > 0 && !features) return fail(h, KK_ERR_INVALID_ARG, "features is NULL");
  KK_CUDA(h, h->d_mm.ensure(sizeof(int2) * (size_t)(B->m > 0 ? B->m : 1)), "alloc minmax");
  cudaError_t e = launch_row_features(h->stream, view(A), view(B), h->d_mm.as<int2>(), features,
                                      h->num_sms);
  if (e != cudaSuccess) return cuda_fail(h, e, "features launch");
  return KK_OK;
}

kk_status kk_spgemm_set_predictor(kk_spgemm_handle h, const float* params_host, float quantile) {
  if (!h) return KK_ERR_INVALID_ARG;
  if (!params_host) {
    h->have_pred = false;
    return KK_OK;
  }
  if (!(quantile <= 1.0f)) return fail(h, KK_ERR_INVALID_ARG, "quantile must be <= 1");
  KK_CUDA(h, h->d_params.ensure(sizeof(float) * KK_MLP_NUM_PARAMS), "alloc params");
  KK_CUDA(h, cudaMemcpyAsync(h->d_params.p, params_host, sizeof(float) * KK_MLP_NUM_PARAMS,
                             cudaMemcpyHostToDevice, h->stream), "copy params");
  KK_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  h->have_pred = true;
  h->quantile = quantile;
  return KK_OK;
}

kk_status kk_spgemm_learned_symbolic(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                                     int64_t* c_rowptr, int64_t* nnz_c) {
  if (!h) return KK_ERR_INVALID_ARG;
  kk_status st;
  if ((st = check_csr(h, A, "A", true)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", true)) != KK_OK) return st;
  if (A->n != B->m) return fail(h, KK_ERR_INVALID_ARG, "A.n != B.m");
  if (!c_rowptr || !nnz_c) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr / nnz_c is NULL");
  h->have_symbolic = false;
  h->small = false;
  h->learned_valid = false;
  h->keep = WideKeep{nullptr, nullptr, nullptr, 0, 0};
  h->keep_valid = false;
  const int32_t m = A->m;
  const size_t mm1 = (size_t)(m > 0 ? m : 1);
  const CsrView av = view(A), bv = view(B);
  cudaStream_t s = h->stream;
  Misc* dm = h->d_misc.as<Misc>();
  Misc* hm = static_cast<Misc*>(h->h_pinned);
  int32_t* h_start = reinterpret_cast<int32_t*>(static_cast<char*>(h->h_pinned) + 256);
  int32_t* h_start2 = h_start + 2 * (kMaxBins + 1);

  build_bins(h->opt, false, h->sym_bins);
  build_bins(h->opt, true, h->num_bins);
  const int nbs = (int)h->sym_bins.size(), nbn = (int)h->num_bins.size();
  const int nbl = kLearnedHeavy + 1;
  for (DevBuf* b : {&h->d_sbin, &h->d_nbin, &h->d_lbin, &h->d_plain, &h->d_sball, &h->d_nbin2})
    KK_CUDA(h, b->ensure(mm1), "alloc bins");
  for (DevBuf* b : {&h->d_srows, &h->d_nrows, &h->d_cnt, &h->d_rowlo, &h->d_span, &h->d_cap,
                    &h->d_lrows, &h->d_lrows2})
    KK_CUDA(h, b->ensure(sizeof(int32_t) * mm1), "alloc rows");
  KK_CUDA(h, h->d_flop.ensure(sizeof(long long) * mm1), "alloc flop");
  KK_CUDA(h, h->d_lstat.ensure(sizeof(int2) * mm1), "alloc row statistics");
  KK_CUDA(h, h->d_soff.ensure(sizeof(int64_t) * (mm1 + 1)), "alloc staging offsets");
  KK_CUDA(h, h->d_binstart.ensure(sizeof(int32_t) * 4 * (kMaxBins + 1)), "alloc bins");
  int32_t* sym_start = h->d_binstart.as<int32_t>();
  int32_t* num_start = sym_start + (kMaxBins + 1);
  int32_t* l_start = sym_start + 2 * (kMaxBins + 1);
  int32_t* ln_start = sym_start + 3 * (kMaxBins + 1);

  Misc init{};
  init.sorted = 1;
  KK_CUDA(h, cudaMemcpyAsync(dm, &init, sizeof(Misc), cudaMemcpyHostToDevice, s), "init");
  LaunchCtx ctx = ctx_of(h);
  if (m > 0) {
    timer_begin(h->timer, s, "analyze");
    if ((st = analyze_b(h, bv)) != KK_OK) return st;
    timer_end(h->timer, s);
    // the plain row analysis (flop bound, span, symbolic bin of every row,
    // the B-row statistics the features need), then the classification
    timer_begin(h->timer, s, "learned_analyze");
    const long long avg = (long long)av.nnz / m;
    if (avg <= 8)
      launch_analyze_a<1, 8, true>(h, av, bv, dm, s, h->d_sball.as<uint8_t>(), h->d_lstat.as<int2>());
    else
      launch_analyze_a<4, 8, true>(h, av, bv, dm, s, h->d_sball.as<uint8_t>(), h->d_lstat.as<int2>());
    cudaError_t e = launch_learned_classify(
        ctx, av, bv.n, &dm->sorted, h->opt.use_window, h->opt.structure_cache ? 0 : 1,
        h->have_pred ? h->d_params.as<float>() : nullptr,
        h->quantile, h->have_pred ? 1 : 0, h->d_flop.as<long long>(), h->d_span.as<int32_t>(),
        h->d_lstat.as<int2>(), h->d_lbin.as<uint8_t>(), h->d_cap.as<int32_t>());
    timer_end(h->timer, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "learned analyze");
    timer_begin(h->timer, s, "learned_plan");
    if ((st = run_scan(h, m, h->d_cap.as<int32_t>(), h->d_soff.as<int64_t>(), &dm->grand2, av, nullptr)) != KK_OK)
      return st;
    timer_end(h->timer, s);
    if ((st = run_binning(h, m, h->d_lbin.as<uint8_t>(), nbl, h->d_lrows.as<int32_t>(), l_start)) != KK_OK)
      return st;
  } else {
    KK_CUDA(h, cudaMemsetAsync(l_start, 0, sizeof(int32_t) * (nbl + 1), s), "memset");
  }
  KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
  KK_TRY(readback(h, h_start, l_start, sizeof(int32_t) * (nbl + 1), s));
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
  h->b_sorted = hm->sorted;
  h->stats[6] = (int64_t)hm->total_flop;
  h->stats[7] = hm->sorted;
  accept_bcomp(h, bv, m > 0);
  const long long staging = m > 0 ? hm->grand2 : 0;
  std::vector<int32_t> lstart(h_start, h_start + nbl + 1);
  KK_CUDA(h, h->d_scol.ensure(sizeof(int32_t) * (size_t)(staging > 0 ? staging : 1)), "alloc staging");
  KK_CUDA(h, h->d_sval.ensure(sizeof(double) * (size_t)(staging > 0 ? staging : 1)), "alloc staging");
  // DF32 needs B's rows strictly ascending (its error bound counts at most
  // nnz(A(i,:)) contributions per entry); otherwise the product runs in float64
  const int32_t arith = (h->opt.arith == KK_ARITH_FP64 || !h->b_sorted) ? kArithF64 : kArithDF32;
  h->last_arith = arith;
  if (arith == kArithDF32 && bv.nnz > 0) {
    KK_CUDA(h, h->d_bsplit.ensure(sizeof(float2) * (size_t)bv.nnz), "alloc split");
    KK_CUDA(h, cudaMemsetAsync(&dm->range_bad, 0, sizeof(int32_t), s), "memset");
    timer_begin(h->timer, s, "split_b");
    k_split_values<<<grid_for(bv.nnz, 256, h->num_sms * 8), 256, 0, s>>>(
        bv.nnz, bv.vals, h->d_bsplit.as<float2>(), &dm->range_bad);
    timer_end(h->timer, s);
  }
  int64_t light = 0, heavy = 0;
  BComp bcomp{nullptr, nullptr};
  if (m > 0) {
    int bc_built = 0;
    if ((st = ensure_bcomp(h, bv, &bcomp, &bc_built)) != KK_OK) return st;
  }
  h->cache_valid = false;
  if (m > 0) {
    KK_CUDA(h, cudaMemsetAsync(h->d_cnt.p, 0, sizeof(int32_t) * (size_t)m, s), "memset counts");
    for (int c = 0; c < kLearnedHeavy; ++c) {
      const int n = lstart[c + 1] - lstart[c];
      if (n <= 0) continue;
      light += n;
      const int32_t* lrows = h->d_lrows.as<int32_t>() + lstart[c];
      cudaError_t e =
          c < kOnepassClasses
              ? launch_onepass(ctx, 5 + c, av, bv, h->d_bsplit.as<float2>(), &dm->range_bad, arith,
                               h->d_soff.as<int64_t>(), lrows, n, h->d_scol.as<int32_t>(),
                               h->d_sval.as<double>(), h->d_cnt.as<int32_t>())
              : launch_onepass_table(ctx, av, bv, bcomp, h->d_bsplit.as<float2>(), &dm->range_bad,
                                     arith, h->d_soff.as<int64_t>(), h->d_cap.as<int32_t>(), lrows, n,
                                     h->d_scol.as<int32_t>(), h->d_sval.as<double>(),
                                     h->d_cnt.as<int32_t>());
      if (e != cudaSuccess) return cuda_fail(h, e, "one-pass launch");
    }
    heavy = lstart[kLearnedHeavy + 1] - lstart[kLearnedHeavy];
    // rows left to the plain two-phase path (heavy rows and overflowed rows),
    // with the symbolic bins the analysis gave every row
    cudaError_t e = launch_learned_leftover(ctx, m, h->d_lbin.as<uint8_t>(), h->d_cnt.as<int32_t>(),
                                            h->d_plain.as<uint8_t>(), h->d_sball.as<uint8_t>(),
                                            h->d_sbin.as<uint8_t>());
    if (e != cudaSuccess) return cuda_fail(h, e, "leftover launch");
    if ((st = run_binning(h, m, h->d_sbin.as<uint8_t>(), nbs, h->d_srows.as<int32_t>(), sym_start)) != KK_OK)
      return st;
    KK_TRY(readback(h, h_start, sym_start, sizeof(int32_t) * (nbs + 1), s));
    KK_CUDA(h, cudaStreamSynchronize(s), "sync");
    bool any_win = false;
    int64_t wide_rows = 0;
    for (int b = 0; b < nbs; ++b) {
      if (h->sym_bins[b].tier == kTierWindow && h_start[b + 1] > h_start[b]) any_win = true;
      if (h->sym_bins[b].tier == kTierCta || h->sym_bins[b].tier == kTierDense)
        wide_rows += h_start[b + 1] - h_start[b];
    }
    WinCache wcache;
    if ((st = cache_for_symbolic(h, m, any_win, av, bv, &wcache)) != KK_OK) return st;
    if ((st = keep_for_symbolic(h, m, wide_rows, av, bv)) != KK_OK) return st;
    ctx = ctx_of(h);
    int64_t plain_rows = 0;
    for (int b = 0; b < nbs; ++b) {
      const int cnt = h_start[b + 1] - h_start[b];
      if (cnt <= 0) continue;
      plain_rows += cnt;
      const int32_t* rows = h->d_srows.as<int32_t>() + h_start[b];
      cudaError_t e2 = h->sym_bins[b].tier == kTierWindow
                           ? launch_symbolic_window(ctx, h->sym_bins[b], av, bv, bcomp, rows, cnt,
                                                    h->d_cnt.as<int32_t>(), wcache)
                           : launch_symbolic_bin(ctx, h->sym_bins[b], av, bv, h->b_sorted, rows, cnt,
                                                 h->d_cnt.as<int32_t>());
      if (e2 != cudaSuccess) return cuda_fail(h, e2, "symbolic launch");
    }
    h->stats[12] = light;
    h->stats[13] = plain_rows - heavy;  // overflowed one-pass rows
    h->stats[14] = heavy;
    h->stats[15] = staging;
    timer_begin(h->timer, s, "scan");
    if ((st = run_scan(h, m, h->d_cnt.as<int32_t>(), c_rowptr, &dm->grand, av, h->d_nbin.as<uint8_t>())) != KK_OK)
      return st;
    timer_end(h->timer, s);
    if ((st = run_binning(h, m, h->d_nbin.as<uint8_t>(), nbn, h->d_nrows.as<int32_t>(), num_start)) != KK_OK)
      return st;
    e = launch_mask_bins(ctx, m, h->d_plain.as<uint8_t>(), h->d_nbin.as<uint8_t>(), h->d_nbin2.as<uint8_t>());
    if (e != cudaSuccess) return cuda_fail(h, e, "mask launch");
    if ((st = run_binning(h, m, h->d_nbin2.as<uint8_t>(), nbn, h->d_lrows2.as<int32_t>(), ln_start)) != KK_OK)
      return st;
  } else {
    KK_CUDA(h, cudaMemsetAsync(c_rowptr, 0, sizeof(int64_t), s), "memset rowptr");
    KK_CUDA(h, cudaMemsetAsync(num_start, 0, sizeof(int32_t) * (nbn + 1), s), "memset");
    KK_CUDA(h, cudaMemsetAsync(ln_start, 0, sizeof(int32_t) * (nbn + 1), s), "memset");
  }
  KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
  KK_TRY(readback(h, h_start, num_start, sizeof(int32_t) * (nbn + 1), s));
  KK_TRY(readback(h, h_start2, ln_start, sizeof(int32_t) * (nbn + 1), s));
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
  h->nnz_c = m > 0 ? hm->grand : 0;
  h->num_start.assign(h_start, h_start + nbn + 1);
  h->lnum_start.assign(h_start2, h_start2 + nbn + 1);
  h->stats[24] = (int64_t)hm->kept;
  h->stats[25] = (int64_t)hm->bc_pairs;
  h->am = m;
  h->an = A->n;
  h->bn = B->n;
  h->annz = A->nnz;
  h->bnnz = B->nnz;
  h->have_symbolic = true;
  h->learned_valid = true;
  *nnz_c = h->nnz_c;
  return KK_OK;
}

kk_status kk_spgemm_learned_numeric(kk_spgemm_handle h, const kk_csr* A, const kk_csr* B,
                                    const int64_t* c_rowptr, int32_t* c_colind, double* c_vals) {
  if (!h) return KK_ERR_INVALID_ARG;
  if (!h->learned_valid) return fail(h, KK_ERR_NOT_SYMBOLIC, "learned numeric before learned symbolic");
  kk_status st;
  if ((st = check_csr(h, A, "A", true)) != KK_OK) return st;
  if ((st = check_csr(h, B, "B", true)) != KK_OK) return st;
  if (A->m != h->am || A->n != h->an || B->n != h->bn || A->nnz != h->annz || B->nnz != h->bnnz)
    return fail(h, KK_ERR_STRUCTURE_MISMATCH, "A/B dims or nnz differ from the learned symbolic call");
  if (!c_rowptr) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr is NULL");
  if (h->nnz_c > 0 && (!c_colind || !c_vals)) return fail(h, KK_ERR_INVALID_ARG, "C arrays are NULL");
  if (h->am == 0 || h->nnz_c == 0) return KK_OK;
  const CsrView av = view(A), bv = view(B);
  Misc* dm = h->d_misc.as<Misc>();
  keep_for_numeric(h, av, bv);
  LaunchCtx ctx = ctx_of(h);
  cudaError_t e = launch_copy_staged(ctx, h->am, h->d_lbin.as<uint8_t>(), h->d_plain.as<uint8_t>(),
                                     h->d_soff.as<int64_t>(), c_rowptr, h->d_scol.as<int32_t>(),
                                     h->d_sval.as<double>(), c_colind, c_vals);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy launch");
  const int32_t arith = h->last_arith;
  const float2* bsplit = arith == kArithDF32 ? h->d_bsplit.as<float2>() : nullptr;
  const int nbn = (int)h->num_bins.size();
  bool any_win = false;
  for (int b = 0; b < nbn; ++b)
    if (h->num_bins[b].tier == kTierWindow && h->lnum_start[b + 1] > h->lnum_start[b]) any_win = true;
  BComp bcomp{nullptr, nullptr};
  if (any_win) {
    int built = 0;
    if ((st = ensure_bcomp(h, bv, &bcomp, &built)) != KK_OK) return st;
  }
  WinCacheView wview;
  WinScratch wscratch;
  if ((st = cache_view(h, av, bv, &wview, &wscratch, &ctx)) != KK_OK) return st;
  for (int b = 0; b < nbn; ++b) {
    const int cnt = h->lnum_start[b + 1] - h->lnum_start[b];
    if (cnt <= 0) continue;
    const int32_t* rows = h->d_lrows2.as<int32_t>() + h->lnum_start[b];
    e = h->num_bins[b].tier == kTierWindow
            ? launch_numeric_window(ctx, h->num_bins[b], av, bv, bcomp, wview, wscratch, bsplit, &dm->range_bad,
                                    arith, c_rowptr, rows, cnt, c_colind, c_vals)
            : launch_numeric_bin(ctx, h->num_bins[b], av, bv, h->b_sorted, bsplit, &dm->range_bad, arith,
                                 c_rowptr, rows, cnt, c_colind, c_vals, h->opt.debug_checks);
    if (e != cudaSuccess) return cuda_fail(h, e, "numeric launch");
  }
  return KK_OK;
}

// ---------------------------------------------------------------------------
// Batched form (kk_batched.h)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

unsigned long long fnv1a(const void* p, size_t n, unsigned long long h = 1469598103934665603ull) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

kk_status ensure_pinned(kk_spgemm_handle h, int32_t count) {
  if ((size_t)count + 1 <= h->h_bcap) return KK_OK;
  for (void** p : {&h->h_bdesc, &h->h_bdesc2, &h->h_boff})
    if (*p) {
      cudaFreeHost(*p);
      *p = nullptr;
    }
  const size_t cap = (size_t)count + 1 + (size_t)count / 4;
  KK_CUDA(h, cudaMallocHost(&h->h_bdesc, sizeof(PairDesc) * cap), "pinned descriptors");
  KK_CUDA(h, cudaMallocHost(&h->h_bdesc2, sizeof(PairDesc) * cap), "pinned descriptors");
  KK_CUDA(h, cudaMallocHost(&h->h_boff, sizeof(int64_t) * cap), "pinned offsets");
  h->h_bcap = cap;
  return KK_OK;
}

// Runs `enqueue` directly, or through a CUDA graph captured on the first call
// with `key` and replayed afterwards (non-default streams only).
template <class F>
kk_status run_maybe_graph(kk_spgemm_handle h, bool use_graph, cudaGraphExec_t* exec,
                          unsigned long long* exec_key, unsigned long long key, F enqueue) {
  if (!use_graph) return enqueue();
  if (*exec && *exec_key == key) {
    KK_CUDA(h, cudaGraphLaunch(*exec, h->stream), "graph launch");
    return KK_OK;
  }
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  KernelTimer* saved = h->timer;
  h->timer = nullptr;  // no event records inside a captured graph
  KK_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed), "begin capture");
  kk_status st = enqueue();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  h->timer = saved;
  if (st != KK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *exec = nullptr;
    return cuda_fail(h, e, "graph instantiate");
  }
  *exec_key = key;
  KK_CUDA(h, cudaGraphLaunch(*exec, h->stream), "graph launch");
  return KK_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

kk_csr packed_a(kk_spgemm_handle h) {
  return kk_csr{(int32_t)h->p_RA, (int32_t)h->p_RB, (int32_t)h->p_NA, h->d_pa_rp.as<int32_t>(),
                h->d_pa_ci.as<int32_t>(), h->d_pa_v.as<double>()};
}
kk_csr packed_b(kk_spgemm_handle h) {
  return kk_csr{(int32_t)h->p_RB, h->p_kmax, (int32_t)h->p_NB, h->d_pb_rp.as<int32_t>(),
                h->d_pb_ci.as<int32_t>(), h->d_pb_v.as<double>()};
}

// Packed batch, symbolic: the pairs become one block-diagonal product
// diag(A_k) * diag(B_k) (A's columns shifted to their B rows, B's columns kept
// local), whose rows are C's rows in pair order with local columns: the plain
// two-phase path computes every product with all of its tiers, binning rows of
// all pairs together.  The pair descriptors must already be in hd.
kk_status batched_packed_symbolic(kk_spgemm_handle h, int32_t count, const kk_csr* A, const kk_csr* B,
                                  PairDesc* hd, int64_t* c_rowptr, int64_t* c_offsets,
                                  int64_t* total_nnz) {
  long long RA = 0, NA = 0, RB = 0, NB = 0;
  int32_t kmax = 0;
  std::vector<long long> base(4 * (size_t)(count > 0 ? count : 1));
  for (int k = 0; k < count; ++k) {
    base[4 * k] = RA;
    base[4 * k + 1] = NA;
    base[4 * k + 2] = RB;
    base[4 * k + 3] = NB;
    RA += A[k].m;
    NA += A[k].nnz;
    RB += B[k].m;
    NB += B[k].nnz;
    if (B[k].n > kmax) kmax = B[k].n;
  }
  if (NA > 0x7fffffffll || NB > 0x7fffffffll || RB > 0x7fffffffll)
    return fail(h, KK_ERR_INVALID_ARG, "packed batch exceeds int32 indices; use batched_mode = 1");
  cudaStream_t s = h->stream;
  KK_CUDA(h, h->d_pa_rp.ensure(sizeof(int32_t) * (size_t)(RA + 1)), "alloc packed batch");
  KK_CUDA(h, h->d_pa_ci.ensure(sizeof(int32_t) * (size_t)(NA > 0 ? NA : 1)), "alloc packed batch");
  KK_CUDA(h, h->d_pa_v.ensure(sizeof(double) * (size_t)(NA > 0 ? NA : 1)), "alloc packed batch");
  KK_CUDA(h, h->d_pb_rp.ensure(sizeof(int32_t) * (size_t)(RB + 1)), "alloc packed batch");
  KK_CUDA(h, h->d_pb_ci.ensure(sizeof(int32_t) * (size_t)(NB > 0 ? NB : 1)), "alloc packed batch");
  KK_CUDA(h, h->d_pb_v.ensure(sizeof(double) * (size_t)(NB > 0 ? NB : 1)), "alloc packed batch");
  KK_CUDA(h, h->d_pbase.ensure(sizeof(long long) * base.size()), "alloc packed batch");
  KK_CUDA(h, h->d_bdesc.ensure(sizeof(PairDesc) * (size_t)(count > 0 ? count : 1)), "alloc batch");
  KK_CUDA(h, h->d_boff.ensure(sizeof(int64_t) * ((size_t)count + 1)), "alloc batch");
  PairDesc* dd = h->d_bdesc.as<PairDesc>();
  if (count > 0) {
    KK_CUDA(h, cudaMemcpyAsync(dd, hd, sizeof(PairDesc) * count, cudaMemcpyHostToDevice, s), "upload");
    KK_CUDA(h, cudaMemcpyAsync(h->d_pbase.p, base.data(), sizeof(long long) * base.size(),
                               cudaMemcpyHostToDevice, s), "upload");
  }
  // pageable sources above: staged before return, so base may go out of scope
  KK_CUDA(h, launch_b_pack(s, h->num_sms, count, dd, h->d_pbase.as<long long>(), false,
                           h->d_pa_rp.as<int32_t>(), h->d_pa_ci.as<int32_t>(), h->d_pa_v.as<double>(),
                           h->d_pb_rp.as<int32_t>(), h->d_pb_ci.as<int32_t>(), h->d_pb_v.as<double>(),
                           RA, NA, RB, NB), "pack");
  if (count == 0) {
    KK_CUDA(h, cudaMemsetAsync(h->d_pa_rp.p, 0, sizeof(int32_t), s), "memset");
    KK_CUDA(h, cudaMemsetAsync(h->d_pb_rp.p, 0, sizeof(int32_t), s), "memset");
  }
  h->p_RA = RA;
  h->p_NA = NA;
  h->p_RB = RB;
  h->p_NB = NB;
  h->p_kmax = kmax;
  const kk_csr Ap = packed_a(h), Bp = packed_b(h);
  int64_t nnz = 0;
  h->p_learned = h->opt.batched_learned != 0;
  kk_status st = h->p_learned ? kk_spgemm_learned_symbolic(h, &Ap, &Bp, c_rowptr, &nnz)
                              : kk_spgemm_symbolic(h, &Ap, &Bp, c_rowptr, &nnz);
  if (st != KK_OK) return st;
  KK_CUDA(h, launch_b_offsets(s, count, dd, RA, c_rowptr, h->d_boff.as<int64_t>()), "offsets");
  KK_CUDA(h, cudaMemcpyAsync(h->h_boff, h->d_boff.p, sizeof(int64_t) * ((size_t)count + 1),
                             cudaMemcpyDeviceToHost, s), "readback");
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  const int64_t* off = static_cast<const int64_t*>(h->h_boff);
  if (c_offsets)
    for (int k = 0; k <= count; ++k) c_offsets[k] = off[k];
  h->b_total = nnz;
  h->p_valid = true;
  *total_nnz = nnz;
  return KK_OK;
}

// Packed batch, numeric: values (and, when the caller's arrays moved, the
// structure) packed again, then the plain numeric phase.
kk_status batched_packed_numeric(kk_spgemm_handle h, int32_t count, bool moved, const int64_t* c_rowptr,
                                 int32_t* c_colind, double* c_vals) {
  cudaStream_t s = h->stream;
  PairDesc* dd = h->d_bdesc.as<PairDesc>();
  PairDesc* hd2 = static_cast<PairDesc*>(h->h_bdesc2);
  if (count > 0)
    KK_CUDA(h, cudaMemcpyAsync(dd, hd2, sizeof(PairDesc) * count, cudaMemcpyHostToDevice, s), "upload");
  KK_CUDA(h, launch_b_pack(s, h->num_sms, count, dd, h->d_pbase.as<long long>(), !moved,
                           h->d_pa_rp.as<int32_t>(), h->d_pa_ci.as<int32_t>(), h->d_pa_v.as<double>(),
                           h->d_pb_rp.as<int32_t>(), h->d_pb_ci.as<int32_t>(), h->d_pb_v.as<double>(),
                           h->p_RA, h->p_NA, h->p_RB, h->p_NB), "pack");
  const kk_csr Ap = packed_a(h), Bp = packed_b(h);
  // the first numeric call after a learned symbolic call copies the values the
  // speculative pass computed; later calls recompute from the current values
  const bool fresh = h->p_learned;
  h->p_learned = false;
  return fresh ? kk_spgemm_learned_numeric(h, &Ap, &Bp, c_rowptr, c_colind, c_vals)
               : kk_spgemm_numeric(h, &Ap, &Bp, c_rowptr, c_colind, c_vals);
}

}  // namespace

extern "C" {

kk_status kk_spgemm_batched_symbolic(kk_spgemm_handle h, int32_t count, const kk_csr* A,
                                     const kk_csr* B, int64_t* c_rowptr, int64_t* c_offsets,
                                     int64_t* total_nnz) {
  if (!h) return KK_ERR_INVALID_ARG;
  if (count < 0 || (count > 0 && (!A || !B)) || !total_nnz)
    return fail(h, KK_ERR_INVALID_ARG, "bad batch arguments");
  h->b_valid = false;
  h->have_symbolic = false;
  h->small = false;
  h->learned_valid = false;
  kk_status st;
  long long R = 0, nnzb = 0;
  for (int k = 0; k < count; ++k) {
    if ((st = check_csr(h, &A[k], "A[k]", false)) != KK_OK) return st;
    if ((st = check_csr(h, &B[k], "B[k]", false)) != KK_OK) return st;
    if (A[k].n != B[k].m) return fail(h, KK_ERR_INVALID_ARG, "A[k].n != B[k].m at k=" + std::to_string(k));
    R += A[k].m;
    nnzb += B[k].nnz;
  }
  if (R > 0x7fffffffll) return fail(h, KK_ERR_INVALID_ARG, "batch has more than 2^31-1 rows");
  if (R > 0 && !c_rowptr) return fail(h, KK_ERR_INVALID_ARG, "c_rowptr is NULL");
  if ((st = ensure_pinned(h, count)) != KK_OK) return st;
  PairDesc* hd = static_cast<PairDesc*>(h->h_bdesc);
  long long rb = 0, sb = 0;
  for (int k = 0; k < count; ++k) {
    hd[k] = PairDesc{view(&A[k]), view(&B[k]), rb, sb, 1, 0};
    rb += A[k].m;
    sb += B[k].nnz;
  }
  h->p_valid = false;
  auto packed = [&]() -> kk_status {
    kk_status st3;
    if ((st3 = batched_packed_symbolic(h, count, A, B, hd, c_rowptr, c_offsets, total_nnz)) != KK_OK)
      return st3;
    std::memcpy(h->h_bdesc2, hd, sizeof(PairDesc) * (size_t)count);
    h->b_count = count;
    h->b_R = R;
    h->b_nnzb = nnzb;
    h->b_valid = true;
    return KK_OK;
  };
  if (h->opt.batched_mode != 1) return packed();
  batched_bin_tables(h->b_sym, h->b_num, h->opt.sym_load_pct, h->opt.num_load_pct);
  const size_t R1 = (size_t)(R > 0 ? R : 1);
  const int nblk = (int)((R + kBinRows - 1) / kBinRows);
  const int nblk_scan = (int)((R + kScanRows - 1) / kScanRows);
  const int nbmax = h->b_sym.nb > h->b_num.nb ? h->b_sym.nb : h->b_num.nb;
  KK_CUDA(h, h->d_bdesc.ensure(sizeof(PairDesc) * (size_t)(count > 0 ? count : 1)), "alloc batch");
  for (DevBuf* b : {&h->d_rowpair, &h->d_bsrows, &h->d_bnrows, &h->d_bcnt})
    KK_CUDA(h, b->ensure(sizeof(int32_t) * R1), "alloc batch");
  KK_CUDA(h, h->d_bflop.ensure(sizeof(long long) * R1), "alloc batch");
  KK_CUDA(h, h->d_bsbin.ensure(R1), "alloc batch");
  KK_CUDA(h, h->d_bnbin.ensure(R1), "alloc batch");
  KK_CUDA(h, h->d_btiles.ensure(sizeof(int32_t) * 2 * (kMaxBBins + 1)), "alloc batch");
  KK_CUDA(h, h->d_bstart.ensure(sizeof(int32_t) * 2 * (kMaxBBins + 1)), "alloc batch");
  KK_CUDA(h, h->d_bqueue.ensure(sizeof(int) * 2), "alloc batch");
  KK_CUDA(h, h->d_boff.ensure(sizeof(int64_t) * ((size_t)count + 1)), "alloc batch");
  KK_CUDA(h, h->d_blk.ensure(sizeof(int32_t) * (size_t)nbmax * (size_t)(nblk > 0 ? nblk : 1)), "alloc bins");
  KK_CUDA(h, h->d_scan.ensure(sizeof(long long) * (size_t)(nblk_scan > 0 ? nblk_scan : 1)), "alloc scan");
  if (h->d_span.bytes == 0) KK_CUDA(h, h->d_span.ensure(4), "alloc");
  if (h->d_flop.bytes == 0) KK_CUDA(h, h->d_flop.ensure(8), "alloc");
  cudaStream_t s = h->stream;
  Misc* dm = h->d_misc.as<Misc>();
  Misc* hm = static_cast<Misc*>(h->h_pinned);
  int32_t* sym_start = h->d_bstart.as<int32_t>();
  int32_t* num_start = sym_start + (kMaxBBins + 1);
  PairDesc* dd = h->d_bdesc.as<PairDesc>();
  const CsrView none{0, 0, 0, nullptr, nullptr, nullptr};
  auto enqueue = [&]() -> kk_status {
    LaunchCtx ctx = ctx_of(h);
    kk_status st2;
    if (count > 0)
      KK_CUDA(h, cudaMemcpyAsync(dd, hd, sizeof(PairDesc) * count, cudaMemcpyHostToDevice, s), "upload");
    KK_CUDA(h, cudaMemsetAsync(dm, 0, sizeof(Misc), s), "memset");
    KK_CUDA(h, cudaMemsetAsync(&dm->sorted, 0xFF, sizeof(int32_t), s), "memset");
    if (R > 0) {
      KK_CUDA(h, launch_b_prepare(s, h->num_sms, count, dd, R, h->d_rowpair.as<int32_t>(), &dm->status), "prepare");
      KK_CUDA(h, launch_b_analyze_a(s, h->num_sms, R, dd, h->d_rowpair.as<int32_t>(), h->b_sym,
                                    h->opt.team_vec_min_len, h->d_bflop.as<long long>(), h->d_bsbin.as<uint8_t>(),
                                    &dm->total_flop, &dm->status), "analyze");
      if ((st2 = run_binning(h, (int32_t)R, h->d_bsbin.as<uint8_t>(), h->b_sym.nb, h->d_bsrows.as<int32_t>(),
                             sym_start)) != KK_OK)
        return st2;
      KK_CUDA(h, cudaMemsetAsync(h->d_bcnt.p, 0, sizeof(int32_t) * (size_t)R, s), "memset");
      KK_CUDA(h, launch_b_symbolic(ctx, dd, h->d_rowpair.as<int32_t>(), h->d_bsrows.as<int32_t>(), sym_start,
                                   h->d_btiles.as<int32_t>(), h->b_sym, h->d_bqueue.as<int>(),
                                   h->d_bcnt.as<int32_t>()), "batched symbolic");
      if ((st2 = run_scan(h, (int32_t)R, h->d_bcnt.as<int32_t>(), c_rowptr, &dm->grand, none, nullptr)) != KK_OK)
        return st2;
      KK_CUDA(h, launch_b_nclassify(s, h->num_sms, R, dd, h->d_rowpair.as<int32_t>(), c_rowptr,
                                    h->d_bflop.as<long long>(), h->b_num, h->opt.team_vec_min_len,
                                    h->d_bnbin.as<uint8_t>(), &dm->status), "classify");
      if ((st2 = run_binning(h, (int32_t)R, h->d_bnbin.as<uint8_t>(), h->b_num.nb, h->d_bnrows.as<int32_t>(),
                             num_start)) != KK_OK)
        return st2;
      KK_CUDA(h, launch_b_offsets(s, count, dd, R, c_rowptr, h->d_boff.as<int64_t>()), "offsets");
    } else {
      KK_CUDA(h, cudaMemsetAsync(h->d_boff.p, 0, sizeof(int64_t) * ((size_t)count + 1), s), "memset");
      if (c_rowptr) KK_CUDA(h, cudaMemsetAsync(c_rowptr, 0, sizeof(int64_t), s), "memset");
    }
    KK_CUDA(h, cudaMemcpyAsync(h->h_boff, h->d_boff.p, sizeof(int64_t) * ((size_t)count + 1),
                               cudaMemcpyDeviceToHost, s), "readback");
    if (count > 0)
      KK_CUDA(h, cudaMemcpyAsync(h->h_bdesc2, dd, sizeof(PairDesc) * count, cudaMemcpyDeviceToHost, s),
              "readback");
    KK_TRY(readback(h, hm, dm, sizeof(Misc), s));
    return KK_OK;
  };
  const bool use_graph = h->opt.batched_graph && s != nullptr && s != cudaStreamLegacy &&
                         s != cudaStreamPerThread;
  unsigned long long key = fnv1a(hd, sizeof(PairDesc) * (size_t)count);
  key = fnv1a(&c_rowptr, sizeof(c_rowptr), key);
  key = fnv1a(&count, sizeof(count), key);
  // a batch already found to hold rows beyond the persistent kernels'
  // accumulators goes straight to the block-diagonal form
  if (h->b_overflow && key == h->b_overflow_key) return packed();
  if ((st = run_maybe_graph(h, use_graph, &h->g_sym, &h->g_sym_key, key, enqueue)) != KK_OK) return st;
  KK_CUDA(h, cudaStreamSynchronize(s), "sync");
  if (hm->status == KK_ERR_CAPACITY) {
    // Rows whose flop bound or nnz exceed the persistent kernels' shared-memory
    // accumulators: the whole batch runs as one block-diagonal product through
    // the plain two-phase kernels (every tier, no capacity limit); its numeric
    // calls follow (h->p_valid).
    KK_CUDA(h, cudaMemsetAsync(&dm->status, 0, sizeof(int), s), "memset");
    h->b_overflow = true;
    h->b_overflow_key = key;
    return packed();
  }
  if ((st = check_device_status(h, hm->status)) != KK_OK) return st;
  const int64_t* off = static_cast<const int64_t*>(h->h_boff);
  h->b_total = off[count];
  if (c_offsets)
    for (int k = 0; k <= count; ++k) c_offsets[k] = off[k];
  h->b_count = count;
  h->b_R = R;
  h->b_nnzb = nnzb;
  h->stats[6] = (int64_t)hm->total_flop;
  h->b_valid = true;
  *total_nnz = h->b_total;
  return KK_OK;
}

kk_status kk_spgemm_batched_numeric(kk_spgemm_handle h, int32_t count, const kk_csr* A,
                                    const kk_csr* B, const int64_t* c_rowptr, int32_t* c_colind,
                                    double* c_vals) {
  if (!h) return KK_ERR_INVALID_ARG;
  if (!h->b_valid) return fail(h, KK_ERR_NOT_SYMBOLIC, "batched numeric before batched symbolic");
  if (count != h->b_count || (count > 0 && (!A || !B)))
    return fail(h, KK_ERR_STRUCTURE_MISMATCH, "batch size differs from the batched symbolic call");
  if (h->b_total > 0 && (!c_rowptr || !c_colind || !c_vals))
    return fail(h, KK_ERR_INVALID_ARG, "C arrays are NULL");
  kk_status st;
  PairDesc* hd2 = static_cast<PairDesc*>(h->h_bdesc2);
  bool changed = false;
  for (int k = 0; k < count; ++k) {
    if ((st = check_csr(h, &A[k], "A[k]", true)) != KK_OK) return st;
    if ((st = check_csr(h, &B[k], "B[k]", true)) != KK_OK) return st;
    const PairDesc& d = hd2[k];
    if (A[k].m != d.A.m || A[k].n != d.A.n || A[k].nnz != d.A.nnz || B[k].n != d.B.n || B[k].nnz != d.B.nnz)
      return fail(h, KK_ERR_STRUCTURE_MISMATCH, "pair " + std::to_string(k) + " differs from the symbolic call");
    const CsrView a = view(&A[k]), b = view(&B[k]);
    if (a.rowptr != d.A.rowptr || a.colind != d.A.colind || a.vals != d.A.vals || b.rowptr != d.B.rowptr ||
        b.colind != d.B.colind || b.vals != d.B.vals)
      changed = true;
  }
  bool moved = false;  // index arrays at other addresses (values alone may move freely)
  for (int k = 0; k < count && changed; ++k) {
    const CsrView a = view(&A[k]), b = view(&B[k]);
    if (a.rowptr != hd2[k].A.rowptr || a.colind != hd2[k].A.colind || b.rowptr != hd2[k].B.rowptr ||
        b.colind != hd2[k].B.colind)
      moved = true;
  }
  if (changed) {
    KK_CUDA(h, cudaStreamSynchronize(h->stream), "sync");  // pending uploads read the pinned copy
    for (int k = 0; k < count; ++k) {
      hd2[k].A = view(&A[k]);
      hd2[k].B = view(&B[k]);
    }
  }
  if (h->b_R == 0 || h->b_total == 0) return KK_OK;
  if (h->p_valid) return batched_packed_numeric(h, count, moved, c_rowptr, c_colind, c_vals);
  const int32_t arith = h->opt.arith == KK_ARITH_FP64 ? kArithF64 : kArithDF32;
  h->last_arith = arith;
  KK_CUDA(h, h->d_bsplit2.ensure(sizeof(float2) * (size_t)(h->b_nnzb > 0 ? h->b_nnzb : 1)), "alloc split");
  cudaStream_t s = h->stream;
  PairDesc* dd = h->d_bdesc.as<PairDesc>();
  int32_t* num_start = h->d_bstart.as<int32_t>() + (kMaxBBins + 1);
  auto enqueue = [&]() -> kk_status {
    LaunchCtx ctx = ctx_of(h);
    KK_CUDA(h, cudaMemcpyAsync(dd, hd2, sizeof(PairDesc) * count, cudaMemcpyHostToDevice, s), "upload");
    KK_CUDA(h, launch_b_numeric(ctx, count, dd, h->d_rowpair.as<int32_t>(), h->d_bnrows.as<int32_t>(), num_start,
                                h->d_btiles.as<int32_t>() + (kMaxBBins + 1), h->b_num, h->d_bqueue.as<int>() + 1,
                                arith, h->d_bsplit2.as<float2>(), c_rowptr, c_colind, c_vals),
            "batched numeric");
    return KK_OK;
  };
  const bool use_graph = h->opt.batched_graph && s != nullptr && s != cudaStreamLegacy &&
                         s != cudaStreamPerThread;
  unsigned long long key = fnv1a(hd2, sizeof(PairDesc) * (size_t)count);
  const void* ptrs[3] = {c_rowptr, c_colind, c_vals};
  key = fnv1a(ptrs, sizeof(ptrs), key);
  key = fnv1a(&arith, sizeof(arith), key);
  return run_maybe_graph(h, use_graph, &h->g_num, &h->g_num_key, key, enqueue);
}

kk_status kk_spgemm_sync(kk_spgemm_handle h) {
  if (!h) return KK_ERR_INVALID_ARG;
  Misc* hm = static_cast<Misc*>(h->h_pinned);
  KK_TRY(readback(h, hm, h->d_misc.p, sizeof(Misc), h->stream));
  KK_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  if (h->last_arith == kArithDF32 && hm->range_bad) h->last_arith = kArithF64;
  const int status = hm->status;
  if (status != 0) {
    KK_CUDA(h, cudaMemsetAsync(&h->d_misc.as<Misc>()->status, 0, sizeof(int), h->stream), "memset");
    KK_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  }
  return check_device_status(h, status);
}

kk_status kk_spgemm_kernel_times(kk_spgemm_handle h, int32_t max_kernels, const char** names,
                                 double* total_ms, int64_t* launches, int32_t* count,
                                 int32_t reset) {
  if (!h || !count) return KK_ERR_INVALID_ARG;
  *count = 0;
  if (!h->timer) return KK_OK;
  KK_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  h->timer->collect();
  const int n = (int)h->timer->names.size();
  for (int i = 0; i < n && i < max_kernels; ++i) {
    if (names) names[i] = h->timer->names[i];
    if (total_ms) total_ms[i] = h->timer->total_ms[i];
    if (launches) launches[i] = h->timer->launches[i];
  }
  *count = n;
  if (reset) {
    h->timer->names.clear();
    h->timer->total_ms.clear();
    h->timer->launches.clear();
  }
  return KK_OK;
}

kk_status kk_spgemm_destroy(kk_spgemm_handle h) {
  if (!h) return KK_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  delete h->timer;
  h->d_misc.release();
  h->d_flop.release();
  h->d_sbin.release();
  h->d_nbin.release();
  h->d_srows.release();
  h->d_nrows.release();
  h->d_cnt.release();
  h->d_rowlo.release();
  h->d_span.release();
  h->d_blk.release();
  h->d_binstart.release();
  h->d_scan.release();
  h->d_bsplit.release();
  for (DevBuf* b : {&h->d_params, &h->d_lbin, &h->d_plain, &h->d_cap, &h->d_lstat, &h->d_soff, &h->d_scol,
                    &h->d_sval, &h->d_sball, &h->d_nbin2, &h->d_lrows, &h->d_lrows2, &h->d_mm,
                    &h->d_bdesc, &h->d_rowpair, &h->d_bflop, &h->d_bsbin, &h->d_bnbin, &h->d_bsrows,
                    &h->d_bnrows, &h->d_bcnt, &h->d_btiles, &h->d_bstart, &h->d_bqueue, &h->d_bsplit2,
                    &h->d_boff, &h->d_bc, &h->d_bclen, &h->d_cw, &h->d_cm, &h->d_cn, &h->d_left, &h->d_wbits,
                    &h->d_wslot, &h->d_wnext, &h->d_pa_rp, &h->d_pa_ci, &h->d_pa_v, &h->d_pb_rp, &h->d_pb_ci,
                    &h->d_pb_v, &h->d_pbase})
    b->release();
  for (void* p : {h->h_bdesc, h->h_bdesc2, h->h_boff})
    if (p) cudaFreeHost(p);
  if (h->g_sym) cudaGraphExecDestroy(h->g_sym);
  if (h->g_num) cudaGraphExecDestroy(h->g_num);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  delete h;
  return KK_OK;
}

}  // extern "C"
