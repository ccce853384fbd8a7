// Symbolic phase without any allocation (kk_spgemm_symbolic_noalloc in
// include/kk_noalloc.h).
//
// Every scratch array lives in file-scope device memory of fixed size, so the
// entry point never calls cudaMalloc / cudaFree and needs no handle.  Host
// code may not take these arrays' addresses directly (a host-side reference to
// a __device__ symbol is a stand-in, not a device pointer): on the first call
// on a device the addresses are looked up with cudaGetSymbolAddress while that
// device is current and cached per device.
//
// Work: one CTA per row first checks every index the row will read (A's row
// bounds and columns, the bounds and columns of each referenced B row), then
// counts the distinct columns of C(i,:) with a shared-memory bit vector swept
// over the row's non-empty 32768-column windows (the dense symbolic
// accumulator of the paper's Sec. "Standard SpGEMM Kernel"), writes the count
// to the scratch array, and two scan kernels turn the counts into C's row
// pointers (scratch block sums).
#include <mutex>

#include "kk_device.cuh"
#include "kk_internal.h"
#include "kk_noalloc.h"

namespace kk {
namespace {

constexpr int kNaBlock = 256;
constexpr int kNaChunkBits = 32768;   // bit vector of 4 KB in static shared memory
constexpr int kNaScanRows = 2048;     // rows per scan block
constexpr int kNaMaxBlocks = (KK_NOALLOC_MAX_ROWS + kNaScanRows - 1) / kNaScanRows;

// Scratch shared by every call on this device (held until the process exits).
static __device__ __align__(256) int32_t g_na_counts[KK_NOALLOC_MAX_ROWS];
static __device__ __align__(256) long long g_na_blocks[kNaMaxBlocks + 1];
static __device__ __align__(256) int g_na_status[4];

struct NaScratch {
  int32_t* counts = nullptr;
  long long* blocks = nullptr;
  int* status = nullptr;
};

std::mutex g_na_mutex;
NaScratch g_na_dev[64];
bool g_na_ready[64] = {false};

// Block-wide min / max of (l, h) through the per-warp slots red_lo / red_hi.
__device__ void na_block_minmax(int* red_lo, int* red_hi, int& l, int& h) {
  for (int o = 16; o > 0; o >>= 1) {
    l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
    h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red_lo[warp] = l;
    red_hi[warp] = h;
  }
  __syncthreads();
  l = 0x7fffffff;
  h = -1;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    l = min(l, red_lo[w]);
    h = max(h, red_hi[w]);
  }
  __syncthreads();
}

// Checks every index row i's products read, before any of them is used to
// index: A's row bounds (A.rowptr[0] must be 0), A's columns inside B's rows,
// the bounds of each referenced B row inside B's entries, and B's columns
// inside [0, B.n).  Returns true (for the whole block) if any check failed.
__device__ bool na_row_bad(const CsrView& A, const CsrView& B, int i, int pa, int pe) {
  int bad = 0;
  if (i == 0 && threadIdx.x == 0 && A.rowptr[0] != 0) bad = 1;
  if (pa < 0 || pe < pa || pe > A.nnz) bad = 1;
  if (__syncthreads_or(bad)) return true;
  for (int p = pa + threadIdx.x; p < pe; p += blockDim.x) {
    const int j = A.colind[p];
    if ((unsigned)j >= (unsigned)B.m) {
      bad = 1;
      continue;
    }
    const int bs = B.rowptr[j], be = B.rowptr[j + 1];
    if (bs < 0 || be < bs || be > B.nnz) bad = 1;
  }
  if (__syncthreads_or(bad)) return true;
  // every referenced B row is now known to lie inside B's entries
  for (int p = pa + threadIdx.x; p < pe; p += blockDim.x) {
    const int j = A.colind[p];
    for (int q = B.rowptr[j]; q < B.rowptr[j + 1]; ++q)
      if ((unsigned)B.colind[q] >= (unsigned)B.n) bad = 1;
  }
  return __syncthreads_or(bad) != 0;
}

__global__ void __launch_bounds__(kNaBlock)
k_na_count(CsrView A, CsrView B, int32_t* __restrict__ counts, int* __restrict__ status) {
  __shared__ uint32_t bits[kNaChunkBits / 32];
  __shared__ int red_lo[kNaBlock / 32], red_hi[kNaBlock / 32], red_c[kNaBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = blockIdx.x; i < A.m; i += gridDim.x) {
    const int pa = A.rowptr[i], pe = A.rowptr[i + 1];
    if (na_row_bad(A, B, i, pa, pe)) {
      if (threadIdx.x == 0) {
        atomicCAS(status, 0, KK_ERR_BAD_INDEX);
        counts[i] = 0;
      }
      continue;
    }
    // smallest column of the row's products (the first window starts there)
    int c0 = 0x7fffffff, unused = -1;
    for (int p = pa + threadIdx.x; p < pe; p += blockDim.x) {
      const int j = A.colind[p];
      for (int q = B.rowptr[j]; q < B.rowptr[j + 1]; ++q) c0 = min(c0, B.colind[q]);
    }
    na_block_minmax(red_lo, red_hi, c0, unused);
    int total = 0;
    // One pass per non-empty window of kNaChunkBits columns: a pass counts the
    // columns in [c0, c0 + kNaChunkBits) and finds the smallest column past
    // the window, where the next pass starts (empty windows are skipped, so
    // the number of passes is at most the number of products).
    while (c0 != 0x7fffffff) {
      for (int w = threadIdx.x; w < kNaChunkBits / 32; w += blockDim.x) bits[w] = 0u;
      __syncthreads();
      int next = 0x7fffffff, unused2 = -1;
      for (int p = pa + threadIdx.x; p < pe; p += blockDim.x) {
        const int j = A.colind[p];
        for (int q = B.rowptr[j]; q < B.rowptr[j + 1]; ++q) {
          const int c = B.colind[q];
          const long long o = (long long)c - c0;
          if (o >= 0 && o < kNaChunkBits) atomicOr(&bits[o >> 5], 1u << (o & 31));
          else if (o >= kNaChunkBits) next = min(next, c);
        }
      }
      __syncthreads();
      int c = 0;
      for (int w = threadIdx.x; w < kNaChunkBits / 32; w += blockDim.x) c += __popc(bits[w]);
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      if (lane == 0) red_c[warp] = c;
      __syncthreads();
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += red_c[w];
      __syncthreads();
      na_block_minmax(red_lo, red_hi, next, unused2);
      c0 = next;
    }
    if (threadIdx.x == 0) counts[i] = total;
  }
}

__global__ void __launch_bounds__(kNaBlock)
k_na_block_sums(int32_t m, const int32_t* __restrict__ counts, long long* __restrict__ blocks) {
  __shared__ long long red[kNaBlock / 32];
  long long s = 0;
  const long long base = (long long)blockIdx.x * kNaScanRows;
  for (int t = threadIdx.x; t < kNaScanRows; t += blockDim.x)
    if (base + t < m) s += counts[base + t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kNaBlock / 32; ++w) t += red[w];
    blocks[blockIdx.x] = t;
  }
}

// One CTA: exclusive scan of the block sums (sequential over at most
// kNaMaxBlocks entries by one thread; small), then every block expands its rows.
__global__ void k_na_scan_blocks(int32_t nblk, long long* __restrict__ blocks) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long run = 0;
  for (int b = 0; b < nblk; ++b) {
    const long long v = blocks[b];
    blocks[b] = run;
    run += v;
  }
  blocks[nblk] = run;
}

__global__ void __launch_bounds__(kNaBlock)
k_na_rowptr(int32_t m, const int32_t* __restrict__ counts, const long long* __restrict__ blocks,
            int32_t nblk, int64_t* __restrict__ rowptr) {
  // one warp walks the block's rows sequentially in 32-row slices
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const long long base = (long long)blockIdx.x * kNaScanRows;
  long long run = blocks[blockIdx.x];
  for (int t0 = 0; t0 < kNaScanRows; t0 += 32) {
    const long long r = base + t0 + lane;
    const long long v = r < m ? counts[r] : 0;
    long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (r < m) rowptr[r] = run + incl - v;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (blockIdx.x == nblk - 1 && lane == 0) rowptr[m] = blocks[nblk];
}

kk_status na_setup(NaScratch& out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KK_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ready[dev]) {
    NaScratch s;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&s.counts), g_na_counts) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.blocks), g_na_blocks) != cudaSuccess ||
        cudaGetSymbolAddress(reinterpret_cast<void**>(&s.status), g_na_status) != cudaSuccess) {
      cudaGetLastError();
      return KK_ERR_CUDA;
    }
    g_na_dev[dev] = s;
    g_na_ready[dev] = true;
  }
  out = g_na_dev[dev];
  return KK_OK;
}

}  // namespace
}  // namespace kk

using namespace kk;

extern "C" kk_status kk_spgemm_symbolic_noalloc(const kk_csr* A, const kk_csr* B, int64_t* c_rowptr,
                                                int64_t* nnz_c, void* cuda_stream) {
  if (!A || !B || !c_rowptr || !nnz_c) return KK_ERR_INVALID_ARG;
  if (A->m < 0 || A->n < 0 || A->nnz < 0 || B->m < 0 || B->n < 0 || B->nnz < 0) return KK_ERR_INVALID_ARG;
  if (!A->rowptr || !B->rowptr || (A->nnz > 0 && !A->colind) || (B->nnz > 0 && !B->colind))
    return KK_ERR_INVALID_ARG;
  if (A->n != B->m) return KK_ERR_INVALID_ARG;
  if (A->m > KK_NOALLOC_MAX_ROWS) return KK_ERR_CAPACITY;
  NaScratch sc;
  kk_status st = na_setup(sc);
  if (st != KK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int32_t m = A->m;
  const CsrView av{A->m, A->n, A->nnz, A->rowptr, A->colind, A->vals};
  const CsrView bv{B->m, B->n, B->nnz, B->rowptr, B->colind, B->vals};
  if (cudaMemsetAsync(sc.status, 0, sizeof(int) * 4, s) != cudaSuccess) return KK_ERR_CUDA;
  if (m == 0) {
    if (cudaMemsetAsync(c_rowptr, 0, sizeof(int64_t), s) != cudaSuccess) return KK_ERR_CUDA;
    *nnz_c = 0;
    return cudaStreamSynchronize(s) == cudaSuccess ? KK_OK : KK_ERR_CUDA;
  }
  const int nblk = (m + kNaScanRows - 1) / kNaScanRows;
  int grid = m < 65535 ? m : 65535;
  k_na_count<<<grid, kNaBlock, 0, s>>>(av, bv, sc.counts, sc.status);
  k_na_block_sums<<<nblk, kNaBlock, 0, s>>>(m, sc.counts, sc.blocks);
  k_na_scan_blocks<<<1, 32, 0, s>>>(nblk, sc.blocks);
  k_na_rowptr<<<nblk, kNaBlock, 0, s>>>(m, sc.counts, sc.blocks, nblk, c_rowptr);
  if (cudaGetLastError() != cudaSuccess) return KK_ERR_CUDA;
  int64_t total = 0;
  int status = 0;
  if (cudaMemcpyAsync(&total, c_rowptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&status, sc.status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return KK_ERR_CUDA;
  if (status != 0) return static_cast<kk_status>(status);
  *nnz_c = total;
  return KK_OK;
}
