// Internal host-side interfaces between the translation units of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kk_spgemm.h"

namespace kk {

// Per-kernel CUDA-event timer (enabled by options.timing).
struct KernelTimer;
void timer_begin(KernelTimer* t, cudaStream_t s, const char* name);
void timer_end(KernelTimer* t, cudaStream_t s);

struct LaunchCtx {
  cudaStream_t stream;
  KernelTimer* timer;  // may be null
  int* status;         // device status word
  int num_sms;
  int max_smem_optin;
  const int32_t* row_lo;  // first column of each row's span window (window tier)
};

struct CsrView {
  int32_t m, n, nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* vals;
};

// Accumulator tiers.
enum Tier : int32_t { kTierTeam = 0, kTierCta = 1, kTierDense = 2, kTierWindow = 3 };

// Window tier: a row whose columns of C all lie in [row_lo, row_lo + W) gets a
// dense bit vector of W bits (plus per-word ranks in the numeric phase).
constexpr int kNumWindowClasses = 4;
constexpr int32_t kWindowBits[kNumWindowClasses] = {4096, 16384, 49152, 65536};
constexpr int32_t kWindowMaxNnz = 256;   // numeric window rows: nnz(C(i,:)) <= this
constexpr int32_t kWindowFlopRatio = 128;  // window used only when W <= ratio * flop

// One bin of rows: its tier and the accumulator geometry.
struct BinSpec {
  int32_t tier;
  int32_t team;   // lanes per row (team tier); threads per CTA otherwise
  int32_t slots;  // hash slots (team / CTA tiers); chunk width in columns (dense)
  int32_t flat;   // 1: lanes walk the flattened (A entry, B entry) products
  int64_t lo, hi; // bin range of the binning quantity (flop or nnz), inclusive
};

// Arithmetic mode for the numeric kernels.
enum ArithMode : int32_t { kArithF64 = 1, kArithDF32 = 2 };

// Symbolic launch: rows[0..nrows) of A (a device array) get cnt[i] = nnz(C(i,:)).
cudaError_t launch_symbolic_bin(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                const CsrView& B, int32_t b_sorted, const int32_t* rows,
                                int32_t nrows, int32_t* cnt);

// Numeric launch.  b_split: B's values pre-split into DF32 pairs (float2), used
// when arith == kArithDF32 and *b_range_bad == 0 (read on the device).
cudaError_t launch_numeric_bin(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                               const CsrView& B, int32_t b_sorted, const float2* b_split,
                               const int32_t* b_range_bad, int32_t arith,
                               const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                               int32_t* c_colind, double* c_vals, int32_t debug_checks);

// Window-tier launches (kk_window.cu).
cudaError_t launch_symbolic_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                   const CsrView& B, const int32_t* rows, int32_t nrows,
                                   int32_t* cnt);
cudaError_t launch_numeric_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                  const CsrView& B, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith,
                                  const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                  int32_t* c_colind, double* c_vals);

// Shared-memory bytes a bin's kernel needs per CTA (0 if it does not fit).
size_t symbolic_smem_bytes(const BinSpec& bin);
size_t numeric_smem_bytes(const BinSpec& bin);

}  // namespace kk
