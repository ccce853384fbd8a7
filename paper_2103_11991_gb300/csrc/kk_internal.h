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

// Bit vectors of wide-tier rows kept by the symbolic phase for the numeric
// phase of the same arrays: rows whose nnz(C(i,:)) exceeds min_cnt (their
// values go to C with atomics) get a slot of `words` u32 when one is left.
struct WideKeep {
  uint32_t* bits;     // max_slots slots of `words` words
  int32_t* slot;      // per row: slot or -1
  int32_t* next;      // slot counter
  int32_t max_slots;  // 0: nothing kept / nothing to use
  int32_t min_cnt;
};

struct LaunchCtx {
  cudaStream_t stream;
  KernelTimer* timer;  // may be null
  int* status;         // device status word
  int num_sms;
  int max_smem_optin;
  const int32_t* row_lo;  // first column of each row's span window (window tier)
  const long long* flop;  // flop bound of each row (wide tier)
  WideKeep keep;          // kept wide-tier bit vectors (wide tier)
  int debug_checks;       // options.debug_checks
  int stage_long_rows;    // options.stage_long_rows (wide symbolic: bulk-copy staging)
  // structure fingerprints of the index arrays at the symbolic call ([0]) and
  // at this numeric call ([1]); null when the kept structure is not in use
  const unsigned long long* fingerprint;
  // 1: the window tier's rows of at most kWindowMaxNnz columns (the
  // kept-structure value pass and its rebuild) run in float64 whatever the
  // call's arithmetic (options.arith = AUTO: on GB300 native float64 measured
  // faster there, 1.91 ms against 2.42 for the 27-point value pass)
  int kept_f64;
};

struct CsrView {
  int32_t m, n, nnz;
  const int32_t* rowptr;
  const int32_t* colind;
  const double* vals;
  // Jacobi-fused numeric phase (null otherwise): row i of A enters the product
  // as jac_s[i] * A(i,:) plus 1 at entry jac_p[i] (the row's first diagonal
  // entry), i.e. as row i of I - omega D^-1 A, without a scaled copy of A.  The
  // thread tier forms s_i and that position from the row itself with
  // jac_omega; the other tiers' rows get them from a row-scale kernel.
  const double* jac_s;
  const int32_t* jac_p;
  double jac_omega;
};

#ifdef __CUDACC__
// Row i's Jacobi scaling (loaded once per row): on = false for the plain product.
struct ARowScale {
  double s;
  int p;
  bool on;
};
__device__ __forceinline__ ARowScale a_row_scale(const CsrView& A, int i) {
  ARowScale r{1.0, -1, A.jac_s != nullptr};
  if (r.on) {
    r.s = A.jac_s[i];
    r.p = A.jac_p[i];
  }
  return r;
}
// Value of A's entry p as the numeric phase multiplies it: the stored value v,
// or for the Jacobi-fused product s_i * v (+ 1 at the row's first diagonal
// entry), formed once per A entry as it is loaded.
__device__ __forceinline__ double a_scaled(const ARowScale& r, int p, double v) {
  return r.on ? (p == r.p ? fma(r.s, v, 1.0) : r.s * v) : v;
}
__device__ __forceinline__ double a_value(const CsrView& A, int i, int p) {
  return a_scaled(a_row_scale(A, i), p, A.vals[p]);
}
#endif

// Accumulator tiers.  The thread tier counts as the team tier in statistics.
enum Tier : int32_t { kTierTeam = 0, kTierCta = 1, kTierDense = 2, kTierWindow = 3, kTierThread = 4 };
__host__ __device__ constexpr int32_t stat_tier(int32_t t) { return t == kTierThread ? kTierTeam : t; }

// Thread tier (kk_thread.cu): one thread per row, accumulator in registers.
constexpr int kThreadSymMax = 16;     // symbolic rows: flop bound <= this
constexpr int kThreadNumMax = 8;      // numeric rows: nnz(C(i,:)) <= this ...
constexpr int kThreadNumMaxFlop = 16; // ... and flop bound <= this
// Small products (kk_small.cu): one launch per phase, a thread per row, for A
// with at most options.small_max_rows rows (at most kSmallMaxRowsCap), C rows
// of at most kSmallN columns, tried when A's rows average at most
// kSmallMaxMeanFlop products.
constexpr int kSmallThreads = 256;     // symbolic CTA
constexpr int kSmallNumThreads = 64;   // numeric CTA (more CTAs for a few thousand rows)
constexpr int kSmallMaxRowsCap = 8192;
constexpr int kSmallN = 16;
constexpr int kSmallMaxMeanFlop = 32;

// Window tier: a row whose columns of C all lie in [row_lo, row_lo + W) gets a
// dense bit vector of W bits (plus per-word ranks in the numeric phase).
constexpr int kNumWindowClasses = 5;
constexpr int32_t kWindowBits[kNumWindowClasses] = {4096, 12288, 24576, 40960, 65536};
__host__ __device__ constexpr int32_t window_bits(int w) {
  return w == 0 ? 4096 : w == 1 ? 12288 : w == 2 ? 24576 : w == 3 ? 40960 : 65536;
}
constexpr int32_t kWindowMaxNnz = 256;   // numeric window rows: nnz(C(i,:)) <= this
constexpr int32_t kWindowMaxNnzWide = 1024;  // ... or this, in the large-value window bins
constexpr int32_t kWindowFlopRatio = 128;  // symbolic window used only when W <= ratio * flop
constexpr int32_t kWindowFlopRatioNum = 512;  // large-value numeric window bins
// Large-value numeric window bins (nnz(C(i,:)) in (kWindowMaxNnz, kWindowMaxNnzWide]),
// with value arrays of kWindowMidNnz or kWindowMaxNnzWide slots (the smaller
// array leaves room for more warps per SM).
constexpr int32_t kWindowMidNnz = 512;
constexpr int kNumWideWindowClasses = 3;
constexpr int32_t kWideWindowBits[kNumWideWindowClasses] = {24576, 40960, 65536};
constexpr int kMaxWindowBins = kNumWindowClasses + 2 * kNumWideWindowClasses;

// Compressed B (the paper's B_C): row j of B as (column >> 5, 32-bit column
// mask) pairs in column order, stored at B's own row offsets
// bc[B.rowptr[j] .. B.rowptr[j] + len[j]).  Built only for sorted B.
struct BComp {
  const int2* bc;
  const int32_t* len;
};

// Per-row structure kept by the symbolic window kernel for the numeric phase
// of the same A and B: the row's non-empty window words (index relative to
// the word of row_lo, at most kCacheWords) and their bits; n[i] = number of
// words, -1 if the row has no kept structure.
constexpr int kCacheWords = 64;
struct WinCache {
  uint16_t* w;
  uint32_t* m;
  int32_t* n;
  unsigned long long* kept;  // += rows whose structure was kept
};
struct WinCacheView {
  const uint16_t* w;
  const uint32_t* m;
  const int32_t* n;
};
// Scratch of the numeric window launch: rows left to the window kernel by the
// kept-structure kernel (count first, then the rows).
struct WinScratch {
  int32_t* rows;
  int32_t* count;
};
// Analysis of B (kk_window.cu): clears *sorted_flag unless every row is
// strictly ascending, sets KK_ERR_BAD_INDEX on out-of-range structure, and,
// when bc is non-null, writes the compressed rows (pairs counted into *pairs).
// Sparse matrix addition (kk_spadd.cu): symbolic counts and the slots of A's
// and B's entries in C (rows of more than 256 combined entries go through
// long_rows / *long_count, zeroed by the caller); numeric adds into C's values
// (zeroed by the caller) and writes C's columns.
cudaError_t launch_spadd_symbolic(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, int32_t* cnt,
                                  int32_t* apos, int32_t* bpos, int32_t* long_rows,
                                  int32_t* long_count);
cudaError_t launch_spadd_numeric(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, double alpha,
                                 double beta, const int64_t* c_rowptr, const int32_t* apos,
                                 const int32_t* bpos, int32_t* c_colind, double* c_vals);

// Numeric phase of window rows with kept structure (kk_kept.cu); rows without
// it are appended to left_rows / *left_count for the rebuild kernel.
cudaError_t launch_num_kept(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                            const WinCacheView& cache, const float2* b_split, const int32_t* b_range_bad,
                            int32_t arith, const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                            int32_t* c_colind, double* c_vals, int32_t* left_rows, int32_t* left_count);

cudaError_t launch_analyze_b(const LaunchCtx& ctx, const CsrView& B, int32_t* sorted_flag,
                             int2* bc, int32_t* len, unsigned long long* pairs);

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

// Wide tier (kk_wide.cu): CTA-per-row bit vector over all k columns, used for
// the CTA and dense bins when it fits in shared memory.
bool wide_symbolic_fits(const LaunchCtx& ctx, int32_t k);
int32_t wide_word_count(int32_t k);                           // words of a k-bit vector
int32_t wide_keep_min_cnt(const LaunchCtx& ctx, int32_t k);  // rows above this go to C by atomics
bool wide_numeric_fits(const LaunchCtx& ctx, int32_t k);
cudaError_t launch_symbolic_wide(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                 const long long* flop, const int32_t* rows, int32_t nrows,
                                 int32_t* cnt);
cudaError_t launch_numeric_wide(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                int32_t* c_colind, double* c_vals);

cudaError_t launch_symbolic_thread(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                   const int32_t* rows, int32_t nrows, int32_t* cnt);
cudaError_t launch_small_symbolic(const LaunchCtx& ctx, const CsrView& A, const CsrView& B, int64_t* c_rowptr,
                                  int32_t* cnt, int32_t* flags, long long* out);
cudaError_t launch_small_numeric(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                 const int64_t* c_rowptr, int32_t* c_colind, double* c_vals);
cudaError_t launch_numeric_thread(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                  const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                  int32_t* c_colind, double* c_vals);

// Window-tier launches (kk_window.cu).
cudaError_t launch_symbolic_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                   const CsrView& B, const BComp& bcomp, const int32_t* rows,
                                   int32_t nrows, int32_t* cnt, const WinCache& cache);
cudaError_t launch_numeric_window(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                                  const CsrView& B, const BComp& bcomp, const WinCacheView& cache,
                                  const WinScratch& scratch, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith,
                                  const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                                  int32_t* c_colind, double* c_vals);

// Speculative one-pass (learned form) over rows whose predicted table is
// 2^log2s slots (log2s in 5..9); see k_num_warp_vec<LOG2S, true>.
cudaError_t launch_onepass(const LaunchCtx& ctx, int32_t log2s, const CsrView& A, const CsrView& B,
                           const float2* b_split, const int32_t* b_range_bad, int32_t arith,
                           const int64_t* soff, const int32_t* rows, int32_t nrows, int32_t* scol,
                           double* sval, int32_t* cnt_out);

// Learned form (kk_learned.cu).  Rows predicted to need at most
// 16 << (kOnepassClasses - 1) entries take the speculative one-pass.
constexpr int kOnepassClasses = 5;
// Learned bins: [0, kOnepassClasses) hash one-pass by capacity class,
// [kOnepassClasses, kLearnedHeavy) window one-pass by window class,
// kLearnedHeavy = plain path.
constexpr int kLearnedHeavy = kOnepassClasses + kNumWindowClasses;
cudaError_t launch_onepass_window(const LaunchCtx& ctx, int32_t wclass, const CsrView& A,
                                  const CsrView& B, const BComp& bcomp, const float2* b_split,
                                  const int32_t* b_range_bad, int32_t arith, const int64_t* soff,
                                  const int32_t* cap, const int32_t* rows, int32_t nrows,
                                  int32_t* scol, double* sval, int32_t* cnt_out);
// Speculative one-pass for window rows through a word table (kk_onepass.cu).
cudaError_t launch_onepass_table(const LaunchCtx& ctx, const CsrView& A, const CsrView& B,
                                 const BComp& bcomp, const float2* b_split,
                                 const int32_t* b_range_bad, int32_t arith, const int64_t* soff,
                                 const int32_t* cap, const int32_t* rows, int32_t nrows,
                                 int32_t* scol, double* sval, int32_t* cnt_out);
cudaError_t launch_learned_classify(const LaunchCtx& ctx, const CsrView& A, int32_t bn,
                                    const int32_t* b_sorted, int32_t use_window, int32_t window_onepass,
                                    const float* params,
                                    float quantile, int32_t use_pred, const long long* flop,
                                    const int32_t* row_span, const int2* stat, uint8_t* lbin, int32_t* cap);
cudaError_t launch_learned_leftover(const LaunchCtx& ctx, int32_t m, const uint8_t* lbin,
                                    const int32_t* cnt, uint8_t* plain, const uint8_t* sbin_all,
                                    uint8_t* sbin);
cudaError_t launch_mask_bins(const LaunchCtx& ctx, int32_t m, const uint8_t* plain,
                             const uint8_t* nbin, uint8_t* out);
cudaError_t launch_copy_staged(const LaunchCtx& ctx, int32_t m, const uint8_t* lbin,
                               const uint8_t* plain, const int64_t* soff, const int64_t* rowptr,
                               const int32_t* scol, const double* sval, int32_t* ccol,
                               double* cval);

// Batched form (kk_batched.cu).
struct PairDesc {
  CsrView A, B;
  long long row_base;    // first global row of this pair
  long long split_base;  // first DF32 pair of B's values in the split buffer
  int32_t b_sorted;      // set on the device
  int32_t range_bad;     // set on the device (values outside the DF32 window)
};
constexpr int kMaxBBins = 24;
struct BBinTable {
  int32_t nb;
  int32_t kind[kMaxBBins];   // 0 warp, 1 CTA
  int32_t log2s[kMaxBBins];
  int32_t flat[kMaxBBins];
  long long hi[kMaxBBins];
};
void batched_bin_tables(BBinTable& sym, BBinTable& num, int sym_load_pct, int num_load_pct);
// Packed batch (block-diagonal A and B for the plain kernels); base holds per
// pair the A rows, A entries, B rows and B entries that precede it.
cudaError_t launch_b_pack(cudaStream_t s, int num_sms, int32_t count, const PairDesc* d,
                          const long long* base, bool vals_only, int32_t* pa_rp, int32_t* pa_ci,
                          double* pa_v, int32_t* pb_rp, int32_t* pb_ci, double* pb_v, long long RA,
                          long long NA, long long RB, long long NB);
cudaError_t launch_b_prepare(cudaStream_t s, int num_sms, int32_t count, PairDesc* d, long long R,
                             int32_t* row_pair, int* status);
cudaError_t launch_b_analyze_a(cudaStream_t s, int num_sms, long long R, const PairDesc* d,
                               const int32_t* row_pair, const BBinTable& tab, int32_t vec_min_len,
                               long long* flop, uint8_t* bin, unsigned long long* total_flop, int* status);
cudaError_t launch_b_nclassify(cudaStream_t s, int num_sms, long long R, const PairDesc* d,
                               const int32_t* row_pair, const int64_t* rowptr, const long long* flop,
                               const BBinTable& tab, int32_t vec_min_len, uint8_t* bin, int* status);
cudaError_t launch_b_symbolic(const LaunchCtx& ctx, const PairDesc* d, const int32_t* row_pair,
                              const int32_t* rows, const int32_t* bin_start, int32_t* tile_prefix,
                              const BBinTable& tab, int* queue, int32_t* cnt);
cudaError_t launch_b_numeric(const LaunchCtx& ctx, int32_t count, PairDesc* d, const int32_t* row_pair,
                             const int32_t* rows, const int32_t* bin_start, int32_t* tile_prefix,
                             const BBinTable& tab, int* queue, int32_t arith, float2* split,
                             const int64_t* rowptr, int32_t* ccol, double* cval);
cudaError_t launch_b_offsets(cudaStream_t s, int32_t count, const PairDesc* d, long long R,
                             const int64_t* rowptr, int64_t* off);

// Row features (kk_mlp.cu); mm is scratch int2[B.m].
cudaError_t launch_row_features(cudaStream_t s, const CsrView& A, const CsrView& B, int2* mm,
                                float* feat, int num_sms);

// Shared-memory bytes a bin's kernel needs per CTA (0 if it does not fit).
size_t symbolic_smem_bytes(const BinSpec& bin);
size_t numeric_smem_bytes(const BinSpec& bin);

}  // namespace kk
