// Device-side helpers shared by the SpGEMM kernels: team primitives, the hash
// used by the shared-memory accumulators, the device status word, and the
// float32-pair ("DF32") arithmetic that emulates float64 accumulation on the
// FP32 pipe (GB300 issues FP32 FMAs ~70x faster than FP64 FMAs).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "kk_spgemm.h"

namespace kk {

constexpr int32_t kEmptyKey = -1;
// Upper bound on CAS retries of one atomic accumulator update; a loop that runs
// out records KK_ERR_TIMEOUT instead of spinning forever.
constexpr int kCasRetryLimit = 1 << 20;

__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Teams: TEAM consecutive lanes of a warp (TEAM in 1..32, a power of two).
// ---------------------------------------------------------------------------
template <int TEAM>
__device__ __forceinline__ unsigned team_mask() {
  if constexpr (TEAM == 32) {
    return 0xffffffffu;
  } else {
    const int lane = threadIdx.x & 31;
    return ((1u << TEAM) - 1u) << (lane & ~(TEAM - 1));
  }
}

template <int TEAM>
__device__ __forceinline__ int team_sum(int v, unsigned mask) {
#pragma unroll
  for (int o = TEAM / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, TEAM);
  return v;
}

template <int TEAM>
__device__ __forceinline__ int team_inclusive_scan(int v, int tl, unsigned mask) {
#pragma unroll
  for (int o = 1; o < TEAM; o <<= 1) {
    int u = __shfl_up_sync(mask, v, o, TEAM);
    if (tl >= o) v += u;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Multiplicative hashing of a column index into 2^log2s slots (Knuth).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t hash_slot(int32_t key, int log2s) {
  return ((uint32_t)key * 2654435761u) >> (32 - log2s);
}

// Insert key into an open-addressing set of 2^log2s int32 slots (linear probing).
// Returns 1 if this call inserted it, 0 if it was present.  Probing is bounded
// by the table size; a full table records KK_ERR_CAPACITY.
__device__ __forceinline__ int set_insert(int* tab, int32_t key, int log2s, int* status) {
  const uint32_t mask = (1u << log2s) - 1u;
  uint32_t h = hash_slot(key, log2s);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int cur = tab[h];
    if (cur == key) return 0;
    if (cur == kEmptyKey) {
      int old = atomicCAS(&tab[h], kEmptyKey, key);
      if (old == kEmptyKey) return 1;
      if (old == key) return 0;
    }
    h = (h + 1) & mask;
  }
  set_status(status, KK_ERR_CAPACITY);
  return 0;
}

// Find-or-insert key; returns its slot, or -1 (and KK_ERR_CAPACITY) if full.
__device__ __forceinline__ int map_slot(int* keys, int32_t key, int log2s, int* status) {
  const uint32_t mask = (1u << log2s) - 1u;
  uint32_t h = hash_slot(key, log2s);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int cur = keys[h];
    if (cur == key) return (int)h;
    if (cur == kEmptyKey) {
      int old = atomicCAS(&keys[h], kEmptyKey, key);
      if (old == kEmptyKey || old == key) return (int)h;
    }
    h = (h + 1) & mask;
  }
  set_status(status, KK_ERR_CAPACITY);
  return -1;
}

// ---------------------------------------------------------------------------
// Bulk copies global -> shared memory (the TMA unit's cp.async.bulk) completed
// through an mbarrier in this CTA's shared memory.  Source and destination
// must be 16-byte aligned and the size a multiple of 16 bytes.
// ---------------------------------------------------------------------------
constexpr int kMbarSpinLimit = 1 << 22;  // try_wait rounds before a wait gives up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// makes barrier initialisations visible to the copy unit (and to other threads)
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void proxy_async_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase `parity` of bar; false (and KK_ERR_TIMEOUT in the
// status word) if it did not complete within kMbarSpinLimit rounds.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, int* status) {
  for (int k = 0; k < kMbarSpinLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  set_status(status, KK_ERR_TIMEOUT);
  return false;
}

// ---------------------------------------------------------------------------
// DF32: a float64 value carried as an unevaluated sum hi + lo of two float32s.
//
// Valid window: every nonzero input value has a binary exponent e with
// -50 <= e <= 50 (2^-50 <= |x| < 2^51).  Then every partial product lies in
// [2^-100, 2^102) and sums of up to 2^25 such products stay below FLT_MAX;
// the float32 error terms that fall below the normal range contribute less than
// 2^-149 each, below 2^-49 of the smallest product.  Values outside the window
// make the caller take the native float64 path.
//
// Error: a split loses < 2^-48 relative; a product < 2^-46; each accumulation
// step (two-sum of the high parts, float32 add of the low parts, fast-two-sum
// renormalisation) < 2^-47 of the running magnitude.  For n contributions to one
// entry the error stays below (n + 2) * 2^-46 * sum|a||b|, which is under
// 1e-12 * sum|a||b| for n <= 68.  Small integer values and their products are
// exact.
//
// So a row takes DF32 only where that bound holds for every entry of C(i,:):
// B's rows strictly ascending (checked by the B analysis; otherwise the whole
// product runs in float64), which caps an entry's contributions at
// nnz(A(i,:)), and nnz(A(i,:)) <= kDfMaxTerms.  Longer rows run in float64.
// ---------------------------------------------------------------------------
constexpr int kDfMinExp = -50;
constexpr int kDfMaxExp = 50;
constexpr int kDfMaxTerms = 64;

// True if the DF32 bound holds for a row of A with entries [pa, pe).
__device__ __forceinline__ bool df_row_terms_ok(int pa, int pe) { return pe - pa <= kDfMaxTerms; }

struct DF {
  float hi, lo;
};

// Split x into hi (its leading 24 significant bits, truncated) and lo (the
// remaining 29 bits, rounded to float32).  Returns false if x is nonzero and
// outside the window (then hi = lo = 0).
__device__ __forceinline__ bool df_split(double x, DF& out) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const uint32_t h = (uint32_t)(bits >> 32);
  const uint32_t l = (uint32_t)bits;
  const uint32_t E = (h >> 20) & 0x7FFu;
  out.hi = 0.0f;
  out.lo = 0.0f;
  if (E == 0) return ((h & 0xFFFFFu) | l) == 0u;  // +-0 fine; subnormals outside the window
  if (E < (uint32_t)(1023 + kDfMinExp) || E > (uint32_t)(1023 + kDfMaxExp)) return false;
  const uint32_t sign = h & 0x80000000u;
  // float32 exponent field = E - 1023 + 127 = E - 896, mantissa = top 23 bits
  out.hi = __uint_as_float(sign | ((E - 896u) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
  // remainder r * 2^(e-52), r < 2^29; the scale's float32 exponent field is
  // e - 52 + 127 = E - 948, which lies in [25, 125] inside the window.
  const uint32_t r = l & 0x1FFFFFFFu;
  const float scale = __uint_as_float((E - 948u) << 23);
  const float lo = __uint2float_rn(r) * scale;
  out.lo = __uint_as_float(__float_as_uint(lo) | sign);
  return true;
}

// s += a * b with a, b in DF32, renormalised after the step.
__device__ __forceinline__ void df_fma(DF& s, const DF a, const DF b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);               // exact error of p
  const float t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  // two-sum of the high parts
  const float sh = s.hi + p;
  const float bb = sh - s.hi;
  const float err = (s.hi - (sh - bb)) + (p - bb);
  const float lo = s.lo + (t + err);
  // fast-two-sum renormalisation
  const float hi = sh + lo;
  s.lo = lo - (hi - sh);
  s.hi = hi;
}

// Round hi + lo to the nearest float64 (within one unit in the last place) with
// integer operations only; zero, subnormal and non-finite high parts take the
// float64 route, which is rare.
__device__ __forceinline__ double df_to_double(DF v) {
  float hi = v.hi + v.lo;
  float lo = v.lo - (hi - v.hi);
  const uint32_t hb = __float_as_uint(hi);
  const uint32_t eh = (hb >> 23) & 0xFFu;
  if (eh == 0u || eh == 0xFFu) {
    if (hi == 0.0f && lo == 0.0f) return 0.0;
    return (double)hi + (double)lo;
  }
  long long m = (long long)(((hb & 0x7FFFFFu) | 0x800000u)) << 29;  // 53-bit significand
  const uint32_t lb = __float_as_uint(lo);
  const uint32_t el = (lb >> 23) & 0xFFu;
  if (el != 0u) {
    const unsigned long long ml = (lb & 0x7FFFFFu) | 0x800000u;
    const int sh = (int)el - (int)eh + 29;  // <= 5 because |lo| <= ulp(hi)/2
    long long add = 0;
    if (sh >= 0) {
      add = (long long)(ml << sh);
    } else if (sh > -40) {
      add = (long long)((ml + ((1ull << (-sh)) >> 1)) >> (-sh));
    }
    if ((lb ^ hb) & 0x80000000u) add = -add;
    m += add;
  }
  long long E = (long long)eh - 127 + 1023;
  if (m < (1ll << 52)) {  // hi a power of two and lo of opposite sign
    m <<= 1;
    E -= 1;
  }
  const unsigned long long out = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                 ((unsigned long long)E << 52) |
                                 ((unsigned long long)m & ((1ull << 52) - 1ull));
  return __longlong_as_double((long long)out);
}

__device__ __forceinline__ unsigned long long df_pack(DF v) {
  return ((unsigned long long)__float_as_uint(v.lo) << 32) | __float_as_uint(v.hi);
}
__device__ __forceinline__ DF df_unpack(unsigned long long u) {
  DF v;
  v.hi = __uint_as_float((uint32_t)u);
  v.lo = __uint_as_float((uint32_t)(u >> 32));
  return v;
}

// Atomic s += a*b on a packed DF32 slot (64-bit CAS loop, bounded).
__device__ __forceinline__ void df_atomic_fma(unsigned long long* slot, const DF a, const DF b,
                                              int* status) {
  unsigned long long old = *slot;
  for (int it = 0; it < kCasRetryLimit; ++it) {
    DF s = df_unpack(old);
    df_fma(s, a, b);
    const unsigned long long seen = atomicCAS(slot, old, df_pack(s));
    if (seen == old) return;
    old = seen;
  }
  set_status(status, KK_ERR_TIMEOUT);
}

// Position (0..31) of the k-th (0-based) set bit of m, k < popc(m): a binary
// search on the popcounts of the word's halves, quarters, ...
__device__ __forceinline__ int select_set_bit(uint32_t m, int k) {
  int pos = 0, c;
  c = __popc(m & 0xFFFFu);
  if (k >= c) { k -= c; pos += 16; m >>= 16; }
  c = __popc(m & 0xFFu);
  if (k >= c) { k -= c; pos += 8; m >>= 8; }
  c = __popc(m & 0xFu);
  if (k >= c) { k -= c; pos += 4; m >>= 4; }
  c = __popc(m & 0x3u);
  if (k >= c) { k -= c; pos += 2; m >>= 2; }
  if (k >= (int)(m & 1u)) pos += 1;
  return pos;
}

// The columns of a warp's 32 bit-vector words in ascending order, written by
// consecutive lanes to consecutive entries (coalesced stores, whatever the
// words' popcounts): lane l holds word index w and bits m, incl = the
// inclusive scan of the popcounts over the lanes, total = incl of lane 31.
// write(e, col) is called for the e-th column, e < total.  All 32 lanes call.
template <class Write>
__device__ __forceinline__ void warp_expand_bits(int w, uint32_t m, int incl, int total, Write write) {
  const int lane = threadIdx.x & 31;
  for (int e0 = 0; e0 < total; e0 += 32) {
    const int e = e0 + lane;
    // source lane: the number of lanes whose inclusive count is <= e
    int src = 0;
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) {
      const int v = __shfl_sync(0xffffffffu, incl, src + st - 1);
      if (v <= e) src += st;
    }
    const uint32_t mm = __shfl_sync(0xffffffffu, m, src);
    const int ws = __shfl_sync(0xffffffffu, w, src);
    const int start = __shfl_sync(0xffffffffu, incl, src) - __popc(mm);
    if (e < total) write(e, ws * 32 + select_set_bit(mm, e - start));
  }
}

// Jacobi-fused product's 1/D(i) to about one unit in the last place without
// the float64 divide (a long sequence on the FP64 pipe, which is slow on this
// part): a float32 reciprocal
// refined by two Newton-Raphson steps x <- x + x(1 - d x), each of which about
// doubles the correct bits (24 -> 48 -> 53).  Outside the float32 range the
// float64 divide is used.
__device__ __forceinline__ double jacobi_recip(double d) {
  // |d| in [2^-99, 2^99], decided on the exponent bits (no float64 compare)
  const uint32_t e = ((uint32_t)(__double_as_longlong(d) >> 52)) & 0x7FFu;
  if (e < 1023u - 99u || e > 1023u + 99u) return 1.0 / d;
  double x = (double)__frcp_rn((float)d);
  x = fma(x, fma(-d, x, 1.0), x);
  x = fma(x, fma(-d, x, 1.0), x);
  return x;
}

}  // namespace kk
