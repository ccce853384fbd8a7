// Numeric phase kernels: column indices and values of C (Kokkos Kernels paper,
// Sec. "Standard SpGEMM Kernel": the numeric phase inserts (column, value) pairs
// into the accumulator, value := value + A(i,j) * B(j,c)).  Every row's count is
// known from the symbolic phase, so each row's accumulator is sized from it.
//
// Tiers (as in the symbolic phase):
//   team  - TEAM lanes per row: shared-memory hash map (keys, values), then a
//           team-level bitonic sort of the occupied slots (paper, Sec. "Multi-
//           Level Bitonic Sorting": team-level sort in shared memory) so each row
//           is written with ascending columns;
//   CTA   - one CTA per row, same structure with block-wide sort;
//   dense - one CTA per row, dense value array + bit vector over a window of
//           columns swept across [0, k); set bits are enumerated in column order,
//           so no sort is needed.
//
// Arithmetic: DF32 (float64 emulated by float32 pairs on the FP32 pipe) when the
// values of B and of the row's A entries lie in the DF32 window, native float64
// otherwise.  In vector mode with distinct columns per B row the updates of one
// output entry happen in A-row storage order without atomics.
#include "kk_internal.h"
#include "kk_rowops.cuh"
#include "kk_visit.cuh"

namespace kk {
namespace {

constexpr int kTeamBlock = 256;
constexpr int kCtaBlock = 512;
constexpr int kDenseBlock = 512;



struct NumArgs {
  CsrView A, B;
  int32_t b_sorted;
  const float2* b_split;
  const int32_t* b_range_bad;
  int32_t arith;
  const int64_t* c_rowptr;
  const int32_t* rows;
  int32_t nrows;
  int32_t* c_colind;
  double* c_vals;
  int* status;
  int32_t k;
  int32_t W;  // dense chunk width
  // speculative one-pass (learned form): staging offsets / arrays, row counts
  const int64_t* soff;
  int32_t* scol;
  double* sval;
  int32_t* cnt_out;
};

// ---------------------------------------------------------------------------
// Team tier
// ---------------------------------------------------------------------------
// Teams per CTA for a team-tier map of 2^LOG2S slots (16 bytes per slot: key,
// value, half a sort item): at most 96 KB per CTA.
template <int TEAM, int LOG2S>
struct NumTeamGeom {
  static constexpr int kByTable = (96 * 1024) / ((1 << LOG2S) * 16);
  static constexpr int TPB = (kTeamBlock / TEAM) < kByTable ? (kTeamBlock / TEAM)
                                                             : (kByTable < 1 ? 1 : kByTable);
};

template <int TEAM, int LOG2S, bool FLAT>
__global__ void __launch_bounds__(kTeamBlock) k_num_team(NumArgs g) {
  extern __shared__ u64 smem_u[];
  constexpr int S = 1 << LOG2S;
  constexpr int H = S / 2;
  constexpr int TPB = NumTeamGeom<TEAM, LOG2S>::TPB;
  const int team = threadIdx.x / TEAM;
  const int tl = threadIdx.x % TEAM;
  const int lane = threadIdx.x & 31;
  const unsigned mask = team_mask<TEAM>();
  u64* vals = smem_u + team * S;
  u64* sbuf = smem_u + TPB * S + team * H;
  int* keys = reinterpret_cast<int*>(smem_u + TPB * S + TPB * H) + team * S;
  const bool df_all = g.arith == kArithDF32 && *g.b_range_bad == 0;
  const bool atomic = FLAT || !g.b_sorted;
  const FullRange rng{g.A.colind, g.B.rowptr};
  const int32_t* bcol = g.B.colind;
  const double* bval = g.B.vals;
  const float2* bspl = g.b_split;
  int* status = g.status;
  for (int r = blockIdx.x * TPB + team; r < g.nrows; r += gridDim.x * TPB) {
    const int i = g.rows[r];
    const int64_t off = g.c_rowptr[i];
    const int cnt = (int)(g.c_rowptr[i + 1] - off);
    for (int s = tl; s < S; s += TEAM) {
      keys[s] = kEmptyKey;
      vals[s] = 0ull;
    }
    __syncwarp(mask);
    const int pa = g.A.rowptr[i], pe = g.A.rowptr[i + 1];
    const bool df = df_all && df_row_terms_ok(pa, pe) && row_df_ok<TEAM>(g.A.vals, pa, pe, tl, mask);
    if (df) {
      visit_products<TEAM, FLAT, DF>(pa, pe, 0, 1, tl, mask, rng, PrepDF{g.A, i},
                                     [&](DF a, int, int q) {
                                       const int slot = map_slot(keys, bcol[q], LOG2S, status);
                                       if (slot >= 0) upd_df(vals, slot, a, load_b(bspl, q), atomic, status);
                                     });
    } else {
      visit_products<TEAM, FLAT, double>(pa, pe, 0, 1, tl, mask, rng, PrepF64{g.A, i},
                                         [&](double a, int, int q) {
                                           const int slot = map_slot(keys, bcol[q], LOG2S, status);
                                           if (slot >= 0) upd_f64(vals, slot, a, bval[q], atomic);
                                         });
    }
    __syncwarp(mask);
    // compaction of occupied slots into (key << 32 | slot) items
    int base = 0;
    const int tbase = lane & ~(TEAM - 1);
    for (int s0 = 0; s0 < S; s0 += TEAM) {
      const int s = s0 + tl;
      const int key = keys[s];
      const bool occ = key != kEmptyKey;
      const unsigned bal = __ballot_sync(mask, occ);
      unsigned seg;
      if constexpr (TEAM == 32) seg = bal; else seg = (bal >> tbase) & ((1u << TEAM) - 1u);
      const int pos = base + __popc(seg & ((1u << tl) - 1u));
      if (occ && pos < H) sbuf[pos] = ((u64)(uint32_t)key << 32) | (u64)s;
      base += __popc(seg);
    }
    if (base != cnt && tl == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    const int n = max(0, min(min(base, cnt), H));
    const int P = pow2ceil(n);
    for (int t = n + tl; t < P; t += TEAM) sbuf[t] = ~0ull;
    __syncwarp(mask);
    team_bitonic<TEAM>(sbuf, P, tl, mask);
    for (int t = tl; t < n; t += TEAM) {
      const u64 it = sbuf[t];
      g.c_colind[off + t] = (int32_t)(it >> 32);
      g.c_vals[off + t] = out_value(vals[(uint32_t)it], df);
    }
    __syncwarp(mask);
  }
}

// ---------------------------------------------------------------------------
// Warp-per-row vector kernel (the common case for rows whose referenced B rows
// are long: stencils, FEM).  One warp per row; the warp's lanes split each B
// row; A entries are taken in storage order, so the update of an output entry
// needs no atomic when B's rows have distinct columns.  The lane that inserts
// a key writes its first product, so the value table needs no clearing.  After
// accumulation the occupied keys are compacted and sorted in registers
// (bitonic network, E keys per lane, element e = r*32 + lane), then each sorted
// key finds its value slot again and the row is written coalesced.
// ---------------------------------------------------------------------------
template <int LOG2S>
struct WarpVecGeom {
  static constexpr int S = 1 << LOG2S;
  static constexpr int E = (S / 2) / 32 < 1 ? 1 : (S / 2) / 32;  // keys per lane (P = 32*E >= S/2)
  static constexpr int WPB = 8;                                   // warps per CTA
  // per warp: keys int[S] | vals u64[S] | A staging int4[32] | key staging int[32*E]
  static constexpr size_t kWarpBytes = (size_t)S * 4 + (size_t)S * 8 + 32 * 16 + 32 * E * 4;
};

__device__ __forceinline__ int probe_find(const int* keys, int32_t key, int log2s) {
  const uint32_t mask = (1u << log2s) - 1u;
  uint32_t h = hash_slot(key, log2s);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int cur = keys[h];
    if (cur == key) return (int)h;
    if (cur == kEmptyKey) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// Find-or-insert; *inserted tells whether this call created the key.
__device__ __forceinline__ int probe_insert(int* keys, int32_t key, int log2s, bool* inserted,
                                            int* status) {
  const uint32_t mask = (1u << log2s) - 1u;
  uint32_t h = hash_slot(key, log2s);
  for (uint32_t p = 0; p <= mask; ++p) {
    const int cur = keys[h];
    if (cur == key) {
      *inserted = false;
      return (int)h;
    }
    if (cur == kEmptyKey) {
      const int old = atomicCAS(&keys[h], kEmptyKey, key);
      if (old == kEmptyKey) {
        *inserted = true;
        return (int)h;
      }
      if (old == key) {
        *inserted = false;
        return (int)h;
      }
    }
    h = (h + 1) & mask;
  }
  *inserted = false;
  set_status(status, KK_ERR_CAPACITY);
  return -1;
}

// One product into the warp's map: find-or-insert col; the inserting lane
// stores the first product, later ones accumulate.  a / b carry DF32 pairs
// (df) or the two 32-bit halves of a float64.
// Returns 1 if this product inserted its column, 0 if the column was present,
// -1 if the table was full (the product is then dropped).
template <int LOG2S>
__device__ __forceinline__ int warp_vec_update(int* keys, u64* vals, int col, int2 a, float2 b,
                                               bool df, int* status) {
  bool ins;
  const int slot = probe_insert(keys, col, LOG2S, &ins, status);
  if (slot < 0) return -1;
  if (df) {
    DF ad, bd, s;
    ad.hi = __int_as_float(a.x);
    ad.lo = __int_as_float(a.y);
    bd.hi = b.x;
    bd.lo = b.y;
    if (ins) {
      s.hi = 0.f;
      s.lo = 0.f;
    } else {
      s = df_unpack(vals[slot]);
    }
    df_fma(s, ad, bd);
    vals[slot] = df_pack(s);
  } else {
    const double av = __longlong_as_double(((long long)a.y << 32) | (unsigned)a.x);
    const double bvv = __longlong_as_double(((long long)__float_as_int(b.y) << 32) |
                                            (unsigned)__float_as_int(b.x));
    double* v = reinterpret_cast<double*>(&vals[slot]);
    *v = ins ? av * bvv : fma(av, bvv, *v);
  }
  return ins ? 1 : 0;
}

// Bitonic sort of 32*E int keys held in registers, element e = r*32 + lane.
template <int E>
__device__ __forceinline__ void warp_bitonic_regs(int (&v)[E], int lane) {
  constexpr int P = 32 * E;
  constexpr int LOG2P = (P >= 1024) ? 10 : (P >= 512) ? 9 : (P >= 256) ? 8 : (P >= 128) ? 7 : (P >= 64) ? 6 : 5;
#pragma unroll
  for (int lk = 1; lk <= LOG2P; ++lk) {
    const int k = 1 << lk;
#pragma unroll
    for (int lj = lk - 1; lj >= 0; --lj) {
      const int j = 1 << lj;
      if (j >= 32) {
        const int jr = j >> 5;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if ((r & jr) == 0) {
            const int r2 = r | jr;
            const int e = r * 32 + lane;
            const bool up = (e & k) == 0;
            const int a = v[r], b = v[r2];
            const bool sw = (a > b) == up;
            v[r] = sw ? b : a;
            v[r2] = sw ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int e = r * 32 + lane;
          const int o = __shfl_xor_sync(0xffffffffu, v[r], j);
          const bool keep_min = ((e & j) == 0) == ((e & k) == 0);
          v[r] = keep_min ? min(v[r], o) : max(v[r], o);
        }
      }
    }
  }
}

// SPEC = true: speculative one-pass of the learned form.  The row's count is
// not known; the table holds S slots and the staging area S/2 entries at
// g.soff[i].  A row whose distinct columns exceed S/2 (or fill the table)
// overflows: it is abandoned and marked with g.cnt_out[i] = -1 for the plain
// two-phase re-run.  Otherwise its sorted columns and values go to the staging
// area and g.cnt_out[i] receives its count.
template <int LOG2S, bool SPEC>
__global__ void __launch_bounds__(256, 3) k_num_warp_vec(NumArgs g) {
  using G = WarpVecGeom<LOG2S>;
  constexpr int S = G::S;
  constexpr int E = G::E;
  constexpr int P = 32 * E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* base = smem_raw + (size_t)warp * G::kWarpBytes;
  u64* vals = reinterpret_cast<u64*>(base);
  int* keys = reinterpret_cast<int*>(base + (size_t)S * 8);
  int4* ainfo = reinterpret_cast<int4*>(base + (size_t)S * 12);
  int* kst = reinterpret_cast<int*>(base + (size_t)S * 12 + 32 * 16);
  const bool df_all = g.arith == kArithDF32 && *g.b_range_bad == 0;
  const int32_t* __restrict__ acol = g.A.colind;
  const double* __restrict__ aval = g.A.vals;
  const int32_t* __restrict__ brp = g.B.rowptr;
  const int32_t* __restrict__ bcol = g.B.colind;
  const double* __restrict__ bval = g.B.vals;
  const float2* __restrict__ bspl = g.b_split;
  int* status = g.status;
  int* pstatus = SPEC ? nullptr : status;  // a full table is an overflow, not an error
  int32_t* out_col = SPEC ? g.scol : g.c_colind;
  double* out_val = SPEC ? g.sval : g.c_vals;
  // contiguous share of rows per CTA (neighbouring rows reuse B rows in L1)
  const int per_cta = (g.nrows + gridDim.x - 1) / gridDim.x;
  const int r_begin = blockIdx.x * per_cta;
  const int r_end = min(g.nrows, r_begin + per_cta);
  for (int r = r_begin + warp; r < r_end; r += G::WPB) {
    const int i = g.rows[r];
    const int64_t off = SPEC ? g.soff[i] : g.c_rowptr[i];
    const int cnt = SPEC ? S / 2 : (int)(g.c_rowptr[i + 1] - off);
    int n_ins = 0;
    bool ovf = false;
#pragma unroll
    for (int s = lane * 4; s < S; s += 128) *reinterpret_cast<int4*>(&keys[s]) = make_int4(-1, -1, -1, -1);
    __syncwarp();
    const int pa = g.A.rowptr[i], pe = g.A.rowptr[i + 1];
    bool df = df_all && df_row_terms_ok(pa, pe);
    if (df && pe - pa > 32) {
      // multi-chunk row: check the whole row against the DF32 window first
      int bad = 0;
      for (int p = pa + lane; p < pe; p += 32) {
        DF t;
        bad |= df_split(aval[p], t) ? 0 : 1;
      }
      df = __any_sync(0xffffffffu, bad) == 0;
    }
    for (int p0 = pa; p0 < pe && !ovf; p0 += 32) {
      const int p = p0 + lane;
      int4 info = make_int4(0, 0, 0, 0);
      double a64 = 0.0;
      int bad = 0;
      if (p < pe) {
        const int j = acol[p];
        const int bs = brp[j];
        info.x = bs;
        info.y = brp[j + 1] - bs;
        a64 = a_value(g.A, i, p);
        if (df) {
          DF ad;
          bad = df_split(a64, ad) ? 0 : 1;
          info.z = __float_as_int(ad.hi);
          info.w = __float_as_int(ad.lo);
        }
      }
      if (df && __any_sync(0xffffffffu, bad)) df = false;  // single-chunk row outside the window
      if (!df) {
        const long long ab = __double_as_longlong(a64);
        info.z = (int)(ab & 0xffffffffll);
        info.w = (int)(ab >> 32);
      }
      ainfo[lane] = info;
      __syncwarp();
      const int nch = min(32, pe - p0);
      const unsigned maxlen = __reduce_max_sync(0xffffffffu, (unsigned)info.y);
      if (maxlen <= 32u) {
        // every referenced B row fits one pass of the warp: issue the loads of
        // kBatch A entries before their updates (memory-level parallelism)
        constexpr int kBatch = 8;
        for (int t0 = 0; t0 < nch && !ovf; t0 += kBatch) {
          int cols[kBatch];
          float2 bv[kBatch];
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            cols[u] = -1;
            bv[u] = make_float2(0.f, 0.f);
            const int t = t0 + u;
            if (t < nch) {
              const int2 in = *reinterpret_cast<const int2*>(&ainfo[t]);
              if (lane < in.y) {
                const int q = in.x + lane;
                cols[u] = bcol[q];
                if (df) {
                  bv[u] = bspl[q];
                } else {
                  const long long bb = __double_as_longlong(bval[q]);
                  bv[u] = make_float2(__int_as_float((int)(bb & 0xffffffffll)), __int_as_float((int)(bb >> 32)));
                }
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kBatch; ++u) {
            if (t0 + u < nch) {
              int res = 0;
              if (cols[u] >= 0) {
                const int2 az = *reinterpret_cast<const int2*>(&ainfo[t0 + u].z);
                res = warp_vec_update<LOG2S>(keys, vals, cols[u], az, bv[u], df, pstatus);
              }
              if (SPEC) {
                n_ins += __popc(__ballot_sync(0xffffffffu, res == 1));
                if (__any_sync(0xffffffffu, res < 0) || n_ins > S / 2) ovf = true;
              }
              __syncwarp();  // this A entry's updates are visible before the next one's
            }
          }
        }
      } else {
        for (int t = 0; t < nch && !ovf; ++t) {
          const int4 in = ainfo[t];
          for (int q0 = 0; q0 < in.y && !ovf; q0 += 32) {
            const int q = in.x + q0 + lane;
            int res = 0;
            if (q0 + lane < in.y) {
              float2 b2;
              if (df) {
                b2 = bspl[q];
              } else {
                const long long bb = __double_as_longlong(bval[q]);
                b2 = make_float2(__int_as_float((int)(bb & 0xffffffffll)), __int_as_float((int)(bb >> 32)));
              }
              res = warp_vec_update<LOG2S>(keys, vals, bcol[q], make_int2(in.z, in.w), b2, df, pstatus);
            }
            if (SPEC) {
              n_ins += __popc(__ballot_sync(0xffffffffu, res == 1));
              if (__any_sync(0xffffffffu, res < 0) || n_ins > S / 2) ovf = true;
            }
          }
          __syncwarp();  // this A entry's updates are visible before the next one's
        }
      }
      __syncwarp();
    }
    if (SPEC && ovf) {
      if (lane == 0) g.cnt_out[i] = -1;
      __syncwarp();
      continue;
    }
    // compaction of occupied keys
    int n = 0;
#pragma unroll 4
    for (int s0 = 0; s0 < S; s0 += 32) {
      const int key = keys[s0 + lane];
      const bool occ = key != kEmptyKey;
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      const int pos = n + __popc(bal & ((1u << lane) - 1u));
      if (occ && pos < P) kst[pos] = key;
      n += __popc(bal);
    }
    if (!SPEC && n != cnt && lane == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    if (SPEC && lane == 0) g.cnt_out[i] = n;
    const int nn = max(0, min(min(n, cnt), P));
    __syncwarp();
    int v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = r * 32 + lane;
      v[r] = e < nn ? kst[e] : 0x7fffffff;
    }
    warp_bitonic_regs<E>(v, lane);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = r * 32 + lane;
      if (e < nn) {
        const int slot = probe_find(keys, v[r], LOG2S);
        out_col[off + e] = v[r];
        out_val[off + e] = slot >= 0 ? out_value(vals[slot], df) : 0.0;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// CTA tier: warps of the CTA share one hash map; flattened traversal, atomics.
// ---------------------------------------------------------------------------
template <int LOG2S>
__global__ void __launch_bounds__(kCtaBlock) k_num_cta(NumArgs g) {
  extern __shared__ u64 smem_u[];
  constexpr int S = 1 << LOG2S;
  constexpr int H = S / 2;
  __shared__ int scan_scratch[33];
  __shared__ int flag;
  u64* vals = smem_u;
  u64* sbuf = smem_u + S;
  int* keys = reinterpret_cast<int*>(smem_u + S + H);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const bool df_all = g.arith == kArithDF32 && *g.b_range_bad == 0;
  const FullRange rng{g.A.colind, g.B.rowptr};
  const int32_t* bcol = g.B.colind;
  const double* bval = g.B.vals;
  const float2* bspl = g.b_split;
  int* status = g.status;
  for (int r = blockIdx.x; r < g.nrows; r += gridDim.x) {
    const int i = g.rows[r];
    const int64_t off = g.c_rowptr[i];
    const int cnt = (int)(g.c_rowptr[i + 1] - off);
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      keys[s] = kEmptyKey;
      vals[s] = 0ull;
    }
    const int pa = g.A.rowptr[i], pe = g.A.rowptr[i + 1];
    const bool df = df_all && df_row_terms_ok(pa, pe) && block_df_ok(g.A.vals, pa, pe, &flag);  // syncs
    if (df) {
      visit_products<32, true, DF>(pa, pe, warp, nwarps, lane, 0xffffffffu, rng, PrepDF{g.A, i},
                                   [&](DF a, int, int q) {
                                     const int slot = map_slot(keys, bcol[q], LOG2S, status);
                                     if (slot >= 0) upd_df(vals, slot, a, load_b(bspl, q), true, status);
                                   });
    } else {
      visit_products<32, true, double>(pa, pe, warp, nwarps, lane, 0xffffffffu, rng,
                                       PrepF64{g.A, i}, [&](double a, int, int q) {
                                         const int slot = map_slot(keys, bcol[q], LOG2S, status);
                                         if (slot >= 0) upd_f64(vals, slot, a, bval[q], true);
                                       });
    }
    __syncthreads();
    int base = 0;
    for (int s0 = 0; s0 < S; s0 += blockDim.x) {
      const int s = s0 + threadIdx.x;
      const int key = keys[s];
      const int occ = key != kEmptyKey ? 1 : 0;
      int tot;
      const int pos = base + block_exclusive_scan(occ, scan_scratch, &tot);
      if (occ && pos < H) sbuf[pos] = ((u64)(uint32_t)key << 32) | (u64)s;
      base += tot;
    }
    if (base != cnt && threadIdx.x == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
    const int n = max(0, min(min(base, cnt), H));
    const int P = pow2ceil(n);
    for (int t = n + threadIdx.x; t < P; t += blockDim.x) sbuf[t] = ~0ull;
    __syncthreads();
    block_bitonic(sbuf, P);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const u64 it = sbuf[t];
      g.c_colind[off + t] = (int32_t)(it >> 32);
      g.c_vals[off + t] = out_value(vals[(uint32_t)it], df);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Dense tier: value array + bit vector over columns [c0, c0 + W).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kDenseBlock) k_num_dense(NumArgs g) {
  extern __shared__ u64 smem_u[];
  __shared__ int scan_scratch[33];
  __shared__ int flag;
  const int W = g.W;
  const int words = W >> 5;
  u64* vals = smem_u;
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem_u + W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const bool df_all = g.arith == kArithDF32 && *g.b_range_bad == 0;
  const int32_t* acol = g.A.colind;
  const int32_t* brp = g.B.rowptr;
  const int32_t* bcol = g.B.colind;
  const double* bval = g.B.vals;
  const float2* bspl = g.b_split;
  int* status = g.status;
  const int k = g.k;
  for (int r = blockIdx.x; r < g.nrows; r += gridDim.x) {
    const int i = g.rows[r];
    const int64_t off = g.c_rowptr[i];
    const int64_t cnt = g.c_rowptr[i + 1] - off;
    const int pa = g.A.rowptr[i], pe = g.A.rowptr[i + 1];
    const bool df = df_all && df_row_terms_ok(pa, pe) && block_df_ok(g.A.vals, pa, pe, &flag);
    int64_t run = 0;
    for (long long c0l = 0; c0l < k; c0l += W) {
      const int c0 = (int)c0l;
      const int cend = (k - c0 > W) ? c0 + W : k;
      const bool whole = (k <= W) || !g.b_sorted;
      for (int w = threadIdx.x; w < W; w += blockDim.x) vals[w] = 0ull;
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
      if (df) {
        visit_products<32, true, DF>(pa, pe, warp, nwarps, lane, 0xffffffffu, rng,
                                     PrepDF{g.A, i}, [&](DF a, int, int q) {
                                       const uint32_t o = (uint32_t)(bcol[q] - c0);
                                       if (o < (uint32_t)W) {
                                         atomicOr(&bits[o >> 5], 1u << (o & 31));
                                         df_atomic_fma(&vals[o], a, load_b(bspl, q), status);
                                       }
                                     });
      } else {
        visit_products<32, true, double>(pa, pe, warp, nwarps, lane, 0xffffffffu, rng,
                                         PrepF64{g.A, i}, [&](double a, int, int q) {
                                           const uint32_t o = (uint32_t)(bcol[q] - c0);
                                           if (o < (uint32_t)W) {
                                             atomicOr(&bits[o >> 5], 1u << (o & 31));
                                             atomicAdd(reinterpret_cast<double*>(&vals[o]), a * bval[q]);
                                           }
                                         });
      }
      __syncthreads();
      for (int w0 = 0; w0 < words; w0 += blockDim.x) {
        const int w = w0 + threadIdx.x;
        const uint32_t word = w < words ? bits[w] : 0u;
        int tot;
        const int pre = block_exclusive_scan(__popc(word), scan_scratch, &tot);
        int64_t pos = run + pre;
        uint32_t rest = word;
        while (rest) {
          const int b = __ffs(rest) - 1;
          rest &= rest - 1;
          if (pos < cnt) {
            const int o = w * 32 + b;
            g.c_colind[off + pos] = c0 + o;
            g.c_vals[off + pos] = out_value(vals[o], df);
          }
          ++pos;
        }
        run += tot;
      }
      __syncthreads();
    }
    if (run != cnt && threadIdx.x == 0) set_status(status, KK_ERR_STRUCTURE_MISMATCH);
  }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int TEAM, int LOG2S, bool FLAT>
cudaError_t launch_team(const LaunchCtx& ctx, const NumArgs& g) {
  constexpr int TPB = NumTeamGeom<TEAM, LOG2S>::TPB;
  const size_t smem = (size_t)TPB * (1u << LOG2S) * (8 + 4 + 4);
  auto kern = k_num_team<TEAM, LOG2S, FLAT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long blocks = (g.nrows + TPB - 1) / TPB;
  blocks = blocks > (long long)ctx.num_sms * 32 ? (long long)ctx.num_sms * 32 : blocks;
  kern<<<(unsigned)blocks, TPB * TEAM, smem, ctx.stream>>>(g);
  return cudaGetLastError();
}

template <int TEAM, bool FLAT>
cudaError_t dispatch_team(const LaunchCtx& ctx, int log2s, const NumArgs& g) {
  switch (log2s) {
    case 5: return launch_team<TEAM, 5, FLAT>(ctx, g);
    case 6: return launch_team<TEAM, 6, FLAT>(ctx, g);
    case 7: return launch_team<TEAM, 7, FLAT>(ctx, g);
    case 8: return launch_team<TEAM, 8, FLAT>(ctx, g);
    case 9: return launch_team<TEAM, 9, FLAT>(ctx, g);
    case 10: return launch_team<TEAM, 10, FLAT>(ctx, g);
    case 11: return launch_team<TEAM, 11, FLAT>(ctx, g);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOG2S, bool SPEC = false>
cudaError_t launch_warp_vec(const LaunchCtx& ctx, const NumArgs& g) {
  using G = WarpVecGeom<LOG2S>;
  const size_t smem = (size_t)G::WPB * G::kWarpBytes;
  auto kern = k_num_warp_vec<LOG2S, SPEC>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long blocks = (g.nrows + G::WPB * 4 - 1) / (G::WPB * 4);
  const long long cap = (long long)ctx.num_sms * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, G::WPB * 32, smem, ctx.stream>>>(g);
  return cudaGetLastError();
}

template <int LOG2S>
cudaError_t launch_cta(const LaunchCtx& ctx, const NumArgs& g) {
  const size_t smem = (size_t)(1u << LOG2S) * (8 + 4 + 4);
  auto kern = k_num_cta<LOG2S>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long blocks = g.nrows < ctx.num_sms * 4 ? g.nrows : ctx.num_sms * 4;
  kern<<<(unsigned)blocks, kCtaBlock, smem, ctx.stream>>>(g);
  return cudaGetLastError();
}

}  // namespace

size_t numeric_smem_bytes(const BinSpec& bin) {
  if (bin.tier == kTierTeam) {
    int tpb = kTeamBlock / bin.team, by = (96 * 1024) / (bin.slots * 16);
    if (by < 1) by = 1;
    return (size_t)(tpb < by ? tpb : by) * bin.slots * 16;
  }
  if (bin.tier == kTierCta) return (size_t)bin.slots * 16;
  return (size_t)bin.slots * 8 + (size_t)bin.slots / 8;
}

cudaError_t launch_numeric_bin(const LaunchCtx& ctx, const BinSpec& bin, const CsrView& A,
                               const CsrView& B, int32_t b_sorted, const float2* b_split,
                               const int32_t* b_range_bad, int32_t arith,
                               const int64_t* c_rowptr, const int32_t* rows, int32_t nrows,
                               int32_t* c_colind, double* c_vals, int32_t) {
  if (nrows <= 0) return cudaSuccess;
  if (bin.tier == kTierThread)
    return launch_numeric_thread(ctx, A, B, c_rowptr, rows, nrows, c_colind, c_vals);
  NumArgs g{A, B, b_sorted, b_split, b_range_bad, arith, c_rowptr, rows, nrows,
            c_colind, c_vals, ctx.status, B.n, bin.slots, nullptr, nullptr, nullptr, nullptr};
  int log2s = 0;
  while ((1 << log2s) < bin.slots) ++log2s;
  cudaError_t e = cudaErrorInvalidValue;
  if (bin.tier == kTierTeam) {
    if (!bin.flat && bin.team == 32 && b_sorted && log2s >= 5 && log2s <= 9) {
      timer_begin(ctx.timer, ctx.stream, "num_warp_vec");
      switch (log2s) {
        case 5: e = launch_warp_vec<5>(ctx, g); break;
        case 6: e = launch_warp_vec<6>(ctx, g); break;
        case 7: e = launch_warp_vec<7>(ctx, g); break;
        case 8: e = launch_warp_vec<8>(ctx, g); break;
        case 9: e = launch_warp_vec<9>(ctx, g); break;
      }
      timer_end(ctx.timer, ctx.stream);
      return e;
    }
    timer_begin(ctx.timer, ctx.stream, bin.flat ? "num_team_flat" : "num_team_vec");
    if (bin.flat) {
      if (bin.team == 8) e = dispatch_team<8, true>(ctx, log2s, g);
      else if (bin.team == 32) e = dispatch_team<32, true>(ctx, log2s, g);
    } else {
      if (bin.team == 8) e = dispatch_team<8, false>(ctx, log2s, g);
      else if (bin.team == 32) e = dispatch_team<32, false>(ctx, log2s, g);
    }
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  if ((bin.tier == kTierCta || bin.tier == kTierDense) && wide_numeric_fits(ctx, B.n)) {
    timer_begin(ctx.timer, ctx.stream, "num_wide");
    e = launch_numeric_wide(ctx, A, B, c_rowptr, rows, nrows, c_colind, c_vals);
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  if (bin.tier == kTierCta) {
    timer_begin(ctx.timer, ctx.stream, "num_cta");
    switch (log2s) {
      case 12: e = launch_cta<12>(ctx, g); break;
      case 13: e = launch_cta<13>(ctx, g); break;
      default: e = cudaErrorInvalidValue;
    }
    timer_end(ctx.timer, ctx.stream);
    return e;
  }
  timer_begin(ctx.timer, ctx.stream, "num_dense");
  const size_t smem = numeric_smem_bytes(bin);
  e = set_smem(k_num_dense, smem);
  if (e == cudaSuccess) {
    long long blocks = nrows < ctx.num_sms ? nrows : ctx.num_sms;
    k_num_dense<<<(unsigned)blocks, kDenseBlock, smem, ctx.stream>>>(g);
    e = cudaGetLastError();
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

cudaError_t launch_onepass(const LaunchCtx& ctx, int32_t log2s, const CsrView& A, const CsrView& B,
                           const float2* b_split, const int32_t* b_range_bad, int32_t arith,
                           const int64_t* soff, const int32_t* rows, int32_t nrows, int32_t* scol,
                           double* sval, int32_t* cnt_out) {
  if (nrows <= 0) return cudaSuccess;
  NumArgs g{A, B, 1, b_split, b_range_bad, arith, nullptr, rows, nrows, nullptr, nullptr,
            ctx.status, B.n, 0, soff, scol, sval, cnt_out};
  timer_begin(ctx.timer, ctx.stream, "onepass_warp");
  cudaError_t e = cudaErrorInvalidValue;
  switch (log2s) {
    case 5: e = launch_warp_vec<5, true>(ctx, g); break;
    case 6: e = launch_warp_vec<6, true>(ctx, g); break;
    case 7: e = launch_warp_vec<7, true>(ctx, g); break;
    case 8: e = launch_warp_vec<8, true>(ctx, g); break;
    case 9: e = launch_warp_vec<9, true>(ctx, g); break;
  }
  timer_end(ctx.timer, ctx.stream);
  return e;
}

}  // namespace kk
