// Device building blocks shared by the single-instance kernels and the
// batched persistent kernel, so that both compute bit-identical segment sums,
// grid prefixes, spacings, keys and in-segment decisions.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace gbr {

// Striped (coalesced) load of one segment: lane holds elements
//   binary64: 2*lane + 64*i + {0,1},   i < 8
//   binary32: 4*lane + 128*i + {0..3}, i < 4
// Missing elements of a ragged last segment read as +0.
template <typename T, bool kVec>
__device__ __forceinline__ void load_seg_striped(const T* __restrict__ w, long long base, long long M, int lane,
                                                 typename FixedTraits<T>::Bits (&b)[kSegV]) {
  using Bits = typename FixedTraits<T>::Bits;
  const bool full = base + kSeg <= M;
  if (sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const long long e = base + 2 * lane + 64 * i;
      if (kVec && full) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(w + e));
        b[2 * i] = (Bits)v.x;
        b[2 * i + 1] = (Bits)v.y;
      } else {
        b[2 * i] = e < M ? (Bits)__ldg(reinterpret_cast<const unsigned long long*>(w + e)) : (Bits)0;
        b[2 * i + 1] = e + 1 < M ? (Bits)__ldg(reinterpret_cast<const unsigned long long*>(w + e + 1)) : (Bits)0;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long e = base + 4 * lane + 128 * i;
      if (kVec && full) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(w + e));
        b[4 * i] = (Bits)v.x;
        b[4 * i + 1] = (Bits)v.y;
        b[4 * i + 2] = (Bits)v.z;
        b[4 * i + 3] = (Bits)v.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          b[4 * i + q] = e + q < M ? (Bits)__ldg(reinterpret_cast<const unsigned*>(w + e + q)) : (Bits)0;
      }
    }
  }
}

// Lane-major load (lane holds 16 consecutive elements 16*lane + i), used
// where within-segment order matters (prefixes).
template <typename T, bool kVec>
__device__ __forceinline__ void load_seg_blocked(const T* __restrict__ w, long long base, long long M, int lane,
                                                 typename FixedTraits<T>::Bits (&b)[kSegV]) {
  using Bits = typename FixedTraits<T>::Bits;
  const long long e0 = base + (long long)lane * kSegV;
  const bool full = e0 + kSegV <= M;
  if (kVec && full) {
    if (sizeof(T) == 8) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(w + e0 + 2 * i));
        b[2 * i] = (Bits)v.x;
        b[2 * i + 1] = (Bits)v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(w + e0 + 4 * i));
        b[4 * i] = (Bits)v.x;
        b[4 * i + 1] = (Bits)v.y;
        b[4 * i + 2] = (Bits)v.z;
        b[4 * i + 3] = (Bits)v.w;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < kSegV; ++i) {
      const long long e = e0 + i;
      if (sizeof(T) == 8) b[i] = e < M ? (Bits)__ldg(reinterpret_cast<const unsigned long long*>(w + e)) : (Bits)0;
      else b[i] = e < M ? (Bits)__ldg(reinterpret_cast<const unsigned*>(w + e)) : (Bits)0;
    }
  }
}

__device__ __forceinline__ void st_xf(unsigned long long* p, const xf& v) {
  p[0] = v.lo;
  p[1] = v.hi;
  p[2] = (unsigned long long)v.e;
}
__device__ __forceinline__ xf ld_xf(const unsigned long long* p) { return {p[0], p[1], (long long)p[2]}; }


// ---- exact segment sum (Eq. 3 at the segment level) -------------------------
// One warp, one 512-element segment: the segment exponent E (largest exponent
// field, at least 1) and the exact sum F of the weights on the grid
// 2^(E - bias - shift).  Raises ST_ENONFINITE for a negative, NaN or infinite
// weight.  Every lane returns the same F and E.
// Fixed-point value of a valid (non-negative, finite) binary64 on the grid
// 2^(E - 1075), in 32-bit operations: FixedTraits<double>::fixed restricted
// to valid inputs (m >> d is 0 for d >= 53).
__device__ __forceinline__ uint64_t fixed64_valid(uint64_t b, uint32_t E) {
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t t = hi >> 20;  // exponent field (the sign is 0)
  const uint32_t mh = (hi & 0xFFFFFu) | (t ? 0x100000u : 0u);
  const uint32_t d = E - (t ? t : 1u);
  // (mh:lo) >> d in two clamped funnel shifts
  const uint32_t d1 = min(d, 32u);
  const uint32_t xlo = __funnelshift_rc(lo, mh, d1);
  const uint32_t xhi = __funnelshift_rc(mh, 0u, d1);
  const uint32_t rlo = __funnelshift_rc(xlo, xhi, d - d1);
  return ((uint64_t)xhi << 32) | rlo;
}

// The exact segment sum F and exponent E described above; also the sums of
// this lane's elements in consecutive groups of kG (g[j]: elements kG j ..
// kG j + kG - 1 of b; the groups of all lanes add up to F).
template <typename T, int kG>
__device__ __forceinline__ void seg_sum_bits_groups(const typename FixedTraits<T>::Bits (&b)[kSegV], int lane,
                                                    int* status, uint64_t& F, uint32_t& E,
                                                    uint64_t (&g)[kSegV / kG]) {
  using Tr = FixedTraits<T>;
  // the largest sign+exponent field: below the all-ones exponent only when
  // every element is a non-negative finite number
  uint32_t tmax = 0;
#pragma unroll
  for (int i = 0; i < kSegV; ++i) tmax = max(tmax, Tr::top(b[i]));
  tmax = __reduce_max_sync(0xFFFFFFFFu, tmax);
  constexpr uint32_t kTopInf = sizeof(T) == 8 ? 0x7FFu : 0xFFu;
#pragma unroll
  for (int j = 0; j < kSegV / kG; ++j) g[j] = 0;
  if (tmax < kTopInf) {
    E = tmax > 1u ? tmax : 1u;
    if (sizeof(T) == 8) {
#pragma unroll
      for (int i = 0; i < kSegV; ++i) g[i / kG] += fixed64_valid((uint64_t)b[i], E);
    } else {
#pragma unroll
      for (int i = 0; i < kSegV; ++i) g[i / kG] += Tr::fixed(b[i], E);
    }
  } else {
    // rare: negative zeros (valid), or negative, NaN or infinite weights,
    // which add nothing and are reported
    uint32_t emax = 0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < kSegV; ++i) {
      emax = max(emax, seg_top<T>(b[i]));
      bad |= Tr::bad(b[i]);
    }
    emax = __reduce_max_sync(0xFFFFFFFFu, emax);
    E = emax > 1u ? emax : 1u;
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) raise_status(status, ST_ENONFINITE);
#pragma unroll
    for (int i = 0; i < kSegV; ++i) g[i / kG] += Tr::fixed(b[i], E);
  }
  uint64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kSegV / kG; ++j) sum += g[j];
  F = warp_sum_u64(sum);
}
template <typename T>
__device__ __forceinline__ void seg_sum_bits(const typename FixedTraits<T>::Bits (&b)[kSegV], int lane, int* status,
                                             uint64_t& F, uint32_t& E) {
  uint64_t g[1];
  seg_sum_bits_groups<T, kSegV>(b, lane, status, F, E, g);
}
template <typename T, bool kVec>
__device__ __forceinline__ void seg_sum(const T* __restrict__ w, long long base, long long M, int lane, int* status,
                                        uint64_t& F, uint32_t& E) {
  typename FixedTraits<T>::Bits b[kSegV];
  load_seg_striped<T, kVec>(w, base, M, lane, b);
  seg_sum_bits<T>(b, lane, status, F, E);
}

// A segment sum in grid units: F * 2^(E - Emax + kGridHead), truncated.
__device__ __forceinline__ u128 grid_value(unsigned long long F, int E, int Emax) {
  const int sh = E - Emax + kGridHead;
  uint64_t hi = 0, lo = F;
  if (sh >= 0) shl128(hi, lo, sh);
  else shr128(hi, lo, -sh);
  return u128{lo, hi};
}

// ---- spacings (Algorithm 1) ---------------------------------------------
constexpr int kZFrac = 88;  // spacing grid 2^-88

// -log v of the draw taken from Philox word x, exactly on the 2^-88 grid.
// Both draw formats go through the binary32-pair table logarithm (about
// 2^-45 relative): binary64 draws (2 (x >> 12) + 1) 2^-53 and binary32 draws
// (2 (x >> 41) + 1) 2^-24.  tab: the table, staged in shared memory.
template <bool F32>
__device__ __forceinline__ u128 spacing_fixed(uint64_t word, const LogTab* tab) {
  const df z = F32 ? neg_log_draw(2ULL * (word >> 41) + 1ULL, 24, *tab) : neg_log_draw(2ULL * (word >> 12) + 1ULL, 53, *tab);
  const u128 f = f_to_fixed128<kZFrac>(z.hi);
  return (z.lo >= 0.0f) ? u128_add(f, f_to_fixed128<kZFrac>(z.lo)) : u128_sub(f, f_to_fixed128<kZFrac>(-z.lo));
}
// ---- stratified and systematic points ----------------------------------------
// Schemes of the uniforms: Algorithm 1's sorted uniforms, or one point per
// stratum ((i-1)/N, i/N] -- U_i = (i-1+v_{i-1})/N (stratified) or
// (i-1+v_0)/N (systematic) -- the variants named in the paper's conclusion.
// The strata points reuse the spacing machinery unchanged: their "spacings"
//   s_0 = v'_0,  s_k = 1 + v'_k - v'_{k-1} (0 < k < N),  s_N = 1 - v'_{N-1}
// (v'_k = v_k stratified, v_0 systematic; all on the 2^-88 grid, exact) have
// the prefix sums Z_i = i - 1 + v'_{i-1} and Z_{N+1} = N, so the keys
// ceil(Z_i S / Z_{N+1}) are those of the strata points.
enum : int { kSchemeMultinomial = 0, kSchemeStratified = 1, kSchemeSystematic = 2 };
// Draw v of Philox word x on the 2^-88 grid (exact): binary64 draws
// (2 (x >> 12) + 1) 2^-53, binary32 draws (2 (x >> 41) + 1) 2^-24.
template <bool F32>
__device__ __forceinline__ u128 draw_fixed(uint64_t x) {
  if (F32) return u128{0ULL, 2ULL * (x >> 41) + 1ULL};  // (2m+1) 2^64
  const uint64_t m = 2ULL * (x >> 12) + 1ULL;           // < 2^53
  return u128{m << 35, m >> 29};                         // (2m+1) 2^35
}
__device__ __forceinline__ u128 strata_spacing(long long k, long long N, const u128& vk, const u128& vp) {
  const u128 one = {0ULL, 1ULL << 24};  // 1 on the 2^-88 grid
  if (k == 0) return vk;
  if (k >= N) return u128_sub(one, vp);
  return u128_sub(u128_add(one, vk), vp);
}

// Philox word k of the stream (seed, instance).
__device__ __forceinline__ uint64_t philox_word(unsigned long long seed, unsigned long long inst, long long k) {
  uint64_t words[4];
  philox4x64_10((uint64_t)(k / 4), 0ULL, 0ULL, 0ULL, seed, inst, words);
  const unsigned q = (unsigned)(k & 3);
  return q == 0 ? words[0] : q == 1 ? words[1] : q == 2 ? words[2] : words[3];
}
// Product of two xf, out of line: one copy of the 128x128-bit multiply for
// the scalar (once per call) paths.
static __device__ __noinline__ xf xf_mul_ool(xf a, xf b) { return xf_mul(a, b); }
// 1 / Z_{N+1} (Z_{N+1} > 0): a binary64 estimate of the reciprocal of the
// top 64 mantissa bits (relative error below 2^-51), then two Newton steps
// r <- r (2 - m r) on the 128-bit mantissa, each squaring the relative error
// (2^-51 -> 2^-102 -> the 2^-124 truncation floor of the products).  Integer
// work only, apart from the one estimate.
static __device__ __noinline__ xf recip_total(u128 t) {
  const xf m = xf_make(t.hi, t.lo, 0);  // t = (hi:lo) 2^e, top mantissa bit at 125
  const unsigned long long top = (m.hi << 2) | (m.lo >> 62);
  const double y = 1.0 / __ull2double_rn(top);  // ~ 2^-(62 + e) / m
  xf r = xf_from_f64_bits((uint64_t)__double_as_longlong(y));
  r.e -= 62 + m.e;
  const xf two = xf_from_u64(2, 0);
#pragma unroll 1
  for (int k = 0; k < 2; ++k) r = xf_mul_ool(r, xf_sub(two, xf_mul_ool(m, r)));
  return r;
}

// ---- one tile of the spacing scan ------------------------------------------
// 256 threads x 4 draws (one Philox block per thread): spacings on the 2^-88
// grid, exact 128-bit block scan, tiles chained by decoupled look-back on the
// tile index (tiles are numbered in the order they start, so a tile only
// waits on tiles that are already running).  Writes Z_1..Z_N, Z_{N+1} and
// 1/Z_{N+1}.  tab: the logarithm table in shared memory (binary64 draws).
constexpr int kUThreads = 256;
constexpr int kUWarps = kUThreads / kWarp;
constexpr int kUItems = 4;
static_assert(kUThreads * kUItems == kUTile, "uniform tile");

struct UniformTileSmem {
  u128 wsum[kUWarps];
  u128 woff[kUWarps];
};

// 1/Z_{N+1} as an xf, once per call by the thread that produced Z_{N+1}
// (out of line: binary64-pair division).
static __device__ __noinline__ void store_recip(unsigned long long* dst, u128 t) {
  const xf r = recip_total(t);
  dst[0] = r.lo;
  dst[1] = r.hi;
  dst[2] = (unsigned long long)r.e;
}

// The spacings of draws k0 .. k0+3 (one Philox block, words) under a scheme
// (N = ndraw - 1).  The stratified spacing of draw k also needs word k-1:
// the previous lane's last word, or the previous block's for lane 0.
template <bool F32>
__device__ __forceinline__ void block_spacings(int scheme, long long k0, long long ndraw, unsigned long long seed,
                                               unsigned long long inst, const uint64_t (&words)[4], const LogTab* tab,
                                               u128 (&f)[4]) {
  const long long N = ndraw - 1;
  if (scheme == kSchemeMultinomial) {
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = k0 + q < ndraw ? spacing_fixed<F32>(words[q], tab) : u128{0ULL, 0ULL};
    return;
  }
  u128 vprev;
  if (scheme == kSchemeSystematic) {
    uint64_t w0[4];
    philox4x64_10(0ULL, 0ULL, 0ULL, 0ULL, seed, inst, w0);
    vprev = draw_fixed<F32>(w0[0]);
#pragma unroll
    for (int q = 0; q < 4; ++q) f[q] = k0 + q < ndraw ? strata_spacing(k0 + q, N, vprev, vprev) : u128{0ULL, 0ULL};
    return;
  }
  uint64_t wp = __shfl_up_sync(0xFFFFFFFFu, words[3], 1);
  if ((threadIdx.x & 31) == 0 && k0 > 0) {
    uint64_t pw[4];
    philox4x64_10((uint64_t)(k0 / 4 - 1), 0ULL, 0ULL, 0ULL, seed, inst, pw);
    wp = pw[3];
  }
  vprev = draw_fixed<F32>(wp);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const u128 vk = draw_fixed<F32>(words[q]);
    f[q] = k0 + q < ndraw ? strata_spacing(k0 + q, N, vk, vprev) : u128{0ULL, 0ULL};
    vprev = vk;
  }
}

template <bool F32>
__device__ __forceinline__ void uniform_tile(long long tile, long long ndraw, unsigned long long seed,
                                             unsigned long long inst, u128* __restrict__ Z, u128* __restrict__ Ztot,
                                             PathConsts* consts, TileDesc<u128>* desc, int* status, int spin_limit,
                                             bool withhold_first, const LogTab* tab, UniformTileSmem& us,
                                             int scheme = kSchemeMultinomial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long k0 = tile * kUTile + (long long)threadIdx.x * kUItems;
  // the thread's four draws are the four words of one Philox block
  uint64_t words[4];
  philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, seed, inst, words);
  u128 pre[kUItems];  // thread-local inclusive prefixes
  u128 fq[kUItems];
  block_spacings<F32>(scheme, k0, ndraw, seed, inst, words, tab, fq);
  u128 run = {0ULL, 0ULL};
#pragma unroll
  for (int q = 0; q < kUItems; ++q) {
    run = u128_add(run, fq[q]);
    pre[q] = run;
  }
  const u128 incl = warp_incl_scan_v(run, lane);
  const u128 lane_off = u128_sub(incl, run);
  if (lane == 31) us.wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const u128 v = lane < kUWarps ? us.wsum[lane] : u128{0ULL, 0ULL};
    const u128 wi = warp_incl_scan_v(v, lane);
    const u128 agg = shfl_v(wi, kUWarps - 1);
    u128 excl = {0ULL, 0ULL};
    if (tile == 0) {
      if (lane == 0 && !withhold_first) lb_publish(desc, 0, agg, true);
    } else {
      if (lane == 0) lb_publish(desc, tile, agg, false);
      excl = lb_exclusive(desc, tile, lane, spin_limit, status);
      if (lane == 0) lb_publish_inc(desc, tile, u128_add(excl, agg));
    }
    if (lane < kUWarps) us.woff[lane] = u128_add(excl, u128_sub(wi, v));
  }
  __syncthreads();
  const u128 off = u128_add(us.woff[warp], lane_off);
#pragma unroll
  for (int q = 0; q < kUItems; ++q) {
    const long long k = k0 + q;
    if (k < ndraw - 1) {
      Z[k] = u128_add(off, pre[q]);
    } else if (k == ndraw - 1) {
      const u128 t = u128_add(off, pre[q]);
      *Ztot = t;
      store_recip(consts->invZ, t);
    }
  }
}

// ---- map keys and in-segment decisions ---------------------------------------
__device__ __forceinline__ bool u128_lt(const u128& a, const u128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
// key = ceil(Z_i * c) with c = S_grid / Z_{N+1}: U_i * S in grid units,
// rounded up (so that "prefix >= key" is "W >= U").  Exact: the 256-bit
// product of c's mantissa and Z_i, shifted by c's (call-uniform) exponent,
// plus one when any bit below the unit is set.
__device__ __forceinline__ u128 map_key(const xf& c, u128 z) {
  if (xf_zero(c) || (z.hi | z.lo) == 0) return u128{0ULL, 0ULL};
  uint64_t p0h, p0l, p1h, p1l, p2h, p2l, p3h, p3l;
  mul64(c.lo, z.lo, p0h, p0l);
  mul64(c.lo, z.hi, p1h, p1l);
  mul64(c.hi, z.lo, p2h, p2l);
  mul64(c.hi, z.hi, p3h, p3l);
  // P = w3:w2:w1:w0
  const uint64_t w0 = p0l;
  uint64_t w1 = p0h + p1l;
  uint64_t c1 = w1 < p0h;
  w1 += p2l;
  c1 += w1 < p2l;
  uint64_t w2 = p3l + p1h;
  uint64_t c2 = w2 < p3l;
  w2 += p2h;
  c2 += w2 < p2h;
  w2 += c1;
  c2 += w2 < c1;
  const uint64_t w3 = p3h + c2;
  if (c.e >= 0) {  // key = P << e, below 2^126: only small products (e <= 1)
    const int e = c.e > 2 ? 2 : (int)c.e;
    uint64_t hi = w1, lo = w0;
    shl128(hi, lo, e);
    return u128{lo, hi};
  }
  const long long k = -c.e;  // key = ceil(P / 2^k)
  if (k >= 256) return u128{1ULL, 0ULL};
  const int j = (int)(k >> 6), b = (int)(k & 63);
  // the 192 bits from word j up, and whether any bit below bit k is set
  uint64_t a0, a1, a2;
  bool frac;
  if (j == 0) {
    a0 = w0; a1 = w1; a2 = w2;
    frac = (w0 & ((1ULL << b) - 1ULL)) != 0;
  } else if (j == 1) {
    a0 = w1; a1 = w2; a2 = w3;
    frac = w0 != 0 || (w1 & ((1ULL << b) - 1ULL)) != 0;
  } else if (j == 2) {
    a0 = w2; a1 = w3; a2 = 0;
    frac = (w0 | w1) != 0 || (w2 & ((1ULL << b) - 1ULL)) != 0;
  } else {
    a0 = w3; a1 = 0; a2 = 0;
    frac = (w0 | w1 | w2) != 0 || (w3 & ((1ULL << b) - 1ULL)) != 0;
  }
  uint64_t lo = b ? (a0 >> b) | (a1 << (64 - b)) : a0;
  uint64_t hi = b ? (a1 >> b) | (a2 << (64 - b)) : a1;
  lo += frac ? 1ULL : 0ULL;
  if (frac && lo == 0) ++hi;
  return u128{lo, hi};
}

// K = ceil(rem / 2^sh) clamped to [1, F]: the segment-grid target of a key
// that lies rem grid units above the segment's start.
__device__ __forceinline__ unsigned long long ceil_units(u128 rem, int sh, unsigned long long F) {
  if (u128_is_zero(rem)) return 1;
  unsigned long long K;
  if (sh >= 0) {
    if (sh >= 128) {
      K = 1;
    } else {
      uint64_t ah = 0, al = 0;  // 2^sh - 1
      if (sh >= 64) {
        ah = (sh == 64) ? 0 : ((1ULL << (sh - 64)) - 1);
        al = ~0ULL;
      } else {
        al = (1ULL << sh) - 1;
      }
      uint64_t nl = rem.lo + al;
      uint64_t nh = rem.hi + ah + (nl < rem.lo ? 1ULL : 0ULL);
      shr128(nh, nl, sh);
      K = nh ? F : nl;
    }
  } else {
    // rem * 2^-sh; anything at or above 2^63 is past F anyway
    const int ls = -sh;
    K = (rem.hi || ls >= 63 || (rem.lo >> (63 - ls))) ? F : (rem.lo << ls);
  }
  if (K > F) K = F;
  if (K < 1) K = 1;
  return K;
}

// Exact inclusive prefixes of a segment on its own grid, lane-major (lane l
// holds elements 16 l .. 16 l + 15): pref[q] = sum of fixed values up to that
// element.  Non-decreasing across the warp.
template <typename T>
__device__ __forceinline__ void seg_prefixes(const typename FixedTraits<T>::Bits (&b)[kSegV], uint32_t E, int lane,
                                             uint64_t (&pref)[kSegV]) {
  uint64_t run = 0;
#pragma unroll
  for (int q = 0; q < kSegV; ++q) {
    run += FixedTraits<T>::fixed(b[q], E);
    pref[q] = run;
  }
  const uint64_t off = warp_incl_scan_u64(run, lane) - run;
#pragma unroll
  for (int q = 0; q < kSegV; ++q) pref[q] += off;
}

}  // namespace gbr
