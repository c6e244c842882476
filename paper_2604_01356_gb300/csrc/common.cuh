// Device building blocks shared by the resampling kernels (sm_103a).
//
// Arithmetic policy.  On GB300 binary64 add/mul/fma issue at ~1.8 per clock
// per SM (about 1/66 of binary32) and the binary64 log is far slower still,
// so nothing here spends binary64 work per weight or per draw on the bulk
// path.  Weights are summed EXACTLY as 64-bit fixed-point integers inside
// 512-element segments (one segment per warp, one shared exponent per
// segment); only segment-level quantities use binary64 (as double-double
// pairs).  Spacings -log(v) are evaluated with binary32 pairs and summed as
// exact 64/128-bit integers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbr {

// Status codes; the numeric values are those of rs_status in gbresample.h.
enum : int { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENONFINITE = 4, ST_EZEROSUM = 5, ST_ETIMEOUT = 6 };

// First error wins.
__device__ __forceinline__ void raise_status(int* status, int code) { atomicCAS(status, 0, code); }

constexpr int kWarp = 32;
constexpr int kSegV = 16;                 // elements per lane in a segment
constexpr int kSeg = kWarp * kSegV;       // 512 elements per segment (one warp)
static_assert(kSeg == 512, "segment length is shared with the host (kSegLen)");

// ---------------------------------------------------------------------------
// Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Multipliers and Weyl
// key increments are the published Philox-4x64 constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                              uint64_t k1, uint64_t out[4]) {
  const uint64_t mA = 0xD2E7470EE14C6C93ULL, mB = 0xCA5A826395121157ULL;
  const uint64_t wA = 0x9E3779B97F4A7C15ULL, wB = 0xBB67AE8584CAA73BULL;
#pragma unroll 1
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += wA;
      k1 += wB;
    }
    const uint64_t hiA = __umul64hi(mA, c0), loA = mA * c0;
    const uint64_t hiB = __umul64hi(mB, c2), loB = mB * c2;
    const uint64_t n0 = hiB ^ c1 ^ k0;
    const uint64_t n2 = hiA ^ c3 ^ k1;
    c0 = n0;
    c1 = loB;
    c2 = n2;
    c3 = loA;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// ---------------------------------------------------------------------------
// binary32 pair ("df") arithmetic: error-free transforms (Knuth TwoSum,
// Dekker FastTwoSum, FMA-based TwoProduct).
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  df t = df_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_fast_two_sum(p, e);
}

// ---------------------------------------------------------------------------
// -log(v) for a draw v = X * 2^-p (X odd, 0 < v < 1), in binary32-pair
// arithmetic, relative error about 2^-45.  Table-driven method (P. T. P. Tang,
// "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16(4), 1990):
//   v = 2^-e * m, m in [1/2, 1);  c = 1 - k/256 is the table point nearest m;
//   log m = log c + log1p(r),  r = (m - c)/c,  |r| <= 2^-8;
//   log1p(r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 - r^6/6 (truncation < 2^-56).
// m - c is formed exactly in integer arithmetic; -log c and 1/c come from a
// 129-entry table of binary32 pairs built on the host from the C library's
// binary64 log.  Callers stage the table in shared memory.
// ---------------------------------------------------------------------------
struct LogTab {
  float2 nlogc[129];  // -log(1 - k/256) as (hi, lo)
  float2 invc[129];   // 1/(1 - k/256) as (hi, lo)
};

// X: 1 <= X < 2^p, p <= 62.  Returns -log(X * 2^-p) as a binary32 pair.
__device__ __forceinline__ df neg_log_draw(uint64_t X, int p, const LogTab& T) {
  // normalise so the top bit of X sits at bit 62: m = Xn * 2^-63 in [1/2, 1)
  const int lz = __clzll(X) - 1;  // X < 2^63
  const uint64_t Xn = X << lz;
  const int e = p - 63 + lz;  // v = m * 2^-e, e >= 0
  // D = (1 - m) * 2^63, exact, 0 < D <= 2^62
  const uint64_t D = (1ULL << 63) - Xn;
  // k = round(256 * (1 - m)), c = 1 - k/256
  const int k = (int)((D + (1ULL << 54)) >> 55);
  // m - c = (k * 2^55 - D) * 2^-63, |.| <= 2^54: exact signed integer
  const int64_t R = (int64_t)((uint64_t)k << 55) - (int64_t)D;
  // R as a binary32 pair scaled by 2^-63, from two 32-bit integer conversions:
  // R = Rh*2^30 + Rl, |Rh| <= 2^24 (exact), 0 <= Rl < 2^30 (rounded to 24
  // bits), so the pair holds R to 2^-48 relative.
  const int32_t Rh = (int32_t)(R >> 30);
  const int32_t Rl = (int32_t)(R & ((1LL << 30) - 1));
  const df mc = df_two_sum(__fmul_rn(__int2float_rn(Rh), 0x1p-33f), __fmul_rn(__int2float_rn(Rl), 0x1p-63f));
  const float2 ic = T.invc[k];
  const df r = df_mul(mc, df{ic.x, ic.y});
  // log1p(r): r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6)
  const float rh = r.hi;
  const float p3 = __fmaf_rn(__fmaf_rn(__fmaf_rn(rh, -1.0f / 6.0f, 0.2f), rh, -0.25f), rh, 1.0f / 3.0f);
  const float r3 = __fmul_rn(__fmul_rn(rh, rh), rh);
  const float tail = __fmul_rn(r3, p3);
  const df r2 = df_mul(r, r);
  df lp = df_add(r, df{-0.5f * r2.hi, -0.5f * r2.lo});
  lp = df_add(lp, df{tail, 0.0f});
  // -log v = e*ln2 - log c - log1p(r).  ln2 = L0 + L1 + L2 with L0 holding 16
  // significant bits, so e*L0 is exact for e < 2^8; e*L1 is split exactly by FMA.
  const float L0 = 0x1.62e4p-1f, L1 = 0x1.7f7d1cp-20f, L2 = 0x1.ef357ap-45f;
  const float ef = (float)e;
  const float p1 = __fmul_rn(ef, L1);
  const float p1e = __fmaf_rn(ef, L1, -p1);
  df acc = df_two_sum(__fmul_rn(ef, L0), p1);
  acc.lo = __fadd_rn(acc.lo, __fmaf_rn(ef, L2, p1e));
  acc = df_fast_two_sum(acc.hi, acc.lo);
  const float2 nl = T.nlogc[k];
  acc = df_add(acc, df{nl.x, nl.y});
  acc = df_add(acc, df{-lp.hi, -lp.lo});
  return acc;
}

// ---------------------------------------------------------------------------
// binary64 pair ("dd") arithmetic, used only per segment / per sample.
// ---------------------------------------------------------------------------
struct dd {
  double hi, lo;
};
__device__ __forceinline__ dd dd_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd dd_fast(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = dd_two_sum(a.hi, b.hi);
  dd t = dd_two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = dd_fast(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return dd_fast(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd{-b.hi, -b.lo}); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  double p = __dmul_rn(a.hi, b.hi);
  double e = __fma_rn(a.hi, b.hi, -p);
  e = __fma_rn(a.hi, b.lo, e);
  e = __fma_rn(a.lo, b.hi, e);
  return dd_fast(p, e);
}
// a / b with one correction step (~2^-100 relative).
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  double q1 = __ddiv_rn(a.hi, b.hi);
  dd p = dd_mul(dd{q1, 0.0}, b);
  dd r = dd_sub(a, p);
  double q2 = __ddiv_rn(r.hi, b.hi);
  return dd_fast(q1, q2);
}
// dd + binary64 (for exact-ish prefixes of binary64 weights).
__device__ __forceinline__ dd dd_add_d(dd a, double b) {
  dd s = dd_two_sum(a.hi, b);
  s.lo = __dadd_rn(s.lo, a.lo);
  return dd_fast(s.hi, s.lo);
}
__device__ __forceinline__ bool dd_lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool dd_le(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// x * 2^k for any k in [-2200, 2200] without intermediate overflow/underflow
// surprises (binary64 op per call; used per segment only).
__device__ __forceinline__ double ldexp2(double x, int k) { return scalbn(x, k); }

// Exact value of an unsigned integer F <= 2^63 times 2^k as a dd pair.
__device__ __forceinline__ dd u64_scaled_dd(uint64_t F, int k) {
  const double hi = __ull2double_rn(F);
  // F - hi is an exact signed integer (|.| <= 2^10) since hi is F rounded
  const long long rem = (long long)(F - (uint64_t)hi);
  return {ldexp2(hi, k), ldexp2((double)rem, k)};
}

// Unsigned 128-bit integer (exact sums of fixed-point spacings).
struct u128 {
  uint64_t lo, hi;
};
__device__ __forceinline__ u128 u128_add(u128 a, u128 b) {
  u128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ULL : 0ULL);
  return r;
}
__device__ __forceinline__ u128 u128_add64(u128 a, uint64_t b) {
  u128 r;
  r.lo = a.lo + b;
  r.hi = a.hi + (r.lo < a.lo ? 1ULL : 0ULL);
  return r;
}
__device__ __forceinline__ u128 u128_sub(u128 a, u128 b) {
  u128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ULL : 0ULL);
  return r;
}
__device__ __forceinline__ bool u128_is_zero(u128 a) { return (a.lo | a.hi) == 0; }

// Monotone 64-bit search key of a 128-bit unsigned integer: position of the
// leading bit (7 bits) then the next 57 bits.  Keeps relative precision for
// small values, unlike the high word alone.
__device__ __forceinline__ unsigned long long u128_key(u128 a) {
  if (u128_is_zero(a)) return 0ULL;
  const int lz = a.hi ? __clzll(a.hi) : 64 + __clzll(a.lo);
  uint64_t h = a.hi, l = a.lo;
  if (lz < 64) {
    if (lz) h = (h << lz) | (l >> (64 - lz));
  } else {
    h = l << (lz - 64);
  }
  // h has its leading bit at 63: drop it, keep 57 bits below it
  return ((unsigned long long)(128 - lz) << 57) | ((h << 1) >> 7);
}

// Bit pattern of the binary64 nearest to a 128-bit unsigned integer (round
// half to even), integer operations only.
__device__ __forceinline__ uint64_t u128_to_f64_bits(u128 a) {
  if (u128_is_zero(a)) return 0;
  const int lz = a.hi ? __clzll(a.hi) : 64 + __clzll(a.lo);
  uint64_t h, l;  // a << lz
  if (lz == 0) {
    h = a.hi; l = a.lo;
  } else if (lz < 64) {
    h = (a.hi << lz) | (a.lo >> (64 - lz)); l = a.lo << lz;
  } else {
    h = a.lo << (lz - 64); l = 0;
  }
  uint64_t mant = h >> 11;
  const uint64_t rb = h & 0x7FF;
  if (rb > 0x400 || (rb == 0x400 && (l != 0 || (mant & 1)))) ++mant;
  int e = 127 - lz;
  if (mant >> 53) { mant >>= 1; ++e; }
  return ((uint64_t)(e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFULL);
}
// Same for binary32 (the integers here are below 2^127).
__device__ __forceinline__ uint32_t u128_to_f32_bits(u128 a) {
  if (u128_is_zero(a)) return 0;
  const int lz = a.hi ? __clzll(a.hi) : 64 + __clzll(a.lo);
  uint64_t h, l;
  if (lz == 0) {
    h = a.hi; l = a.lo;
  } else if (lz < 64) {
    h = (a.hi << lz) | (a.lo >> (64 - lz)); l = a.lo << lz;
  } else {
    h = a.lo << (lz - 64); l = 0;
  }
  uint32_t mant = (uint32_t)(h >> 40);
  const uint64_t rb = h & 0xFFFFFFFFFFULL;
  const uint64_t half = 1ULL << 39;
  if (rb > half || (rb == half && (l != 0 || (mant & 1)))) ++mant;
  int e = 127 - lz;
  if (mant >> 24) { mant >>= 1; ++e; }
  return ((uint32_t)(e + 127) << 23) | (mant & 0x7FFFFFu);
}
// Exact widening of a binary32 (finite, non-negative, normal or zero) to binary64 bits.
__device__ __forceinline__ uint64_t f32_to_f64_bits(uint32_t b) {
  if ((b & 0x7FFFFFFFu) == 0) return 0;
  const uint64_t e = (b >> 23) & 0xFF, m = b & 0x7FFFFFu;
  return ((e + 896) << 52) | (m << 29);
}

// Non-negative binary32 x times 2^frac rounded to an unsigned 128-bit integer.
template <int kFrac>
__device__ __forceinline__ u128 f_to_fixed128(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xFF);
  const uint64_t m = (b & 0x7FFFFFu) | (e ? 0x800000u : 0u);
  if (!e) e = 1;
  const int sh = e - 150 + kFrac;  // x * 2^frac = m * 2^sh
  u128 r = {0ULL, 0ULL};
  if (sh >= 64) {
    r.hi = m << (sh - 64);
  } else if (sh > 0) {
    r.lo = m << sh;
    r.hi = m >> (64 - sh);
  } else if (sh == 0) {
    r.lo = m;
  } else if (sh > -40) {
    const int rs = -sh;
    r.lo = (m + (1ULL << (rs - 1))) >> rs;
  }
  return r;
}

// Nearest binary64 of a 128-bit integer (round to nearest even), by integer
// operations plus one exact scaling.
__device__ __forceinline__ double u128_to_double(u128 a) {
  if (a.hi == 0) return __ull2double_rn(a.lo);
  const int lz = __clzll(a.hi);
  // top 64 bits of the normalised value, plus a sticky bit for the rest
  const uint64_t top = lz ? ((a.hi << lz) | (a.lo >> (64 - lz))) : a.hi;
  const uint64_t rest = a.lo << lz;  // bits below top
  // binary64 keeps 53 bits of top; round half to even with rest as sticky
  const uint64_t mant = top >> 11;
  const uint64_t rbits = top & 0x7FF;
  uint64_t m = mant;
  if (rbits > 0x400 || (rbits == 0x400 && (rest != 0 || (mant & 1)))) m += 1;
  // value = m * 2^(64 - lz + 11) ; m may have become 2^53
  return ldexp2((double)m, 64 - lz + 11);
}

// ---------------------------------------------------------------------------
// "xf": a non-negative number m * 2^e with a 128-bit integer mantissa, kept
// normalised (top bit of m at bit 125, two bits of headroom, or m == 0).
// All operations are integer instructions; additions truncate below 2^-125
// of the larger operand.  Used for every prefix above the segment level, so
// no binary64 instruction is spent per segment or per sample.
// ---------------------------------------------------------------------------
struct xf {
  uint64_t lo, hi;
  long long e;
};
constexpr int kXfTop = 125;
constexpr long long kXfZeroE = -(1LL << 40);

__device__ __forceinline__ int clz128(uint64_t hi, uint64_t lo) { return hi ? __clzll(hi) : 64 + __clzll(lo); }
__device__ __forceinline__ void shl128(uint64_t& hi, uint64_t& lo, int k) {  // 0 <= k < 128
  if (k == 0) return;
  if (k >= 64) {
    hi = lo << (k - 64);
    lo = 0;
  } else {
    hi = (hi << k) | (lo >> (64 - k));
    lo <<= k;
  }
}
__device__ __forceinline__ void shr128(uint64_t& hi, uint64_t& lo, int k) {  // k >= 0
  if (k == 0) return;
  if (k >= 128) {
    hi = lo = 0;
  } else if (k >= 64) {
    lo = hi >> (k - 64);
    hi = 0;
  } else {
    lo = (lo >> k) | (hi << (64 - k));
    hi >>= k;
  }
}
__device__ __forceinline__ bool xf_zero(const xf& a) { return (a.hi | a.lo) == 0; }
__device__ __forceinline__ xf xf_make(uint64_t hi, uint64_t lo, long long e) {
  if ((hi | lo) == 0) return {0, 0, kXfZeroE};
  const int sh = kXfTop - (127 - clz128(hi, lo));
  if (sh > 0) shl128(hi, lo, sh);
  else if (sh < 0) shr128(hi, lo, -sh);
  return {lo, hi, e - sh};
}
__device__ __forceinline__ xf xf_from_u64(uint64_t F, long long e) { return xf_make(0, F, e); }
// exact value of a finite non-negative binary64 (bit pattern b)
__device__ __forceinline__ xf xf_from_f64_bits(uint64_t b) {
  const int ex = (int)((b >> 52) & 0x7FF);
  uint64_t m = b & 0xFFFFFFFFFFFFFULL;
  if (ex) m |= 1ULL << 52;
  return xf_from_u64(m, (long long)(ex ? ex : 1) - 1075);
}
__device__ __forceinline__ xf xf_add(xf a, xf b) {
  if (xf_zero(a)) return b;
  if (xf_zero(b)) return a;
  if (a.e < b.e) {
    const xf t = a;
    a = b;
    b = t;
  }
  const long long d = a.e - b.e;
  uint64_t bh = b.hi, bl = b.lo;
  shr128(bh, bl, d > 127 ? 128 : (int)d);
  uint64_t lo = a.lo + bl;
  uint64_t hi = a.hi + bh + (lo < a.lo ? 1ULL : 0ULL);
  long long e = a.e;
  if (hi >> 62) {  // top bit reached 126
    shr128(hi, lo, 1);
    ++e;
  }
  return {lo, hi, e};
}
// a - b for a >= b
__device__ __forceinline__ xf xf_sub(xf a, xf b) {
  if (xf_zero(b)) return a;
  const long long d = a.e - b.e;
  if (d < 0) return {0, 0, kXfZeroE};
  uint64_t bh = b.hi, bl = b.lo;
  shr128(bh, bl, d > 127 ? 128 : (int)d);
  if (bh > a.hi || (bh == a.hi && bl > a.lo)) return {0, 0, kXfZeroE};
  const uint64_t lo = a.lo - bl;
  const uint64_t hi = a.hi - bh - (a.lo < bl ? 1ULL : 0ULL);
  return xf_make(hi, lo, a.e);
}
__device__ __forceinline__ bool xf_lt(const xf& a, const xf& b) {
  if (xf_zero(a)) return !xf_zero(b);
  if (xf_zero(b)) return false;
  if (a.e != b.e) return a.e < b.e;
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ bool xf_le(const xf& a, const xf& b) { return !xf_lt(b, a); }

// 64x64 -> 128
__device__ __forceinline__ void mul64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
  lo = a * b;
  hi = __umul64hi(a, b);
}
// Product of two normalised xf (top 128 bits of the 256-bit mantissa product).
__device__ __forceinline__ xf xf_mul(const xf& a, const xf& b) {
  if (xf_zero(a) || xf_zero(b)) return {0, 0, kXfZeroE};
  uint64_t p0h, p0l, p1h, p1l, p2h, p2l, p3h, p3l;
  mul64(a.lo, b.lo, p0h, p0l);
  mul64(a.lo, b.hi, p1h, p1l);
  mul64(a.hi, b.lo, p2h, p2l);
  mul64(a.hi, b.hi, p3h, p3l);
  // r = p3<<128 + (p1+p2)<<64 + p0, as words r3 r2 r1 (r0 dropped)
  uint64_t r1 = p0h + p1l;
  uint64_t c1 = r1 < p0h;
  r1 += p2l;
  c1 += r1 < p2l;
  uint64_t r2 = p3l + p1h;
  uint64_t c2 = r2 < p3l;
  r2 += p2h;
  c2 += r2 < p2h;
  r2 += c1;
  c2 += r2 < c1;
  const uint64_t r3 = p3h + c2;
  // product < 2^252: keep bits 126..253
  const uint64_t hi = (r3 << 2) | (r2 >> 62);
  const uint64_t lo = (r2 << 2) | (r1 >> 62);
  return xf_make(hi, lo, a.e + b.e + 126);
}
// xf times an unsigned 64-bit integer (truncated to 128 significant bits).
__device__ __forceinline__ xf xf_mul_u64(const xf& a, uint64_t F) {
  if (xf_zero(a) || F == 0) return {0, 0, kXfZeroE};
  uint64_t ph, pl, qh, ql;
  mul64(a.lo, F, ph, pl);
  mul64(a.hi, F, qh, ql);
  // 192-bit product: w2 w1 w0 = (qh, ql + ph, pl)
  uint64_t w1 = ql + ph;
  const uint64_t w2 = qh + (w1 < ql ? 1ULL : 0ULL);
  // keep the top 128 bits below the leading bit of w2:w1:w0
  const int lz = w2 ? __clzll(w2) : 64 + __clzll(w1);
  uint64_t hi, lo;
  long long e = a.e;
  if (lz >= 64) {  // w2 == 0: the product fits in w1:w0
    hi = w1;
    lo = pl;
  } else {  // keep bits (64-lz) .. (191-lz) of the product
    hi = (w2 << lz) | (lz ? (w1 >> (64 - lz)) : 0);
    lo = (w1 << lz) | (lz ? (pl >> (64 - lz)) : 0);
    e += 64 - lz;
  }
  return xf_make(hi, lo, e);
}
// xf times an unsigned 128-bit integer.
__device__ __forceinline__ xf xf_mul_u128(const xf& a, u128 z) {
  return xf_mul(a, xf_make(z.hi, z.lo, 0));
}

// Bit pattern of the binary64 nearest to x (round half to even).
__device__ __forceinline__ uint64_t xf_to_f64_bits(const xf& x) {
  if (xf_zero(x)) return 0;
  long long be = x.e + kXfTop + 1023;  // biased exponent of the leading bit
  int drop = 73;                        // bits below the 53-bit significand
  if (be < 1) {                         // subnormal result
    drop += (int)(1 - be);
    be = 0;
    if (drop >= 128) return 0;
  }
  uint64_t mh = x.hi, ml = x.lo;
  shr128(mh, ml, drop);                 // kept significand (fits in 64 bits)
  uint64_t rh = x.hi, rl = x.lo;        // dropped part
  uint64_t kh = mh, kl = ml;
  shl128(kh, kl, drop);
  rl = x.lo - kl;
  rh = x.hi - kh - (x.lo < kl ? 1ULL : 0ULL);
  uint64_t half_h = 0, half_l = 0;
  if (drop - 1 >= 64) half_h = 1ULL << (drop - 1 - 64);
  else half_l = 1ULL << (drop - 1);
  uint64_t m = ml;
  const bool gt = rh > half_h || (rh == half_h && rl > half_l);
  const bool eq = rh == half_h && rl == half_l;
  if (gt || (eq && (m & 1))) ++m;
  if (be == 0) {
    return m;  // subnormal (a carry into bit 52 correctly yields the smallest normal)
  }
  if (m >> 53) {
    m >>= 1;
    ++be;
  }
  if (be >= 2047) return 0x7FF0000000000000ULL;
  return ((uint64_t)be << 52) | (m & 0xFFFFFFFFFFFFFULL);
}

// Search key of x: the bit pattern of x truncated to binary64 (a monotone
// map; values below the binary64 normal range all map to 0).  Cheap: no
// rounding logic.
__device__ __forceinline__ unsigned long long xf_key(const xf& x) {
  if (xf_zero(x)) return 0ULL;
  const long long be = x.e + kXfTop + 1023;
  if (be < 1) return 0ULL;
  if (be >= 2047) return 0x7FF0000000000000ULL;
  return ((unsigned long long)be << 52) | ((x.hi >> 9) & 0xFFFFFFFFFFFFFULL);
}

// x as a binary64 pair (hi nearest, lo = nearest of the signed remainder).
__device__ __forceinline__ dd xf_to_dd(const xf& x) {
  const uint64_t hb = xf_to_f64_bits(x);
  const double hi = __longlong_as_double((long long)hb);
  const xf h = xf_from_f64_bits(hb);
  if (xf_lt(x, h)) {
    const xf r = xf_sub(h, x);
    return {hi, -__longlong_as_double((long long)xf_to_f64_bits(r))};
  }
  const xf r = xf_sub(x, h);
  return {hi, __longlong_as_double((long long)xf_to_f64_bits(r))};
}
// a / b for normalised non-zero xf, on one thread: the mantissas are divided
// as binary64 pairs scaled to [1, 2) (so nothing over- or underflows) and the
// exponent difference is carried in the integer exponent.
__device__ __forceinline__ xf xf_from_dd(dd v);
__device__ __forceinline__ xf xf_div(const xf& a, const xf& b) {
  if (xf_zero(a) || xf_zero(b)) return {0, 0, kXfZeroE};
  const dd ad = xf_to_dd(xf{a.lo, a.hi, -kXfTop});
  const dd bd = xf_to_dd(xf{b.lo, b.hi, -kXfTop});
  xf q = xf_from_dd(dd_div(ad, bd));
  q.e += a.e - b.e;
  return q;
}

// positive binary64 pair to xf (hi > 0, |lo| <= ulp(hi)/2)
__device__ __forceinline__ xf xf_from_dd(dd v) {
  const xf h = xf_from_f64_bits((uint64_t)__double_as_longlong(v.hi));
  if (v.lo >= 0.0) return xf_add(h, xf_from_f64_bits((uint64_t)__double_as_longlong(v.lo)));
  return xf_sub(h, xf_from_f64_bits((uint64_t)__double_as_longlong(-v.lo)));
}

// ---------------------------------------------------------------------------
// Fixed-point segment arithmetic for binary64 / binary32 weights.
// An element with exponent field t and significand m (implicit bit included,
// e' = max(t,1)) has value m * 2^(e' - kBias).  Inside a segment of shared
// exponent E = max e' it becomes the integer
//   F = floor((m << kShift) / 2^(E - e'))        (truncating grid)
// with unit 2^(E - kBias - kShift).  The largest element keeps every bit and
// 512 elements sum below 2^63, so every segment sum and every within-segment
// prefix is an exact uint64.  Invalid elements (negative, NaN, infinity) have
// t >= 0x7FF (the sign bit lands in t), so E - e' wraps to a huge shift and
// they contribute 0 without a branch; they are reported separately.
// ---------------------------------------------------------------------------
template <typename T>
struct FixedTraits;
template <>
struct FixedTraits<double> {
  using Bits = uint64_t;
  static constexpr int kBias = 1075;
  static constexpr int kShift = 0;  // m < 2^53: 512 of them stay below 2^62
  __device__ static __forceinline__ uint32_t top(Bits b) { return (uint32_t)(b >> 52); }  // sign + exponent
  __device__ static __forceinline__ uint32_t valid_top(Bits b) { return (uint32_t)(b >> 52) < 0x7FFu; }
  // precise invalidity (negative non-zero, NaN, infinity); -0.0 is a valid zero
  __device__ static __forceinline__ bool bad(Bits b) {
    return ((b >> 52) & 0x7FF) == 0x7FF || ((b >> 63) && (b << 1) != 0);
  }
  __device__ static __forceinline__ uint64_t fixed(Bits b, uint32_t E) {
    const uint32_t t = top(b);
    const uint64_t m = (b & 0xFFFFFFFFFFFFFULL) | (t ? (1ULL << 52) : 0ULL);
    uint32_t d = E - (t > 1u ? t : 1u);
    d = d > 63u ? 63u : d;
    return m >> d;
  }
  __device__ static __forceinline__ double value(Bits b) { return __longlong_as_double((long long)b); }
};
template <>
struct FixedTraits<float> {
  using Bits = uint32_t;
  static constexpr int kBias = 150;
  static constexpr int kShift = 30;  // m < 2^24 -> m<<30 < 2^54
  __device__ static __forceinline__ uint32_t top(Bits b) { return b >> 23; }
  __device__ static __forceinline__ uint32_t valid_top(Bits b) { return (b >> 23) < 0xFFu; }
  __device__ static __forceinline__ bool bad(Bits b) { return ((b >> 23) & 0xFF) == 0xFF || ((b >> 31) && (b << 1) != 0); }
  __device__ static __forceinline__ uint64_t fixed(Bits b, uint32_t E) {
    const uint32_t t = top(b);
    const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | (t ? 0x800000u : 0u)) << 30;
    uint32_t d = E - (t > 1u ? t : 1u);
    d = d > 63u ? 63u : d;
    return m >> d;
  }
};

// Segment exponent candidate of one element: its exponent field when it is a
// valid non-negative finite number, else 0 (max with 1 is applied later).
template <typename T>
__device__ __forceinline__ uint32_t seg_top(typename FixedTraits<T>::Bits b) {
  using Tr = FixedTraits<T>;
  const uint32_t t = Tr::top(b);
  return t < (sizeof(T) == 8 ? 0x7FFu : 0xFFu) ? t : 0u;
}
template <typename T>
__device__ __forceinline__ uint64_t to_fixed(typename FixedTraits<T>::Bits b, int E) {
  return FixedTraits<T>::fixed(b, (uint32_t)E);
}

// A segment is a "head" segment when everything before it is too small for
// the segment grid to keep 1e-12 relative accuracy on the prefixes inside it:
// the within-segment truncation is below 512 units, so P_s >= 2^50 units is
// enough.  Head segments of binary64 weights are resolved with exact
// per-element prefixes instead (only the first segment for ordinary weights).
__device__ __forceinline__ bool head_segment(const xf& P, int E, int bias_shift) {
  return xf_zero(P) || P.e + kXfTop < (long long)(E - bias_shift + 50);
}

// ---------------------------------------------------------------------------
// Warp helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}
// inclusive scan across the warp
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Decoupled look-back (Merrill & Garland, "Single-pass parallel prefix scan
// with decoupled look-back", 2016) over per-tile aggregates of type V.  Tiles
// obtain their index from an atomic counter in launch order, so a tile only
// ever waits on tiles that are already running.  Every wait is bounded:
// after `spin_limit` polls the tile records ST_ETIMEOUT, treats the missing
// predecessor as zero and carries on, so the kernel always terminates.
// ---------------------------------------------------------------------------
enum : uint32_t { kFlagEmpty = 0, kFlagAgg = 1, kFlagInc = 2 };

template <typename V>
struct alignas(16) TileDesc {
  uint32_t flag;
  uint32_t pad[3];
  V agg;
  V inc;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename V>
__device__ __forceinline__ V ld_cg(const V* p) {
  // values are read only after an acquire of their flag; bypass L1
  V v;
  const uint64_t* s = reinterpret_cast<const uint64_t*>(p);
  uint64_t* d = reinterpret_cast<uint64_t*>(&v);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(V) / 8); ++i) d[i] = __ldcg(s + i);
  return v;
}

// Add for the value types used in look-back.
__device__ __forceinline__ dd lb_add(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ u128 lb_add(u128 a, u128 b) { return u128_add(a, b); }
__device__ __forceinline__ xf lb_add(xf a, xf b) { return xf_add(a, b); }
template <typename V>
__device__ __forceinline__ V lb_zero();
template <>
__device__ __forceinline__ dd lb_zero<dd>() { return {0.0, 0.0}; }
template <>
__device__ __forceinline__ u128 lb_zero<u128>() { return {0ULL, 0ULL}; }
template <>
__device__ __forceinline__ xf lb_zero<xf>() { return {0ULL, 0ULL, kXfZeroE}; }

template <typename V>
__device__ __forceinline__ V shfl_v(V v, int src) {
  V r;
  const uint64_t* s = reinterpret_cast<const uint64_t*>(&v);
  uint64_t* d = reinterpret_cast<uint64_t*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(V) / 8); ++i) d[i] = __shfl_sync(0xFFFFFFFFu, s[i], src);
  return r;
}
template <typename V>
__device__ __forceinline__ V shfl_up_v(V v, int o) {
  V r;
  const uint64_t* s = reinterpret_cast<const uint64_t*>(&v);
  uint64_t* d = reinterpret_cast<uint64_t*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(V) / 8); ++i) d[i] = __shfl_up_sync(0xFFFFFFFFu, s[i], o);
  return r;
}
template <typename V>
__device__ __forceinline__ V shfl_down_v(V v, int o) {
  V r;
  const uint64_t* s = reinterpret_cast<const uint64_t*>(&v);
  uint64_t* d = reinterpret_cast<uint64_t*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(V) / 8); ++i) d[i] = __shfl_down_sync(0xFFFFFFFFu, s[i], o);
  return r;
}

// Publish the tile aggregate (tile 0 publishes it as inclusive directly).
template <typename V>
__device__ __forceinline__ void lb_publish(TileDesc<V>* desc, int64_t tile, V agg, bool inclusive) {
  TileDesc<V>* d = desc + tile;
  if (inclusive) {
    d->inc = agg;
    d->agg = agg;
  } else {
    d->agg = agg;
  }
  __threadfence();
  st_release_u32(&d->flag, inclusive ? kFlagInc : kFlagAgg);
}

// Publish the inclusive prefix of a tile that earlier published its aggregate.
template <typename V>
__device__ __forceinline__ void lb_publish_inc(TileDesc<V>* desc, int64_t tile, V inc) {
  TileDesc<V>* d = desc + tile;
  d->inc = inc;
  __threadfence();
  st_release_u32(&d->flag, kFlagInc);
}

// Called by one full warp of tile `tile` (> 0).  Returns the exclusive prefix
// of the tile.  Summation order inside a window is a fixed tree, so for exact
// value types (u128) the result does not depend on timing at all.
template <typename V>
__device__ V lb_exclusive(TileDesc<V>* desc, int64_t tile, int lane, int spin_limit, int* status) {
  V excl = lb_zero<V>();
  int64_t base = tile - 1;  // the window covers base - lane
  while (true) {
    const int64_t t = base - lane;
    uint32_t f = kFlagInc;
    V val = lb_zero<V>();
    if (t >= 0) {
      int spins = 0;
      f = ld_acquire_u32(&desc[t].flag);
      while (f == kFlagEmpty) {
        if (++spins > spin_limit) break;
        __nanosleep(64);
        f = ld_acquire_u32(&desc[t].flag);
      }
      if (f == kFlagEmpty) {
        raise_status(status, ST_ETIMEOUT);
        f = kFlagInc;  // give up on this predecessor: count it as zero
      } else {
        val = (f == kFlagInc) ? ld_cg(&desc[t].inc) : ld_cg(&desc[t].agg);
      }
    }
    const unsigned inc_mask = __ballot_sync(0xFFFFFFFFu, f == kFlagInc);
    const int stop = inc_mask ? (__ffs(inc_mask) - 1) : 31;  // nearest inclusive predecessor
    if (lane > stop) val = lb_zero<V>();
    // reduce lanes 0..stop (tree)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      V other = shfl_down_v(val, o);
      if (lane + o < 32) val = lb_add(val, other);
    }
    val = shfl_v(val, 0);
    excl = lb_add(excl, val);
    if (inc_mask) break;
    base -= 32;
  }
  return excl;
}

// Inclusive warp scan for the look-back value types.
template <typename V>
__device__ __forceinline__ V warp_incl_scan_v(V v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    V t = shfl_up_v(v, o);
    if (lane >= o) v = lb_add(t, v);
  }
  return v;
}

// Total order key of a binary64 that agrees with IEEE comparison for every
// non-NaN value (-0 and +0 map to the same key): sign-magnitude to two's
// complement.  Comparing keys as int64 costs integer instructions only.
__device__ __forceinline__ long long ord_key_bits(long long b) { return b >= 0 ? b : -(b & 0x7FFFFFFFFFFFFFFFLL); }
__device__ __forceinline__ long long ord_key(double x) { return ord_key_bits(__double_as_longlong(x)); }

}  // namespace gbr
