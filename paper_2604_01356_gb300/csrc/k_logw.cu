// Weights from log-weights, the step before resampling (Sec. I: the filter
// carries log-likelihoods): w_j = exp(l_j - m), m = max_k l_k.
//
// GB300 form: two HBM-bound passes, no binary64 arithmetic per element.
//   max   grid-stride maximum over an order-preserving 64-bit encoding of the
//         binary64 log-weights (one atomicMax per CTA); NaN and +inf latch
//         RS_ENONFINITE.
//   exp   every l_j - m as an exact sum of six binary32 terms (three-way
//         split of each binary64 operand, two-sum), then exp by Cody-Waite
//         reduction
//         x = n ln2/64 + r (ln2/64 in three binary32 parts, n ln2_1 exact),
//         2^(j/64) from a binary32-pair table and a degree-6 series for e^r
//         (|r| <= ln2/128) in binary32-pair arithmetic; the result is packed
//         into binary64 bits by integer operations.  Relative error about
//         2^-44 of the binary64 value (absolute below 2^-1060 for subnormal
//         results).
// -inf gives a zero weight; all -inf latches RS_EZEROSUM (zero weights out);
// NaN, +inf and |l| >= 2^126 latch RS_ENONFINITE (and give zero weights).
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace gbr {

namespace {

constexpr int kLThreads = 256;

__device__ __forceinline__ unsigned long long order_key(unsigned long long b) {
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ unsigned long long order_bits(unsigned long long k) {
  return (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
}
__device__ __forceinline__ bool bad_logw(unsigned long long b) {
  // NaN, +inf, or |l| >= 2^126 (no meaning as a log-weight); -inf is valid
  return ((b >> 52) & 0x7FF) >= 1023 + 126 && b != 0xFFF0000000000000ULL;
}

__global__ void __launch_bounds__(kLThreads) k_logw_max(const unsigned long long* __restrict__ l, long long M,
                                                        unsigned long long* __restrict__ mkey, int* status) {
  unsigned long long best = 0;
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // four independent coalesced loads in flight per thread
#pragma unroll 1
  for (long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; j0 < M; j0 += 4 * stride) {
    unsigned long long b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = j0 + q * stride < M ? __ldg(l + j0 + q * stride) : 0xFFF0000000000000ULL;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      bad |= bad_logw(b[q]);
      best = max(best, bad_logw(b[q]) ? 0ULL : order_key(b[q]));
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) raise_status(status, ST_ENONFINITE);
  __shared__ unsigned long long s_b[kLThreads / 32];
  if ((threadIdx.x & 31) == 0) s_b[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int i = 0; i < kLThreads / 32; ++i) m = max(m, s_b[i]);
    atomicMax(mkey, m);
  }
}

// binary64 bits -> three binary32 whose sum is x exactly (53 = 24 + 24 + 5
// significant bits); |x| < 2^126.  |x| < 2^-126 is taken as 0 (it moves exp
// by less than 2^-126).
struct f3 {
  float h, m, t;
};
__device__ __forceinline__ float pow2f(int e) {  // 2^e for -126 <= e <= 127, else 0 below
  return e >= -126 ? __int_as_float((e + 127) << 23) : 0.0f;
}
__device__ __forceinline__ f3 f64_split(unsigned long long b) {
  const unsigned sign = (unsigned)(b >> 63);
  const int e = (int)((b >> 52) & 0x7FF);
  const int E = e - 1023;
  if (E < -126) return {0.0f, 0.0f, 0.0f};
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const float h = __int_as_float((int)((sign << 31) | ((unsigned)(E + 127) << 23) | ((unsigned)(mant >> 29) & 0x7FFFFFu)));
  float m = __uint2float_rn((unsigned)((mant >> 5) & 0xFFFFFFu)) * pow2f(E - 47);  // 24 bits, exact
  float t = __uint2float_rn((unsigned)(mant & 0x1Fu)) * pow2f(E - 52);           // 5 bits, exact
  if (sign) {
    m = -m;
    t = -t;
  }
  return {h, m, t};
}

// binary32 pair plus one binary32: two-sum of the high parts, the low part
// folded in, renormalised.  The only rounding is that of the two low parts'
// sum (below 2^-24 of it); half the operations of a pair-plus-pair addition.
__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = df_two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return df_fast_two_sum(s.hi, s.lo);
}

// exp(x) for x = s + e + a + b + c + d <= 0 (s, e an exact two-sum, the
// others small binary32 terms), as binary64 bits.  The reduction consumes
// the terms one by one, so only the small remainder r is ever rounded
// (absolute error about 2^-48 |r|, whatever |x|).
__device__ __forceinline__ unsigned long long exp_neg_bits(float s, float e, float a, float b, float c, float d,
                                                           const float2* __restrict__ T) {
  if (s < -745.5f) return 0ULL;
  const float kInvL = 92.33248261689366f;  // 64 / ln2
  const float L1 = 0.0107421875f;          // ln2/64 = L1 + L2 + L3, L1 with 4 significant bits
  const float L2 = 8.823719690553844e-05f;
  const float L3 = -6.5639296298672378e-13f;
  const int n = __float2int_rn(s * kInvL);  // |n| < 2^17: n L1 exact
  const float fn = (float)n;
  df r = df_two_sum(s - fn * L1, e);  // the first difference is exact (Sterbenz)
  r = df_add_f(r, a);
  r = df_add_f(r, b);
  r = df_add_f(r, c);
  r = df_add_f(r, d);
  const float p = fn * L2;
  const float pe = fmaf(fn, L2, -p);
  r = df_add(r, df{-p, -pe});
  r = df_add_f(r, -fn * L3);
  // e^r = 1 + r + r^2 (1/2 + q), q = r/6 + r^2/24 + r^3/120 + r^4/720 (binary32 suffices)
  const float rh = r.hi;
  const float q = rh * (1.0f / 6.0f + rh * (1.0f / 24.0f + rh * (1.0f / 120.0f + rh * (1.0f / 720.0f))));
  const df r2 = df_mul(r, r);
  df ex = df_add(df_mul_f(r2, q), df{r2.hi * 0.5f, r2.lo * 0.5f});
  ex = df_add(ex, r);
  ex = df_add_f(ex, 1.0f);
  const int k = n >> 6, j = n & 63;
  const df t = {T[j].x, T[j].y};
  const df v = df_mul(t, ex);  // in [0.99, 2.01]
  // (v.hi + v.lo) 2^k as binary64 bits: integer mantissa at v.hi's scale
  const unsigned hb = (unsigned)__float_as_int(v.hi);
  const int eh = (int)((hb >> 23) & 0xFF) - 127;
  long long Mm = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // units 2^(eh - 52)
  if (v.lo != 0.0f) {
    const unsigned lb = (unsigned)__float_as_int(v.lo);
    const int el = (int)((lb >> 23) & 0xFF) - 127;
    const long long ml = (long long)((lb & 0x7FFFFFu) | 0x800000u);
    const int sh = el - 23 - (eh - 52);
    long long add = 0;
    if (sh >= 0) add = ml << sh;
    else if (sh > -63) add = ml >> (-sh);
    Mm += (lb >> 31) ? -add : add;
  }
  int E = eh + k;
  unsigned long long Mu = (unsigned long long)Mm;
  if (Mu >> 53) {
    Mu >>= 1;
    ++E;
  } else if (!(Mu >> 52)) {
    Mu <<= 1;
    --E;
  }
  if (E + 1023 <= 0) {  // below the normal range: a subnormal (truncated)
    const int sh = 1 - (E + 1023);
    return sh > 53 ? 0ULL : (Mu >> sh);
  }
  return ((unsigned long long)(E + 1023) << 52) | (Mu & 0xFFFFFFFFFFFFFULL);
}

__global__ void __launch_bounds__(kLThreads) k_logw_exp(const unsigned long long* __restrict__ l, long long M,
                                                        const unsigned long long* __restrict__ mkey,
                                                        unsigned long long* __restrict__ w, int* status) {
  __shared__ float2 T[64];
  if (threadIdx.x < 64) {
    const double v = exp2((double)threadIdx.x / 64.0);
    const float hi = (float)v;
    T[threadIdx.x] = make_float2(hi, (float)(v - (double)hi));
  }
  __syncthreads();
  const unsigned long long mk = __ldcg(mkey);
  const unsigned long long mb = order_bits(mk);
  const bool none = mk <= order_key(0xFFF0000000000000ULL);  // every l is -inf (or no valid one)
  if (none && blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, ST_EZEROSUM);
  const f3 m = f64_split(mb);
  const long long stride = (long long)gridDim.x * blockDim.x;
  // four independent coalesced elements per thread: loads in flight together,
  // the four exponentials interleaved
#pragma unroll 1
  for (long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; j0 < M; j0 += 4 * stride) {
    unsigned long long b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = j0 + q * stride < M ? __ldg(l + j0 + q * stride) : 0xFFF0000000000000ULL;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      unsigned long long out = 0ULL;
      if (!none && !bad_logw(b[q]) && b[q] != 0xFFF0000000000000ULL) {
        const f3 lx = f64_split(b[q]);
        const df x = df_two_sum(lx.h, -m.h);  // l - m = x.hi + x.lo + (lx.m - m.m) + (lx.t - m.t), exactly
        if (x.hi == 0.0f && lx.m == m.m && lx.t == m.t) out = 0x3FF0000000000000ULL;  // l_j = m: weight 1
        else out = exp_neg_bits(x.hi, x.lo, lx.m, -m.m, lx.t, -m.t, T);
      }
      if (j0 + q * stride < M) w[j0 + q * stride] = out;
    }
  }
}

}  // namespace

cudaError_t launch_softmax_weights(const double* l, long long M, double* w, unsigned long long* mkey, int* status,
                                   cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(mkey, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  long long blocks = (M + 4LL * kLThreads - 1) / (4LL * kLThreads);
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_logw_max<<<(unsigned)blocks, kLThreads, 0, st>>>(reinterpret_cast<const unsigned long long*>(l), M, mkey, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_logw_exp<<<(unsigned)blocks, kLThreads, 0, st>>>(reinterpret_cast<const unsigned long long*>(l), M, mkey,
                                                     reinterpret_cast<unsigned long long*>(w), status);
  return cudaGetLastError();
}

}  // namespace gbr
