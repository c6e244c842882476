// Weights from log-weights, the step before resampling (Sec. I: the filter
// carries log-likelihoods): w_j = exp(l_j - m), m = max_k l_k.
//
// GB300 form: two passes, no binary64 arithmetic per element.
//   max   grid-stride maximum over an order-preserving 64-bit encoding of the
//         binary64 log-weights (one atomicMax per CTA); NaN and +inf latch
//         RS_ENONFINITE.
//   exp   exp(l_j - m) in 64-bit integer arithmetic (no binary64 operation):
//         the difference in fixed point (units 2^-51), Tang's table-driven
//         reduction x = n ln2/256 + r with a 256-entry table of 2^(j/256),
//         e^r - 1 = r + r^2/2 (integer products) + a binary32 tail, and the
//         result rounded into binary64 bits.  Relative error below 2^-49.5
//         (2^-52 when |l|, |m| >= 1); subnormal results within 2 units of
//         2^-1074.
// -inf gives a zero weight; all -inf latches RS_EZEROSUM (zero weights out);
// NaN, +inf and |l| >= 2^126 latch RS_ENONFINITE (and give zero weights).
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

// 2^(j/256) in units 2^-62, rounded to nearest: the integer nearest to
// 2^((62 * 256 + j) / 256), j = 0..255.
__device__ const unsigned long long kExp2Tab[256] = {
    0x4000000000000000ULL, 0x402c6be96af2fb58ULL, 0x4058f6a7ecccd5b6ULL, 0x4085a050ec0a036aULL,
    0x40b268f9de0183baULL, 0x40df50b846ef302bULL, 0x410c57a1b9fe12f6ULL, 0x41397dcbd952c4a6ULL,
    0x4166c34c5615d0ecULL, 0x41942838f07e22a3ULL, 0x41c1aca777db771bULL, 0x41ef50adcaa0d899ULL,
    0x421d1461d66f2023ULL, 0x424af7d9981f7e98ULL, 0x4278fb2b1bce0d15ULL, 0x42a71e6c7ce464afULL,
    0x42d561b3e6243d8aULL, 0x4303c51791b21550ULL, 0x433248adc91fdd02ULL, 0x4360ec8ce577ae44ULL,
    0x438fb0cb4f468808ULL, 0x43be957f7ea712b6ULL, 0x43ed9abffb4c6bc9ULL, 0x441cc0a35c8cf8eaULL,
    0x444c0740496d4294ULL, 0x447b6ead78aad636ULL, 0x44aaf701b0c72feeULL, 0x44daa053c812abd2ULL,
    0x450a6abaa4b77ecdULL, 0x453a564d3cc4b723ULL, 0x456a632296394492ULL, 0x459a9151c70f0819ULL,
    0x45cae0f1f545eb73ULL, 0x45fb521a56ef0042ULL, 0x462be4e23237a6efULL, 0x465c9960dd74bd4bULL,
    0x468d6fadbf2dd4f3ULL, 0x46be67e04e28717cULL, 0x46ef821011734e6bULL, 0x4720be54a071ad01ULL,
    0x47521cc5a2e6a9e0ULL, 0x47839d7ad1009a90ULL, 0x47b5408bf36472e2ULL, 0x47e70610e3393241ULL,
    0x4818ee218a3358eeULL, 0x484af8d5e2a06536ULL, 0x487d2645f7725895ULL, 0x48af7689e44b44eaULL,
    0x48e1e9b9d588e19bULL, 0x49147fee085028d6ULL, 0x4947393eca98fcd6ULL, 0x497a15c47b39d53eULL,
    0x49ad159789f37496ULL, 0x49e038d0777ca5e0ULL, 0x4a137f87d58e025bULL, 0x4a46e9d646edbf6aULL,
    0x4a7a77d47f7b84b1ULL, 0x4aae299b443c4a6bULL, 0x4ae1ff436b663ff7ULL, 0x4b15f8e5dc6cbab0ULL,
    0x4b4a169b900c2d00ULL, 0x4b7e587d905625d1ULL, 0x4bb2bea4f8bd5847ULL, 0x4be7492af621abd6ULL,
    0x4c1bf828c6dc54b8ULL, 0x4c50cbb7bacbf4cbULL, 0x4c85c3f13360c4d5ULL, 0x4cbae0eea3a8c63cULL,
    0x4cf022c9905bfd32ULL, 0x4d25899b8fe8b365ULL, 0x4d5b157e4a7fc325ULL, 0x4d90c68b7a20eb1eULL,
    0x4dc69cdceaa72a9cULL, 0x4dfc988c79d52661ULL, 0x4e32b9b417619617ULL, 0x4e69006dc503ba65ULL,
    0x4e9f6cd3967fdba8ULL, 0x4ed5feffb1b3d155ULL, 0x4f0cb70c4ea39210ULL, 0x4f439513b785cc80ULL,
    0x4f7a993048d088d7ULL, 0x4fb1c37c7145d328ULL, 0x4fe91412b2006e83ULL, 0x50208b0d9e8090dfULL,
    0x50582887dcb8a7e1ULL, 0x508fec9c251a267cULL, 0x50c7d76542a25b72ULL, 0x50ffe8fe12e750c4ULL,
    0x513821818624b40cULL, 0x5170810a9f48c7cfULL, 0x51a907b474015dc9ULL, 0x51e1b59a2cc8da3eULL,
    0x521a8ad704f3404fULL, 0x525387864abb4762ULL, 0x528cabc35f4f799dULL, 0x52c5f7a9b6df5b77ULL,
    0x52ff6b54d8a89c75ULL, 0x533906e05f045106ULL, 0x5372ca67f774358fULL, 0x53acb60762affaaeULL,
    0x53e6c9da74b29ab5ULL, 0x542105fd14c7b869ULL, 0x545b6a8b3d990704ULL, 0x5495f7a0fd3bbb8eULL,
    0x54d0ad5a753e077cULL, 0x550b8bd3dab49cbdULL, 0x5546932976483b15ULL, 0x5581c377a44346f0ULL,
    0x55bd1cdad49f699cULL, 0x55f89f6f8b133af4ULL, 0x56344b525f1ff495ULL, 0x5670209ffc1f2e82ULL,
    0x56ac1f752150a563ULL, 0x56e847eea1e80a49ULL, 0x57249a29651adc07ULL, 0x57611642662e4a33ULL,
    0x579dbc56b48521baULL, 0x57da8c8373adc331ULL, 0x581786e5db7022c2ULL, 0x5854ab9b37dbd1e5ULL,
    0x5891fac0e95612c8ULL, 0x58cf747464a7f584ULL, 0x590d18d3330c7f1eULL, 0x594ae7faf23eda52ULL,
    0x5988e20954889245ULL, 0x59c7071c20cfd70cULL, 0x5a05575132a5cc20ULL, 0x5a43d2c67a54e0c0ULL,
    0x5a827999fcef3242ULL, 0x5ac14be9d45cf869ULL, 0x5b0049d42f6afbb6ULL, 0x5b3f737751d915c8ULL,
    0x5b7ec8f19468bbc9ULL, 0x5bbe4a6164eb92f4ULL, 0x5bfdf7e546520f3eULL, 0x5c3dd19bd0ba1c1aULL,
    0x5c7dd7a3b17dcf75ULL, 0x5cbe0a1bab4226dfULL, 0x5cfe69229605cef5ULL, 0x5d3ef4d75f2ff504ULL,
    0x5d7fad59099f22feULL, 0x5dc092c6adb825b8ULL, 0x5e01a53f7974fd86ULL, 0x5e42e4e2b073d935ULL,
    0x5e8451cfac061b5fULL, 0x5ec5ec25db3f6a41ULL, 0x5f07b404c304c9f1ULL, 0x5f49a98bfe1bc11cULL,
    0x5f8bccdb3d398841ULL, 0x5fce1e124712437cULL, 0x60109d50f86846d8ULL, 0x60534ab7441b6546ULL,
    0x6096266533384a2bULL, 0x60d9307ae507dd9aULL, 0x611c69188f1eb339ULL, 0x615fd05e7d6c83e4ULL,
    0x61a3666d124bb204ULL, 0x61e72b64c690d8afULL, 0x622b1f66299a6599ULL, 0x626f4291e1603dd5ULL,
    0x62b39508aa836d6fULL, 0x62f816eb585de1edULL, 0x633cc85ad5122fbdULL, 0x6381a978219b628fULL,
    0x63c6ba6455dcd8aeULL, 0x640bfb40a0b22959ULL, 0x64516c2e47ff1623ULL, 0x64970d4ea8bf8766ULL,
    0x64dcdec3371793d1ULL, 0x6522e0ad7e639312ULL, 0x6569132f21483ba7ULL, 0x65af7669d9c2cbe4ULL,
    0x65f60a7f79393e2eULL, 0x663ccf91e88a8873ULL, 0x6683c5c3281ee6e9ULL, 0x66caed354ff83222ULL,
    0x6712460a8fc24072ULL, 0x6759d0652ee352afULL, 0x67a18c678c8c8c61ULL, 0x67e97a341fca775bULL,
    0x683199ed779592caULL, 0x6879ebb63ae2edc6ULL, 0x68c26fb128b4cd63ULL, 0x690b2601182b5e56ULL,
    0x69540ec8f895722dULL, 0x699d2a2bd181482aULL, 0x69e6784cc2cd61bdULL, 0x6a2ff94f04b962b0ULL,
    0x6a79ad55e7f6fd10ULL, 0x6ac39484d5bae8c5ULL, 0x6b0daeff4fcde703ULL, 0x6b57fce8f09dd17fULL,
    0x6ba27e656b4eb57aULL, 0x6bed33988bcbfab5ULL, 0x6c381ca636d99642ULL, 0x6c8339b26a25494eULL,
    0x6cce8ae13c57ebdbULL, 0x6d1a1056dd26c382ULL, 0x6d65ca379564e639ULL, 0x6db1b8a7c714a92bULL,
    0x6dfddbcbed791babULL, 0x6e4a33c89d278e49ULL, 0x6e96c0c284192610ULL, 0x6ee382de69bc7bf8ULL,
    0x6f307a412f074892ULL, 0x6f7da70fce881bf9ULL, 0x6fcb096f5c782210ULL, 0x7018a18506ccf314ULL,
    0x70666f76154a7089ULL, 0x70b47367e994ae92ULL, 0x7102ad7fff41e9b4ULL, 0x71511de3ebec8913ULL,
    0x719fc4b95f452d29ULL, 0x71eea2262324cb0cULL, 0x723db6501b9ed447ULL, 0x728d015d47136b40ULL,
    0x72dc8373be41a454ULL, 0x732c3cb9b459d38bULL, 0x737c2d55770fe711ULL, 0x73cc556d6eadce5fULL,
    0x741cb5281e25ee34ULL, 0x746d4cac2325a155ULL, 0x74be1c203627c62bULL, 0x750f23ab2a87593eULL,
    0x75606373ee921c97ULL, 0x75b1dba18b9b4c20ULL, 0x76038c5b260e5eeeULL, 0x765575c7fd81d5a0ULL,
    0x76a7980f6cca15c2ULL, 0x76f9f358ea0c5249ULL, 0x774c87cc06d1812eULL, 0x779f559070195e36ULL,
    0x77f25ccdee6d7ae6ULL, 0x78459dac65f45bb5ULL, 0x78991853d684a285ULL, 0x78ecccec5bb84661ULL,
    0x7940bb9e2cffd89dULL, 0x7994e4919db5d74eULL, 0x79e947ef1d320d2dULL, 0x7a3de5df36dcfeefULL,
    0x7a92be8a92436616ULL, 0x7ae7d219f329b948ULL, 0x7b3d20b6399fc237ULL, 0x7b92aa886214411cULL,
    0x7be86fb985689ddcULL, 0x7c3e7072d904a6ceULL, 0x7c94acddaeea5d3aULL, 0x7ceb252375c9cf9bULL,
    0x7d41d96db915019dULL, 0x7d98c9e62113e1faULL, 0x7deff6b672f84e24ULL, 0x7e47600890f223deULL,
    0x7e9f06067a4360baULL, 0x7ef6e8da4b544f9aULL, 0x7f4f08ae3dc7c426ULL, 0x7fa765aca88f6453ULL
};

// x = l - m in fixed point, units 2^-51, truncated toward zero per operand.
constexpr long long kUnderflowX = 1677906113169425695LL;  // 2^51 745.14 rounded up: below -745.14, exp is 0

// |v| < 2^11 (biased exponent <= 1033): v 2^51 = mant 2^(e - 1024); zero
// and subnormals give 0
__device__ __forceinline__ long long fixed51_small(unsigned long long b) {
  const int e = (int)((b >> 52) & 0x7FF);
  const long long v = (long long)((((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52)) << 9) >> min(1033 - e, 63));
  return (b >> 63) ? -v : v;
}
// any |l|, |m| < 2^126: both at units 2^(Ebig - 61), Ebig the larger
// exponent (at least 10), then the difference at units 2^-51 unless it is
// below -745.14 (false)
__device__ __noinline__ bool fixed51_general(unsigned long long lb, unsigned long long mb, long long& X) {
  const int El = (int)((lb >> 52) & 0x7FF) - 1023, Em = (int)((mb >> 52) & 0x7FF) - 1023;
  const int Ebig = max(max(El, Em), 10);
  auto at = [Ebig](unsigned long long b, int E) {
    const unsigned long long mant = ((b >> 52) & 0x7FF) ? ((b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52)) : 0ULL;
    const int sh = E - Ebig + 9;  // <= 9: below 2^62
    const unsigned long long v = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ULL);
    return (b >> 63) ? -(long long)v : (long long)v;
  };
  const long long D = at(lb, El) - at(mb, Em);  // <= 0 (truncation toward zero is monotone)
  const int s = min(Ebig - 10, 62);
  if (-D > (kUnderflowX >> s)) return false;
  X = (long long)((unsigned long long)D << s);
  return true;
}

// V2 2^(be - 1023 - 62), V2 in [2^62, 2^63), be <= 0: a subnormal (or 0),
// rounded to nearest
__device__ __noinline__ unsigned long long subnormal_bits(unsigned long long V2, int be) {
  const int sh = 11 - be;
  return sh > 63 ? 0ULL : ((V2 + (1ULL << (sh - 1))) >> sh);
}

// exp(x) for x = X 2^-51 in [-745.14, 0] as binary64 bits, in integer
// arithmetic plus a few binary32 operations (Tang's table-driven method):
//   x = n ln2/256 + r: n = round(x 256/ln2) from the high word of X (within
//       1e-3), r in units 2^-59 with ln2/256 = (K1 + K2 2^-32) 2^-51 (K1, K2
//       the rounded integers; the products wrap modulo 2^64 exactly)
//   e^r - 1 = r + r^2/2 + q: r^2/2 from two 32 x 32-bit products, q = r^3/6
//       + r^4/24 + r^5/120 in binary32 (|q| < 2^-31), in units 2^-62
//   2^((n mod 256)/256) e^r = t + t (e^r - 1): one signed 64 x 64-bit high
//       product with the table entry t
//   rounded to nearest into binary64 bits, subnormals included.
// Relative error below 2^-49.5 (about 2^-52 when |l|, |m| >= 1); subnormal
// results within 2 units of 2^-1074.
__device__ __forceinline__ unsigned long long exp_fixed51(long long X, const unsigned long long* __restrict__ T) {
  const int n = (int)(((long long)(int)(X >> 32) * 1549082005LL + (1LL << 40)) >> 41);
  const long long R = (long long)((unsigned long long)X << 8) - (long long)n * (6096987078286LL << 8) -
                      (((long long)n * 2077056591LL + (1LL << 23)) >> 24);
  const int Rh = (int)(R >> 19);  // |R| < 2^49.5
  const long long Rl = R & 0x7FFFF;
  const long long sq2 = (long long)((unsigned long long)((long long)Rh * Rh) >> 19) + (((long long)Rh * Rl) >> 37);
  const float rf = __int2float_rn(Rh) * 9.094947017729282e-13f;  // r (2^-40 units)
  const float q = rf * rf * rf * (0.16666667f + rf * (0.041666668f + rf * 0.008333334f));
  const long long E1 = R * 8 + sq2 + __float2int_rn(q * 4.611686018427388e18f);  // e^r - 1, units 2^-62
  const long long t = (long long)T[n & 255];
  const unsigned long long V = (unsigned long long)(t + __mul64hi(t, E1 * 4));  // in (2^61, 2^63)
  const int lz = (int)(1 - (V >> 62));
  const unsigned long long V2 = V << lz;
  const int be = (n >> 8) - lz + 1023;  // the result's biased exponent
  if (be > 0) return ((unsigned long long)(be - 1) << 52) + ((V2 + (1ULL << 9)) >> 10);
  return subnormal_bits(V2, be);
}

__global__ void __launch_bounds__(kLThreads) k_logw_exp(const unsigned long long* __restrict__ l, long long M,
                                                        const unsigned long long* __restrict__ mkey,
                                                        unsigned long long* __restrict__ w, int* status) {
  __shared__ unsigned long long T[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) T[i] = kExp2Tab[i];
  __syncthreads();
  const unsigned long long mk = __ldcg(mkey);
  const unsigned long long mb = order_bits(mk);
  const bool none = mk <= order_key(0xFFF0000000000000ULL);  // every l is -inf (or no valid one)
  if (none && blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, ST_EZEROSUM);
  const int em = (int)((mb >> 52) & 0x7FF);
  const long long Mx = fixed51_small(mb);  // used when |m| < 2^11
  auto weight = [&](unsigned long long b) {
    // NaN, +-inf and |l| >= 2^126 give 0 (the maximum pass latched the
    // invalid ones)
    const int el = (int)((b >> 52) & 0x7FF);
    unsigned long long out = 0ULL;
    if (!none && el < 1023 + 126) {
      long long X;
      bool in = true;
      if (el <= 1033 && em <= 1033) X = fixed51_small(b) - Mx;
      else in = fixed51_general(b, mb, X);
      if (in && X >= -kUnderflowX) out = exp_fixed51(X, T);
    }
    return out;
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  // four independent coalesced elements per thread, loads in flight together;
  // the last partial round checks each index
  long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
  for (; j0 + 3 * stride < M; j0 += 4 * stride) {
    unsigned long long b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) b[q] = __ldg(l + j0 + q * stride);
#pragma unroll
    for (int q = 0; q < 4; ++q) w[j0 + q * stride] = weight(b[q]);
  }
#pragma unroll 1
  for (; j0 < M; j0 += stride) w[j0] = weight(__ldg(l + j0));
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
