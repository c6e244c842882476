// Sorted uniforms by exponential spacings (Algorithm 1 of arXiv 2604.01356):
//   z_k = -log(v_k), k = 1..N+1;  Z_i = sum_{k<=i} z_k;  U_i = Z_i / Z_{N+1}.
// (The printed normaliser Z_{i+1} is read as Z_{N+1}.)
//
// GB300 form.  One pass over the N+1 draws: each thread takes four
// consecutive draws (the four words of one Philox block), evaluates the
// spacings (binary32-pair table logarithm for both draw formats), converts them EXACTLY to integers on a 2^-88 grid and the block
// scans them as unsigned 128-bit integers; tiles of 1024 draws chain their
// sums by decoupled look-back.  Integer sums make Z
// exact, monotone and independent of scheduling.  The resampling map consumes
// Z directly; when U itself is wanted a second kernel rounds Z_i / Z_{N+1}
// to binary64 (monotone in Z_i by construction).
#include <cmath>

#include "seg_common.cuh"

namespace gbr {

__device__ LogTab g_logtab;

template <bool F32>
__global__ void __launch_bounds__(kUThreads) k_uniform_scan(long long ndraw, unsigned long long seed,
                                                           unsigned long long inst, u128* __restrict__ Z,
                                                           u128* __restrict__ Ztot, PathConsts* consts,
                                                           TileDesc<u128>* desc, unsigned* ctr, int* status,
                                                           int spin_limit, bool withhold_first, int scheme) {
  __shared__ LogTab tab;
  __shared__ UniformTileSmem us;
  __shared__ unsigned s_tile;
  for (int i = threadIdx.x; i < 129; i += kUThreads) {
    tab.nlogc[i] = g_logtab.nlogc[i];
    tab.invc[i] = g_logtab.invc[i];
  }
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
  __syncthreads();
  uniform_tile<F32>(s_tile, ndraw, seed, inst, Z, Ztot, consts, desc, status, spin_limit, withhold_first, &tab, us,
                    scheme);
}

// U_i = Z_i / Z_{N+1} rounded to binary64: integer multiply by the reciprocal
// the scan stored, then integer rounding per element, which keeps U monotone
// in Z.  U <= 1 is enforced (rounding of the reciprocal).
__global__ void __launch_bounds__(256) k_uniform_norm(long long N, const u128* __restrict__ Z,
                                                      const PathConsts* __restrict__ consts, double* __restrict__ U) {
  const xf r = {__ldcg(consts->invZ), __ldcg(consts->invZ + 1), (long long)__ldcg(consts->invZ + 2)};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    long long ub = (long long)xf_to_f64_bits(xf_mul_u128(r, Z[i]));
    if (ub > 0x3FF0000000000000LL) ub = 0x3FF0000000000000LL;
    U[i] = __longlong_as_double(ub);
  }
}

// Small N: the whole of Algorithm 1 by one CTA, one launch and no cleared
// workspace: 512 threads x 4 draws per step (one Philox block per thread),
// spacings on the 2^-88 grid, an exact 128-bit block scan carried across
// steps, then 1/Z_{N+1} (recip_total, as the multi-tile scan stores it) and
// U_i = Z_i / Z_{N+1} rounded as k_uniform_norm does.  The integers are those
// of the multi-tile scan, so Z and U are identical to it.
constexpr int kUSmallThreads = 512;
template <bool F32>
__global__ void __launch_bounds__(kUSmallThreads) k_uniform_small(long long ndraw, unsigned long long seed,
                                                                  unsigned long long inst, u128* __restrict__ Z,
                                                                  double* __restrict__ U, int scheme) {
  constexpr int kW = kUSmallThreads / kWarp;
  __shared__ LogTab tab;
  __shared__ u128 wsum[kW];
  __shared__ xf s_r;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 129; i += kUSmallThreads) {
    tab.nlogc[i] = g_logtab.nlogc[i];
    tab.invc[i] = g_logtab.invc[i];
  }
  __syncthreads();
  const long long N = ndraw - 1;
  u128 carry = {0ULL, 0ULL};
#pragma unroll 1
  for (long long d0 = 0; d0 < ndraw; d0 += 4LL * kUSmallThreads) {
    const long long k0 = d0 + 4LL * tid;
    uint64_t words[4];
    philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, seed, inst, words);
    u128 f[4], inc[4];
    block_spacings<F32>(scheme, k0, ndraw, seed, inst, words, &tab, f);
    u128 run = {0ULL, 0ULL};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      run = u128_add(run, f[q]);
      inc[q] = run;
    }
    const u128 incl = warp_incl_scan_v(run, lane);
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    u128 off = {0ULL, 0ULL}, tot = {0ULL, 0ULL};
#pragma unroll
    for (int i = 0; i < kW; ++i) {
      const u128 x = wsum[i];
      if (i < warp) off = u128_add(off, x);
      tot = u128_add(tot, x);
    }
    __syncthreads();  // wsum is reused by the next step
    off = u128_add(carry, u128_add(off, u128_sub(incl, run)));
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (k0 + q < N) Z[k0 + q] = u128_add(off, inc[q]);
    carry = u128_add(carry, tot);
  }
  if (tid == 0) s_r = u128_is_zero(carry) ? lb_zero<xf>() : recip_total(carry);
  __syncthreads();
  const xf r = s_r;
#pragma unroll 1
  for (long long i = tid; i < N; i += kUSmallThreads) {
    long long ub = (long long)xf_to_f64_bits(xf_mul_u128(r, Z[i]));
    if (ub > 0x3FF0000000000000LL) ub = 0x3FF0000000000000LL;
    U[i] = __longlong_as_double(ub);
  }
}

cudaError_t launch_uniform_small(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst, void* Z,
                                 double* U, cudaStream_t st, int scheme) {
  if (ndraw <= 1) return cudaSuccess;
  if (f32)
    k_uniform_small<true><<<1, kUSmallThreads, 0, st>>>(ndraw, seed, inst, (u128*)Z, U, scheme);
  else
    k_uniform_small<false><<<1, kUSmallThreads, 0, st>>>(ndraw, seed, inst, (u128*)Z, U, scheme);
  return cudaGetLastError();
}

__global__ void k_philox_words(unsigned long long seed, unsigned long long inst, unsigned long long first, long long n,
                               unsigned long long* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long k = first + (unsigned long long)i;
    uint64_t w[4];
    philox4x64_10(k / 4, 0ULL, 0ULL, 0ULL, seed, inst, w);
    const unsigned q = (unsigned)(k & 3);
    out[i] = q == 0 ? w[0] : q == 1 ? w[1] : q == 2 ? w[2] : w[3];
  }
}

void fill_log_table(LogTab& h) {
  for (int k = 0; k <= 128; ++k) {
    const double c = 1.0 - k / 256.0;
    const double nl = -std::log(c);
    const double ic = 1.0 / c;
    const float nh = (float)nl, ih = (float)ic;
    h.nlogc[k] = make_float2(nh, (float)(nl - (double)nh));
    h.invc[k] = make_float2(ih, (float)(ic - (double)ih));
  }
}

cudaError_t init_log_table() {
  LogTab h;
  fill_log_table(h);
  return cudaMemcpyToSymbol(g_logtab, &h, sizeof(h));
}

size_t log_table_bytes() { return sizeof(LogTab); }

cudaError_t upload_log_table(void* dst) {
  LogTab h;
  fill_log_table(h);
  return cudaMemcpy(dst, &h, sizeof(h), cudaMemcpyHostToDevice);
}

cudaError_t launch_uniform_scan(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst, void* Z,
                                void* Ztot, PathConsts* consts, void* desc, unsigned* ctr, int* status,
                                int spin_limit, bool withhold_first, cudaStream_t st, int scheme) {
  const long long tiles = (ndraw + kUTile - 1) / kUTile;
  if (tiles <= 0) return cudaSuccess;
  if (f32)
    k_uniform_scan<true><<<(unsigned)tiles, kUThreads, 0, st>>>(ndraw, seed, inst, (u128*)Z, (u128*)Ztot, consts,
                                                                (TileDesc<u128>*)desc, ctr, status, spin_limit, withhold_first, scheme);
  else
    k_uniform_scan<false><<<(unsigned)tiles, kUThreads, 0, st>>>(ndraw, seed, inst, (u128*)Z, (u128*)Ztot, consts,
                                                                 (TileDesc<u128>*)desc, ctr, status, spin_limit, withhold_first, scheme);
  return cudaGetLastError();
}

cudaError_t launch_uniform_norm(long long N, const void* Z, const PathConsts* consts, double* U, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  long long blocks = (N + 255) / 256;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_uniform_norm<<<(unsigned)blocks, 256, 0, st>>>(N, (const u128*)Z, consts, U);
  return cudaGetLastError();
}

cudaError_t launch_philox(unsigned long long seed, unsigned long long inst, unsigned long long first, long long n,
                          unsigned long long* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_philox_words<<<(unsigned)blocks, 256, 0, st>>>(seed, inst, first, n, out);
  return cudaGetLastError();
}

}  // namespace gbr
