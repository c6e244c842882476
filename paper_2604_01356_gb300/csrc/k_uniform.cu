// Sorted uniforms by exponential spacings (Algorithm 1 of arXiv 2604.01356):
//   z_k = -log(v_k), k = 1..N+1;  Z_i = sum_{k<=i} z_k;  U_i = Z_i / Z_{N+1}.
// (The printed normaliser Z_{i+1} is read as Z_{N+1}.)
//
// GB300 form.  One pass over the N+1 draws: each lane draws 16 consecutive
// Philox words, evaluates the spacings (binary32-pair log for binary64 draws,
// binary32 logf for binary32 draws), converts them EXACTLY to integers on a
// 2^-88 grid and scans them as unsigned 128-bit integers; tiles of 4096 draws
// chain their sums by decoupled look-back.  Integer sums make Z exact,
// monotone and independent of scheduling.  A second small kernel forms
// U_i = fl(Z_i) * fl(1/Z_{N+1}) (monotone in Z_i by construction).
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace gbr {

__device__ LogTab g_logtab;

constexpr int kUThreads = 256;
constexpr int kUWarps = kUThreads / kWarp;
static_assert(kUWarps * kSeg == kUTile, "uniform tile");
constexpr int kZFrac = 88;  // spacing grid 2^-88

template <bool F32>
__global__ void __launch_bounds__(kUThreads) k_uniform_scan(long long ndraw, unsigned long long seed,
                                                           unsigned long long inst, u128* __restrict__ Z,
                                                           u128* __restrict__ Ztot, TileDesc<u128>* desc,
                                                           unsigned* ctr, int* status, int spin_limit) {
  __shared__ LogTab tab;
  __shared__ u128 s_wsum[kUWarps];
  __shared__ u128 s_woff[kUWarps];
  __shared__ unsigned s_tile;
  if (!F32) {
    for (int i = threadIdx.x; i < 129; i += kUThreads) {
      tab.nlogc[i] = g_logtab.nlogc[i];
      tab.invc[i] = g_logtab.invc[i];
    }
  }
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long k0 = tile * kUTile + (long long)warp * kSeg + (long long)lane * kSegV;

  u128 pre[kSegV];  // lane-local inclusive prefixes
  u128 run = {0ULL, 0ULL};
#pragma unroll
  for (int j = 0; j < kSegV / 4; ++j) {
    uint64_t words[4];
    philox4x64_10((uint64_t)(k0 / 4 + j), 0ULL, 0ULL, 0ULL, seed, inst, words);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long k = k0 + j * 4 + q;
      u128 f = {0ULL, 0ULL};
      if (k < ndraw) {
        if (F32) {
          const float v = (float)(2u * (uint32_t)(words[q] >> 41) + 1u) * 0x1p-24f;  // exact
          f = f_to_fixed128<kZFrac>(-logf(v));
        } else {
          const df z = neg_log_draw(2ULL * (words[q] >> 12) + 1ULL, 53, tab);
          f = f_to_fixed128<kZFrac>(z.hi);
          f = (z.lo >= 0.0f) ? u128_add(f, f_to_fixed128<kZFrac>(z.lo)) : u128_sub(f, f_to_fixed128<kZFrac>(-z.lo));
        }
      }
      run = u128_add(run, f);
      pre[j * 4 + q] = run;
    }
  }
  const u128 incl = warp_incl_scan_v(run, lane);
  const u128 lane_off = u128_sub(incl, run);
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const u128 v = lane < kUWarps ? s_wsum[lane] : u128{0ULL, 0ULL};
    const u128 wi = warp_incl_scan_v(v, lane);
    const u128 agg = shfl_v(wi, kUWarps - 1);
    u128 excl = {0ULL, 0ULL};
    if (tile == 0) {
      if (lane == 0) lb_publish(desc, 0, agg, true);
    } else {
      if (lane == 0) lb_publish(desc, tile, agg, false);
      excl = lb_exclusive(desc, tile, lane, spin_limit, status);
      if (lane == 0) lb_publish_inc(desc, tile, u128_add(excl, agg));
    }
    if (lane < kUWarps) s_woff[lane] = u128_add(excl, u128_sub(wi, v));
  }
  __syncthreads();
  const u128 off = u128_add(s_woff[warp], lane_off);
#pragma unroll
  for (int i = 0; i < kSegV; ++i) {
    const long long k = k0 + i;
    if (k < ndraw - 1) Z[k] = u128_add(off, pre[i]);
    else if (k == ndraw - 1) *Ztot = u128_add(off, pre[i]);
  }
}

template <bool F32>
__global__ void __launch_bounds__(256) k_uniform_norm(long long N, const u128* __restrict__ Z,
                                                      const u128* __restrict__ Ztot, double* __restrict__ U) {
  __shared__ double s_r64;
  __shared__ float s_r32;
  if (threadIdx.x == 0) {
    const u128 t = *Ztot;
    if (F32) s_r32 = __frcp_rn(__uint_as_float(u128_to_f32_bits(t)));
    else s_r64 = __drcp_rn(__longlong_as_double((long long)u128_to_f64_bits(t)));
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const u128 z = Z[i];
    long long ub;
    if (F32) {
      const float u = __fmul_rn(__uint_as_float(u128_to_f32_bits(z)), s_r32);
      ub = (long long)f32_to_f64_bits(__float_as_uint(u));
    } else {
      const double u = __dmul_rn(__longlong_as_double((long long)u128_to_f64_bits(z)), s_r64);
      ub = __double_as_longlong(u);
    }
    // U <= 1 (the product of rounded values may exceed 1 by an ulp)
    if (ub > 0x3FF0000000000000LL) ub = 0x3FF0000000000000LL;
    U[i] = __longlong_as_double(ub);
  }
}

__global__ void k_philox_words(unsigned long long seed, unsigned long long inst, unsigned long long first, long long n,
                               unsigned long long* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long k = first + (unsigned long long)i;
    uint64_t w[4];
    philox4x64_10(k / 4, 0ULL, 0ULL, 0ULL, seed, inst, w);
    out[i] = w[k % 4];
  }
}

cudaError_t init_log_table() {
  LogTab h;
  for (int k = 0; k <= 128; ++k) {
    const double c = 1.0 - k / 256.0;
    const double nl = -std::log(c);
    const double ic = 1.0 / c;
    const float nh = (float)nl, ih = (float)ic;
    h.nlogc[k] = make_float2(nh, (float)(nl - (double)nh));
    h.invc[k] = make_float2(ih, (float)(ic - (double)ih));
  }
  return cudaMemcpyToSymbol(g_logtab, &h, sizeof(h));
}

cudaError_t launch_uniform_scan(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst, void* Z,
                                void* Ztot, void* desc, unsigned* ctr, int* status, int spin_limit, cudaStream_t st) {
  const long long tiles = (ndraw + kUTile - 1) / kUTile;
  if (tiles <= 0) return cudaSuccess;
  if (f32)
    k_uniform_scan<true><<<(unsigned)tiles, kUThreads, 0, st>>>(ndraw, seed, inst, (u128*)Z, (u128*)Ztot,
                                                                (TileDesc<u128>*)desc, ctr, status, spin_limit);
  else
    k_uniform_scan<false><<<(unsigned)tiles, kUThreads, 0, st>>>(ndraw, seed, inst, (u128*)Z, (u128*)Ztot,
                                                                 (TileDesc<u128>*)desc, ctr, status, spin_limit);
  return cudaGetLastError();
}

cudaError_t launch_uniform_norm(bool f32, long long N, const void* Z, const void* Ztot, double* U, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  long long blocks = (N + 255) / 256;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (f32) k_uniform_norm<true><<<(unsigned)blocks, 256, 0, st>>>(N, (const u128*)Z, (const u128*)Ztot, U);
  else k_uniform_norm<false><<<(unsigned)blocks, 256, 0, st>>>(N, (const u128*)Z, (const u128*)Ztot, U);
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
