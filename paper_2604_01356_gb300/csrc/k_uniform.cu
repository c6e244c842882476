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
