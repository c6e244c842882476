// The step after resampling (Sec. I of arXiv 2604.01356): the new particle
// set x'_i = x_{r_i}, i = 1..N, a gather of N rows of D elements by the
// resampled indices.
//
// GB300 form: pure data movement, HBM-bound.  The N rows are cut into
// 16-byte (or 8- / 4-byte, when the row length or the pointers do not allow
// 16) units; consecutive threads take consecutive units, so a row longer than
// 128 bytes is read and written by whole sectors, and short rows pack several
// to a warp.  Units per row are a power of two times the unit when possible
// (shift instead of divide); the grid is a whole number of CTAs per SM.
// An index outside [0, M) writes zeros for its row and latches RS_EINVAL in
// the status word.
#include "common.cuh"
#include "internal.h"

namespace gbr {

namespace {

template <typename V>
__global__ void __launch_bounds__(256) k_gather(const V* __restrict__ x, long long M, long long upr, int lg_upr,
                                                const int* __restrict__ idx, long long N, V* __restrict__ y,
                                                int* status) {
  const long long total = N * upr;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += stride) {
    const long long i = lg_upr >= 0 ? (u >> lg_upr) : u / upr;
    const long long c = u - i * upr;
    const long long j = __ldg(idx + i);
    V v;
    if (j >= 0 && j < M) {
      v = __ldg(x + j * upr + c);
    } else {
      v = V{};
      if (c == 0) raise_status(status, ST_EINVAL);
    }
    y[u] = v;
  }
}

template <typename V>
cudaError_t gather_t(const void* x, long long M, long long row_bytes, const int* idx, long long N, void* y,
                     int* status, cudaStream_t st) {
  const long long upr = row_bytes / (long long)sizeof(V);
  int lg = -1;
  if ((upr & (upr - 1)) == 0) {
    lg = 0;
    while ((1LL << lg) < upr) ++lg;
  }
  const long long total = N * upr;
  long long blocks = (total + 255) / 256;
  const long long cap = (long long)num_sms() * 8;  // 8 resident CTAs of 256 per SM
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_gather<V><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const V*>(x), M, upr, lg, idx, N, static_cast<V*>(y),
                                                status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gather(const void* x, long long M, long long row_bytes, const int* idx, long long N, void* y,
                          int* status, cudaStream_t st) {
  if (N <= 0 || row_bytes <= 0) return cudaSuccess;
  const uintptr_t al = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | (uintptr_t)row_bytes;
  if ((al & 15) == 0) return gather_t<uint4>(x, M, row_bytes, idx, N, y, status, st);
  if ((al & 7) == 0) return gather_t<unsigned long long>(x, M, row_bytes, idx, N, y, status, st);
  return gather_t<unsigned>(x, M, row_bytes, idx, N, y, status, st);
}

}  // namespace gbr
