// Inverse-CDF maps (Eq. 2 of arXiv 2604.01356): r_i = smallest j with
// W_j >= U_i, clamped to M-1.
//
// k_map_seg     the end-to-end map from weights.  It is the divide and
//               conquer of Algorithm 5 applied first to the segment level of
//               W: U is split into groups of G consecutive samples (one warp
//               each); the group's first sample locates its segment with a
//               32-ary search down the segment index; later samples of the
//               group walk forward (Algorithm 4's merge walk, with a 32-wide
//               skip); inside a segment the answer comes from exact integer
//               prefixes of the re-read weights.
// k_map_dac     Algorithm 5 on a given W: split U every L samples, find the
//               split points by warp-cooperative 32-ary search, then resolve
//               each leaf inside the W range its two split points bound -
//               staged in shared memory when it is small, else by per-sample
//               binary search (the single-U base case).
// k_map_binary  Algorithm 3: one full-range binary search (Algorithm 2) per u.
// k_map_linear  Algorithm 4: every W element read once; each block owns a W
//               tile, finds its samples by searching U, merge-walks them.
//
// Comparisons on a given binary64 W are exact: values are compared through
// their total-order integer keys, which agree with IEEE comparison for every
// non-NaN value, so all three maps return bit-identical indices.
#include "common.cuh"
#include "internal.h"

namespace gbr {

__device__ __forceinline__ long long ldkey(const double* __restrict__ p) {
  return ord_key_bits(__ldg(reinterpret_cast<const long long*>(p)));
}

// ---------------------------------------------------------------------------
// Map from weights, over the segment records of the first weights pass.
// ---------------------------------------------------------------------------
template <typename T, bool kVec>
__device__ __forceinline__ void load_blocked(const T* __restrict__ w, long long base, long long M, int lane,
                                             typename FixedTraits<T>::Bits (&b)[kSegV]) {
  using Bits = typename FixedTraits<T>::Bits;
  const long long e0 = base + (long long)lane * kSegV;
  if (kVec && e0 + kSegV <= M) {
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

__device__ __forceinline__ dd seg_P(const SegRec* seg, long long s) { return dd{seg[s].P_hi, seg[s].P_lo}; }

// Last segment s with P_s < key (binary64-pair comparison).  A 32-ary search
// on the hi parts down the index, then an exact fix-up on (hi, lo).
__device__ __forceinline__ long long locate_segment(const SegRec* __restrict__ seg, const SegIndex& idx, dd key,
                                                    int lane) {
  const unsigned long long kb = (unsigned long long)__double_as_longlong(key.hi);
  long long c = 0;
  for (int l = idx.nlev - 1; l >= 0; --l) {
    const long long j = c * 32 + lane;
    const unsigned long long e = j < idx.lvl_n[l] ? __ldcg(idx.lvl[l] + j) : ~0ULL;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, e < kb);
    const int cnt = __popc(bal);
    c = c * 32 + (cnt > 0 ? cnt - 1 : 0);
  }
  long long s = c;
  int guard = 0;
  while (s + 1 < idx.nseg && dd_lt(seg_P(seg, s + 1), key) && ++guard < 4096) ++s;
  while (s > 0 && dd_le(key, seg_P(seg, s)) && ++guard < 8192) --s;
  return s;
}

// Head segment of binary64 weights: count the elements whose binary64-pair
// cumulative value P_s + sum_{k<=j} w_k is still below key.
template <bool kVec>
__device__ __forceinline__ int head_count(const double* __restrict__ w, long long base, long long M, dd Ps, dd key,
                                       int lane) {
  using Tr = FixedTraits<double>;
  Tr::Bits b[kSegV];
  load_blocked<double, kVec>(w, base, M, lane, b);
  dd run = {0.0, 0.0};
#pragma unroll
  for (int i = 0; i < kSegV; ++i) run = dd_add_d(run, Tr::bad(b[i]) ? 0.0 : __longlong_as_double((long long)b[i]));
  dd x = warp_incl_scan_v(run, lane);
  x = dd_add(dd_add(x, dd{-run.hi, -run.lo}), Ps);
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < kSegV; ++i) {
    x = dd_add_d(x, Tr::bad(b[i]) ? 0.0 : __longlong_as_double((long long)b[i]));
    cnt += dd_lt(x, key) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  return cnt;
}
template <bool kVec>
__device__ __forceinline__ int head_count(const float*, long long, long long, dd, dd, int) {
  return 0;  // binary32 weights never need it: their grid is finer than the tolerance
}

template <typename T, bool kVec>
__global__ void __launch_bounds__(256, 2) k_map_seg(const T* __restrict__ w, long long M, const SegRec* __restrict__ seg,
                                                 SegIndex idx, const dd* __restrict__ total,
                                                 const double* __restrict__ U, long long N, int G,
                                                 int* __restrict__ out) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nseg = idx.nseg;
  const dd S = *total;
  for (long long g = gw; g * (long long)G < N; g += nw) {
    const long long i0 = g * (long long)G;
    const long long i1 = (i0 + G < N) ? i0 + G : N;
    long long s = -1;     // segment held in registers
    dd Ps = {0, 0}, Pn = {0, 0};
    int E = 1, len = 0;
    bool head = false;
    unsigned long long F = 0;
    uint64_t pref[kSegV];
#pragma unroll
    for (int i = 0; i < kSegV; ++i) pref[i] = 0;
    for (long long i = i0; i < i1; ++i) {
      dd key = {0.0, 0.0};
      if (lane == 0) key = dd_mul(dd{__ldg(U + i), 0.0}, S);
      key = shfl_v(key, 0);
      if (s < 0 || !(dd_lt(Ps, key) && dd_le(key, Pn))) {
        long long ns = -1;
        if (s >= 0 && dd_lt(Pn, key)) {
          // forward skip over the next 32 segments (merge walk)
          const long long j = s + 1 + lane;
          const unsigned long long kb = (unsigned long long)__double_as_longlong(key.hi);
          const unsigned long long e = j < nseg ? __ldcg(idx.lvl[0] + j) : ~0ULL;
          const unsigned bal = __ballot_sync(0xFFFFFFFFu, e < kb);
          const int cnt = __popc(bal);
          if (cnt < 32) {
            ns = s + cnt;
            int guard = 0;
            while (ns + 1 < nseg && dd_lt(seg_P(seg, ns + 1), key) && ++guard < 4096) ++ns;
            while (ns > 0 && dd_le(key, seg_P(seg, ns)) && ++guard < 8192) --ns;
          }
        }
        if (ns < 0) ns = locate_segment(seg, idx, key, lane);
        s = ns;
        const SegRec r = seg[s];
        Ps = dd{r.P_hi, r.P_lo};
        Pn = (s + 1 < nseg) ? seg_P(seg, s + 1) : S;
        E = r.E;
        len = r.len;
        F = r.F;
        head = sizeof(T) == 8 && head_segment(r.P_hi, E, Tr::kBias + Tr::kShift);
        Bits b[kSegV];
        load_blocked<T, kVec>(w, s * kSeg, M, lane, b);
        uint64_t run = 0;
#pragma unroll
        for (int q = 0; q < kSegV; ++q) {
          run += to_fixed<T>(b[q], E);
          pref[q] = run;
        }
        const uint64_t incl = warp_incl_scan_u64(run, lane);
        const uint64_t off = incl - run;
#pragma unroll
        for (int q = 0; q < kSegV; ++q) pref[q] += off;
      }
      if (head) {
        const int hc = head_count<kVec>(w, s * kSeg, M, Ps, key, lane);
        if (lane == 0) {
          long long j = hc < len ? hc : len - 1;
          long long r = s * kSeg + j;
          if (r > M - 1) r = M - 1;
          out[i] = (int)r;
        }
        continue;
      }
      // K = ceil((key - P_s) / unit): the first element whose exact prefix
      // reaches K is the answer.  Clamped to [1, F].
      unsigned long long K = 1;
      if (lane == 0) {
        const dd rem = dd_sub(key, Ps);
        const int sc = Tr::kBias + Tr::kShift - E;
        const double th = ldexp2(rem.hi, sc), tl = ldexp2(rem.lo, sc);
        if (!(th > 0.0)) {
          K = 1;
        } else if (th >= 9.2e18) {
          K = F;
        } else {
          const double c = ceil(th);
          if (c != th) K = (unsigned long long)c;
          else K = (unsigned long long)th + (unsigned long long)(long long)ceil(tl);
        }
        if (K > F) K = F;
        if (K < 1) K = 1;
      }
      K = __shfl_sync(0xFFFFFFFFu, K, 0);
      int cnt = 0;
#pragma unroll
      for (int q = 0; q < kSegV; ++q) cnt += pref[q] < K ? 1 : 0;
#pragma unroll
      for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      if (lane == 0) {
        long long j = cnt < len ? cnt : len - 1;
        long long r = s * kSeg + j;
        if (r > M - 1) r = M - 1;
        out[i] = (int)r;
      }
    }
  }
}

template <typename T, bool kVec>
static cudaError_t map_seg_t(const void* w, long long M, const SegRec* seg, const SegIndex& idx, const void* total,
                             const double* U, long long N, int G, int* out, cudaStream_t st) {
  const long long groups = (N + G - 1) / G;
  long long blocks = (groups + 7) / 8;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_map_seg<T, kVec><<<(unsigned)blocks, 256, 0, st>>>((const T*)w, M, seg, idx, (const dd*)total, U, N, G, out);
  return cudaGetLastError();
}

cudaError_t launch_map_seg(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const SegIndex& idx,
                           const void* total, const double* U, long long N, int G, int* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (f32) return vec ? map_seg_t<float, true>(w, M, seg, idx, total, U, N, G, out, st)
                      : map_seg_t<float, false>(w, M, seg, idx, total, U, N, G, out, st);
  return vec ? map_seg_t<double, true>(w, M, seg, idx, total, U, N, G, out, st)
             : map_seg_t<double, false>(w, M, seg, idx, total, U, N, G, out, st);
}

// ---------------------------------------------------------------------------
// Maps on a given binary64 W.
// ---------------------------------------------------------------------------

// Algorithm 2 on W[a..b] (0-based, inclusive): smallest m with W_m >= key,
// or b if none.
__device__ __forceinline__ long long binary_search(const double* __restrict__ W, long long a, long long b,
                                                   long long key) {
  while (a < b) {
    const long long m = (a + b) >> 1;
    if (ldkey(W + m) < key) a = m + 1;
    else b = m;
  }
  return b;
}

__global__ void __launch_bounds__(256) k_map_binary(const double* __restrict__ W, long long M,
                                                    const double* __restrict__ U, long long N, int* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride)
    out[i] = (int)binary_search(W, 0, M - 1, ldkey(U + i));
}

// Warp-cooperative 32-ary lower bound on W[lo..hi]; the answer is known to
// lie in [lo, hi] (hi = M-1 stands for "clamp").  All 32 lanes must call it.
__device__ __forceinline__ long long warp_lower_bound(const double* __restrict__ W, long long lo, long long hi,
                                                      long long key, int lane) {
  while (hi - lo + 1 > 32) {
    const long long n = hi - lo + 1;
    const long long step = (n + 31) / 32;
    long long p = lo + (long long)(lane + 1) * step - 1;
    if (p > hi) p = hi;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, ldkey(W + p) >= key);
    if (bal == 0) return hi;
    const int f = __ffs(bal) - 1;
    long long nlo = lo;
    if (f > 0) {
      long long q = lo + (long long)f * step - 1;
      if (q > hi) q = hi;
      nlo = q + 1;
    }
    long long nhi = lo + (long long)(f + 1) * step - 1;
    if (nhi > hi) nhi = hi;
    lo = nlo;
    hi = nhi;
  }
  const long long p = lo + lane;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, p <= hi && ldkey(W + (p <= hi ? p : hi)) >= key);
  return bal ? lo + (__ffs(bal) - 1) : hi;
}

// Algorithm 5, GPU form.  Each warp owns leaves of L consecutive samples.
constexpr int kDacWarps = 8;
template <int kStage>
__global__ void __launch_bounds__(256) k_map_dac(const double* __restrict__ W, long long M,
                                                 const double* __restrict__ U, long long N, int L, int stage_max,
                                                 int* __restrict__ out) {
  __shared__ long long s_stage[kDacWarps][kStage];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nleaf = (N + L - 1) / L;
  long long* st = s_stage[warp];
  for (long long leaf = gw; leaf < nleaf; leaf += nw) {
    const long long a = leaf * (long long)L;
    const long long b = (a + L < N ? a + L : N) - 1;
    // split points: the leaf's last and first sample (Algorithm 2 on the
    // range the paper's recursion would pass down; here the full W for the
    // last one and [0, r_b] for the first)
    const long long kb = ldkey(U + b);
    const long long rb = warp_lower_bound(W, 0, M - 1, kb, lane);
    if (a == b) {
      if (lane == 0) out[a] = (int)rb;
      continue;
    }
    const long long ka = ldkey(U + a);
    const long long ra = warp_lower_bound(W, 0, rb, ka, lane);
    if (lane == 0) {
      out[a] = (int)ra;
      out[b] = (int)rb;
    }
    // leaf: samples a+1 .. b-1 have answers in [ra, rb]
    const long long range = rb - ra + 1;
    if (range <= stage_max && range <= kStage) {
      for (long long j = lane; j < range; j += 32) st[j] = ldkey(W + ra + j);
      __syncwarp();
      for (long long i = a + 1 + lane; i < b; i += 32) {
        const long long k = ldkey(U + i);
        long long lo = 0, hi = range - 1;
        while (lo < hi) {
          const long long m = (lo + hi) >> 1;
          if (st[m] < k) lo = m + 1;
          else hi = m;
        }
        out[i] = (int)(ra + hi);
      }
      __syncwarp();
    } else {
      for (long long i = a + 1 + lane; i < b; i += 32) out[i] = (int)binary_search(W, ra, rb, ldkey(U + i));
    }
  }
}

// Algorithm 4, GPU form: block t owns W[t*TW, (t+1)*TW) and the samples whose
// answers fall there, W[t0-1] < u <= W[t1-1]; it stages the tile in shared
// memory and each thread merge-walks a contiguous run of those samples.
constexpr int kLinTile = 2048;
__device__ __forceinline__ long long upper_bound_U(const double* __restrict__ U, long long N, long long key) {
  long long a = 0, b = N;  // first i with key(U_i) > key
  while (a < b) {
    const long long m = (a + b) >> 1;
    if (ldkey(U + m) <= key) a = m + 1;
    else b = m;
  }
  return a;
}

__global__ void __launch_bounds__(256) k_map_linear(const double* __restrict__ W, long long M,
                                                    const double* __restrict__ U, long long N, int* __restrict__ out) {
  __shared__ long long s_w[kLinTile];
  __shared__ long long s_rng[2];
  const long long t0 = (long long)blockIdx.x * kLinTile;
  const long long t1 = (t0 + kLinTile < M) ? t0 + kLinTile : M;
  const int len = (int)(t1 - t0);
  if (threadIdx.x == 0) s_rng[0] = t0 == 0 ? 0 : upper_bound_U(U, N, ldkey(W + t0 - 1));
  if (threadIdx.x == 32) s_rng[1] = t1 == M ? N : upper_bound_U(U, N, ldkey(W + t1 - 1));
  for (int j = threadIdx.x; j < len; j += blockDim.x) s_w[j] = ldkey(W + t0 + j);
  __syncthreads();
  const long long i0 = s_rng[0], i1 = s_rng[1];
  if (i1 <= i0) return;
  const long long cnt = i1 - i0;
  const long long per = (cnt + blockDim.x - 1) / blockDim.x;
  const long long c0 = i0 + (long long)threadIdx.x * per;
  const long long c1 = (c0 + per < i1) ? c0 + per : i1;
  if (c0 >= c1) return;
  // first sample of the run: binary search in the tile, then Algorithm 4's walk
  long long k = ldkey(U + c0);
  int lo = 0, hi = len - 1;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (s_w[m] < k) lo = m + 1;
    else hi = m;
  }
  int j = hi;
  out[c0] = (int)(t0 + j);
  for (long long i = c0 + 1; i < c1; ++i) {
    k = ldkey(U + i);
    while (j < len - 1 && s_w[j] < k) ++j;
    out[i] = (int)(t0 + j);
  }
}

cudaError_t launch_map_binary(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  long long blocks = (N + 255) / 256;
  const long long cap = (long long)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_map_binary<<<(unsigned)blocks, 256, 0, st>>>(W, M, U, N, out);
  return cudaGetLastError();
}

cudaError_t launch_map_linear(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const long long tiles = (M + kLinTile - 1) / kLinTile;
  k_map_linear<<<(unsigned)tiles, 256, 0, st>>>(W, M, U, N, out);
  return cudaGetLastError();
}

cudaError_t launch_map_dac(const double* W, long long M, const double* U, long long N, int L, int stage_max, int* out,
                           cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const long long leaves = (N + L - 1) / L;
  long long blocks = (leaves + kDacWarps - 1) / kDacWarps;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_map_dac<512><<<(unsigned)blocks, 256, 0, st>>>(W, M, U, N, L, stage_max, out);
  return cudaGetLastError();
}

}  // namespace gbr
