// Inverse-CDF maps (Eq. 2 of arXiv 2604.01356): r_i = smallest j with
// W_j >= U_i, clamped to M-1.
//
// k_map_seg     the end-to-end map from weights.  It is the divide and
//               conquer of Algorithm 5 applied first to the segment level of
//               W: U is split into groups of G consecutive samples (one warp
//               each); the group's first sample locates its segment with a
//               search down the segment index (integer prefixes on the global
//               grid); later samples of the group walk forward (Algorithm 4's
//               merge walk, with a 32-segment skip); inside a segment the
//               answer comes from exact integer prefixes of the re-read
//               weights.
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
#include "seg_common.cuh"

namespace gbr {

__device__ __forceinline__ long long ldkey(const double* __restrict__ p) {
  return ord_key_bits(__ldg(reinterpret_cast<const long long*>(p)));
}

// ---------------------------------------------------------------------------
// Map from weights, over the segment records of the first weights pass.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u128 seg_pre(const SegPre* __restrict__ pre, long long s) {
  return u128{__ldcg(&pre[s].lo), __ldcg(&pre[s].hi)};
}
__device__ __forceinline__ xf ld_consts_xf(const unsigned long long* p) {
  return {__ldcg(p), __ldcg(p + 1), (long long)__ldcg(p + 2)};
}

// Last segment s with P_s < key: a 32-ary search down the index on the
// monotone 64-bit keys, then an exact fix-up on the 128-bit prefixes only
// when the keys do not already separate key from its neighbours.
__device__ __forceinline__ long long fixup_seg(const SegPre* __restrict__ pre, long long n, long long s,
                                               const u128& key) {
  int guard = 0;
  while (s + 1 < n && u128_lt(seg_pre(pre, s + 1), key) && ++guard < 4096) ++s;
  while (s > 0 && !u128_lt(seg_pre(pre, s), key) && ++guard < 8192) --s;
  return s;
}
__device__ __forceinline__ long long level0_step(const SegPre* __restrict__ pre, const SegIndex& idx, long long c,
                                                 unsigned long long kb, const u128& key, int lane) {
  const long long j = c * 32 + lane;
  const unsigned long long e = j < idx.lvl_n[0] ? __ldcg(idx.lvl[0] + j) : ~0ULL;
  const int cnt = __popc(__ballot_sync(0xFFFFFFFFu, e < kb));
  const long long s = c * 32 + (cnt > 0 ? cnt - 1 : 0);
  const unsigned long long next = __shfl_sync(0xFFFFFFFFu, e, cnt & 31);
  // key(P_s) < kb < key(P_{s+1}) proves P_s < key <= P_{s+1} (monotone keys)
  if (cnt > 0 && cnt < 32 && next != kb) return s;
  return fixup_seg(pre, idx.n, s, key);
}
__device__ __forceinline__ long long locate_seg(const SegPre* __restrict__ pre, const SegIndex& idx,
                                                unsigned long long kb, const u128& key, int lane) {
  long long c = 0;
  for (int l = idx.nlev - 1; l >= 1; --l) {
    const long long j = c * 32 + lane;
    const unsigned long long e = j < idx.lvl_n[l] ? __ldcg(idx.lvl[l] + j) : ~0ULL;
    const int cnt = __popc(__ballot_sync(0xFFFFFFFFu, e < kb));
    c = c * 32 + (cnt > 0 ? cnt - 1 : 0);
  }
  return level0_step(pre, idx, c, kb, key, lane);
}
// Same with level 1 of the index staged in shared memory.
__device__ __forceinline__ long long locate_seg_smem(const SegPre* __restrict__ pre, const SegIndex& idx,
                                                     const unsigned long long* __restrict__ top, int ntop,
                                                     unsigned long long kb, const u128& key, int lane) {
  int lo = 0, hi = ntop;  // first entry >= kb
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if (top[m] < kb) lo = m + 1;
    else hi = m;
  }
  return level0_step(pre, idx, lo > 0 ? lo - 1 : 0, kb, key, lane);
}

// Head segment of binary64 weights: number of elements j with
// sum_{k<=j} w_k < rem (rem = key - P_s as a value).  The weights are put on a
// 128-bit grid scaled to rem (unit 2^(rem.e + 25), so rem is about 2^100
// units) and summed with saturation at 2^102: the decision is exact up to 512
// units, i.e. 2^-91 of rem, whatever the dynamic range of the segment.
__device__ __forceinline__ u128 sat_add(u128 a, u128 b) {
  const u128 s = u128_add(a, b);
  return (s.hi >> 38) ? u128{0ULL, 1ULL << 38} : s;  // cap at 2^102
}
__device__ __forceinline__ u128 head_val(uint64_t b, long long ue) {
  const uint32_t t = (uint32_t)(b >> 52);
  if (t >= 0x7FFu) return u128{0ULL, 0ULL};
  const uint64_t m = (b & 0xFFFFFFFFFFFFFULL) | (t ? (1ULL << 52) : 0ULL);
  const long long sh = (long long)(t > 1u ? t : 1u) - 1075 - ue;
  if (sh >= 50) return u128{0ULL, m ? (1ULL << 38) : 0ULL};
  if (sh >= 0) {
    uint64_t vh = 0, vl = m;
    shl128(vh, vl, (int)sh);
    return u128{vl, vh};
  }
  return sh > -64 ? u128{m >> (-sh), 0ULL} : u128{0ULL, 0ULL};
}
template <bool kVec>
__device__ __forceinline__ int head_count(const double* __restrict__ w, long long base, long long M, const xf& rem,
                                          int lane) {
  using Tr = FixedTraits<double>;
  if (xf_zero(rem)) return 0;
  // R = rem / unit = rem.m >> 25, in [2^100, 2^101)
  uint64_t rh = rem.hi, rl = rem.lo;
  shr128(rh, rl, 25);
  const long long ue = rem.e + 25;
  Tr::Bits b[kSegV];
  load_seg_blocked<double, kVec>(w, base, M, lane, b);
  u128 run = {0ULL, 0ULL};
#pragma unroll
  for (int i = 0; i < kSegV; ++i) run = sat_add(run, head_val(b[i], ue));
  u128 incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u128 t = shfl_up_v(incl, o);
    if (lane >= o) incl = sat_add(t, incl);
  }
  u128 x = shfl_up_v(incl, 1);
  if (lane == 0) x = u128{0ULL, 0ULL};
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < kSegV; ++i) {
    x = sat_add(x, head_val(b[i], ue));
    cnt += (x.hi < rh || (x.hi == rh && x.lo < rl)) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
  return cnt;
}
template <bool kVec>
__device__ __forceinline__ int head_count(const float*, long long, long long, const xf&, int) {
  return 0;  // binary32 weights never need it: their grid is finer than the tolerance
}

template <typename T, bool kVec>
__global__ void __launch_bounds__(256, 2) k_map_seg(const T* __restrict__ w, long long M,
                                                    const SegRec* __restrict__ seg, const SegPre* __restrict__ pre,
                                                    SegIndex idx, const PathConsts* __restrict__ consts,
                                                    const u128* __restrict__ Z, long long N, int G, int ntop,
                                                    int* __restrict__ out) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  extern __shared__ unsigned long long s_top[];  // level 1 of the index when ntop > 0
  __shared__ xf s_c;
  __shared__ u128 s_S;
  __shared__ long long s_ge;
  __shared__ int s_Emax;
  const long long gw0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // the first sample's spacing sum is fetched while the index is staged
  u128 z_first = {0ULL, 0ULL};
  if (gw0 * (long long)G < N) z_first = Z[gw0 * (long long)G];
  for (int t = threadIdx.x; t < ntop; t += blockDim.x) s_top[t] = __ldcg(idx.lvl[1] + t);
  if (threadIdx.x == 0) {
    s_c = ld_consts_xf(consts->c);
    s_S = u128{__ldcg(consts->S), __ldcg(consts->S + 1)};
    s_ge = (long long)__ldcg((const unsigned long long*)&consts->ge);
    s_Emax = (int)__ldcg((const unsigned long long*)&consts->Emax);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long gw = gw0;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nseg = idx.n;
  for (long long g = gw; g * (long long)G < N; g += nw) {
    const long long i0 = g * (long long)G;
    const long long i1 = (i0 + G < N) ? i0 + G : N;
    long long s = -1;  // segment held in registers
    u128 Ps = {0ULL, 0ULL}, Pn = {0ULL, 0ULL};
    int sh = 0, len = 0;
    bool head = false;
    unsigned long long F = 0;
    uint64_t pref[kSegV];
#pragma unroll
    for (int q = 0; q < kSegV; ++q) pref[q] = 0;
    for (long long i = i0; i < i1; ++i) {
      const u128 z = (g == gw0 && i == i0) ? z_first : Z[i];
      const u128 key = map_key(s_c, z);  // ceil(U_i * S) in grid units
      if (s < 0 || !(u128_lt(Ps, key) && !u128_lt(Pn, key))) {
        const unsigned long long kb = u128_key(key);
        long long ns = -1;
        if (s >= 0 && u128_lt(Pn, key)) {
          // forward skip over the next 32 segments (merge walk)
          const long long j = s + 1 + lane;
          const unsigned long long e = j < nseg ? __ldcg(idx.lvl[0] + j) : ~0ULL;
          const int cnt = __popc(__ballot_sync(0xFFFFFFFFu, e < kb));
          if (cnt < 32) ns = fixup_seg(pre, nseg, s + cnt, key);
        }
        if (ns < 0)
          ns = ntop > 0 ? locate_seg_smem(pre, idx, s_top, ntop, kb, key, lane) : locate_seg(pre, idx, kb, key, lane);
        s = ns;
        // the segment's record, prefixes and weights are independent loads
        Bits b[kSegV];
        load_seg_blocked<T, kVec>(w, s * kSeg, M, lane, b);
        const SegRec r = seg[s];
        Ps = seg_pre(pre, s);
        Pn = (s + 1 < nseg) ? seg_pre(pre, s + 1) : s_S;
        sh = r.E - s_Emax + kGridHead;
        len = r.len;
        F = r.F;
        const xf Px = xf_make(Ps.hi, Ps.lo, 0);
        head = sizeof(T) == 8 && (xf_zero(Px) || Px.e + kXfTop < (long long)sh + 50);
        if (!head) seg_prefixes<T>(b, (uint32_t)r.E, lane, pref);
      }
      const u128 rem = u128_lt(Ps, key) ? u128_sub(key, Ps) : u128{0ULL, 0ULL};
      int cnt;
      if (head) {
        cnt = head_count<kVec>(w, s * kSeg, M, xf_make(rem.hi, rem.lo, s_ge), lane);
      } else {
        // first element whose exact prefix reaches K = ceil(rem / unit_s)
        const unsigned long long K = ceil_units(rem, sh, F);
        cnt = 0;
#pragma unroll
        for (int q = 0; q < kSegV; ++q) cnt += pref[q] < K ? 1 : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      }
      if (lane == 0) {
        const long long j = cnt < len ? cnt : len - 1;
        long long r = s * kSeg + j;
        if (r > M - 1) r = M - 1;
        out[i] = (int)r;
      }
    }
  }
}

constexpr int kMapTopMax = 6144;  // entries (48 KB, the default dynamic shared-memory limit)

template <typename T, bool kVec>
static cudaError_t map_seg_t(const void* w, long long M, const SegRec* seg, const SegPre* pre, const SegIndex& idx,
                             const PathConsts* consts, const void* Z, long long N, int G, int* out, cudaStream_t st) {
  const long long groups = (N + G - 1) / G;
  long long blocks = (groups + 7) / 8;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  // stage level 1 of the segment index in shared memory when it is small
  int ntop = 0;
  if (idx.nlev >= 2 && idx.lvl_n[1] <= kMapTopMax) ntop = (int)idx.lvl_n[1];
  const size_t smem = (size_t)ntop * sizeof(unsigned long long);
  k_map_seg<T, kVec><<<(unsigned)blocks, 256, smem, st>>>((const T*)w, M, seg, pre, idx, consts, (const u128*)Z, N, G,
                                                          ntop, out);
  return cudaGetLastError();
}

cudaError_t launch_map_seg(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const SegPre* pre,
                           const SegIndex& idx, const PathConsts* consts, const void* Z, long long N, int G, int* out,
                           cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (f32) return vec ? map_seg_t<float, true>(w, M, seg, pre, idx, consts, Z, N, G, out, st)
                      : map_seg_t<float, false>(w, M, seg, pre, idx, consts, Z, N, G, out, st);
  return vec ? map_seg_t<double, true>(w, M, seg, pre, idx, consts, Z, N, G, out, st)
             : map_seg_t<double, false>(w, M, seg, pre, idx, consts, Z, N, G, out, st);
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
