// Cumulative weights (Eq. 3 of arXiv 2604.01356): W_j = sum_{k<=j} w_k / S,
// S = sum_k w_k.  The paper only notes that W can be formed alongside the
// normalisation; this file is that step.
//
// GB300 form (no binary64 arithmetic per weight, segment or tile):
//  reduce   one warp per 512-element segment reads its weights with 16-byte
//           coalesced loads, takes the segment's largest exponent E (one warp
//           max) and sums the weights EXACTLY as integers on the segment grid
//           2^(E - bias - shift).  Pure streaming: no inter-block waits.
//  prefix   a small scan over the segment sums (128-bit-mantissa values):
//           up to 128 blocks of 1024 threads, each summing the reduce
//           pass's tile aggregates before it (no inter-block waits), then
//           scanning its own segments; beyond 2^21 segments, blocks chained
//           by decoupled
//           look-back.  Writes each segment's exclusive prefix P_s, a search
//           index over P and the per-call constants (S, S / Z_{N+1}, and 1/S
//           when W is written).
//  write    (only when W itself is requested) one warp per segment re-reads
//           the weights and writes W_j = (P_s + F_j unit) / S rounded to
//           binary64 by integer operations, clamped so that W is
//           non-decreasing and W_M = 1.
#include "common.cuh"
#include "internal.h"

namespace gbr {

constexpr int kWThreads = 256;
constexpr int kWWarps = kWThreads / kWarp;
constexpr int kPThreads = 256;
constexpr int kPTile = kPThreads;  // one segment per thread
static_assert(kPTile == kSegPrefixTile, "prefix tile");

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
__device__ __forceinline__ xf seg_P_xf(const SegRec& r) { return {r.Pm_lo, r.Pm_hi, r.Pe}; }

// ---- reduce: exact segment sums ------------------------------------------
// One warp per segment; each block of 8 warps also writes its tile aggregate
// (the sum of its 8 segments as a 128-bit-mantissa value) for the prefix pass.
template <typename T, bool kVec>
__global__ void __launch_bounds__(kWThreads, 4) k_w_reduce(const T* __restrict__ w, long long M, long long nseg,
                                                       SegRec* __restrict__ seg, xf* __restrict__ tagg,
                                                       int* status) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  constexpr int kBS = Tr::kBias + Tr::kShift;
  __shared__ xf s_val[kWWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long s = ((long long)blockIdx.x * kWThreads + threadIdx.x) >> 5;
  xf v = lb_zero<xf>();
  if (s < nseg) {
    const long long base = s * kSeg;
    Bits b[kSegV];
    load_seg_striped<T, kVec>(w, base, M, lane, b);
    uint32_t emax = 0, invalid = 0;
#pragma unroll
    for (int i = 0; i < kSegV; ++i) {
      emax = max(emax, seg_top<T>(b[i]));
      invalid |= Tr::valid_top(b[i]) ^ 1u;
    }
    emax = __reduce_max_sync(0xFFFFFFFFu, emax);
    const uint32_t E = emax > 1u ? emax : 1u;
    if (__any_sync(0xFFFFFFFFu, invalid)) {
      // rare: tell a negative zero (valid) from negative, NaN or infinite weights
      bool bad = false;
#pragma unroll
      for (int i = 0; i < kSegV; ++i) bad |= Tr::bad(b[i]);
      if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) raise_status(status, ST_ENONFINITE);
    }
    uint64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kSegV; ++i) sum += Tr::fixed(b[i], E);
    sum = warp_sum_u64(sum);
    if (lane == 0) {
      const long long rem = M - base;
      seg[s].F = sum;
      seg[s].E = (int)E;
      seg[s].len = (int)(rem < kSeg ? rem : kSeg);
      v = xf_from_u64(sum, (long long)E - kBS);
    }
  }
  if (lane == 0) s_val[warp] = v;
  __syncthreads();
  if (warp == 0) {
    xf a = lane < kWWarps ? s_val[lane] : lb_zero<xf>();
#pragma unroll
    for (int o = kWWarps / 2; o; o >>= 1) {
      const xf t = shfl_down_v(a, o);
      if (lane + o < kWWarps) a = xf_add(a, t);
    }
    if (lane == 0) tagg[blockIdx.x] = a;
  }
}

// ---- prefix: exclusive prefixes over segments, index and constants -------
// The per-call constants, written by the thread that owns the last segment:
// S, c = S * (1/Z_{N+1}) (an integer product; the reciprocal comes from the
// spacing scan) and, only when W itself is written, 1/S (binary64-pair
// division, out of line).
__device__ __noinline__ void write_consts(PathConsts* consts, xf S, bool with_z, bool need_invS, int* status) {
  st_xf(consts->S, S);
  if (xf_zero(S)) {
    raise_status(status, ST_EZEROSUM);
    st_xf(consts->invS, lb_zero<xf>());
    st_xf(consts->c, lb_zero<xf>());
    return;
  }
  if (need_invS) st_xf(consts->invS, xf_div(xf_from_u64(1, 0), S));
  st_xf(consts->c, with_z ? xf_mul(S, ld_xf(consts->invZ)) : lb_zero<xf>());
}

__device__ __forceinline__ void write_seg_prefix(SegRec* __restrict__ seg, const SegIndex& idx, long long s,
                                                 const xf& P) {
  seg[s].Pm_lo = P.lo;
  seg[s].Pm_hi = P.hi;
  seg[s].Pe = P.e;
  const unsigned long long key = xf_key(P);
  seg[s].key = key;
#pragma unroll 1
  for (int l = 0; l < idx.nlev; ++l) {
    const long long mask = (1LL << (5 * l)) - 1;
    if (s & mask) break;
    idx.lvl[l][s >> (5 * l)] = key;
  }
}

// Block b owns kPThreads*items consecutive segments.  Its base (the sum of all
// earlier segments) is the sum of the tile aggregates before it, read directly
// by the block's threads; then a block-wide scan of its own segment values
// gives every P_s.  No block waits for another.
constexpr int kRedMaxBlocks = 128;
constexpr int kRedMaxItems = 16;
constexpr int kRThreads = 1024;
template <int kBS>
__global__ void __launch_bounds__(kRThreads) k_seg_prefix_red(long long nseg, int items, SegRec* __restrict__ seg,
                                                             const xf* __restrict__ tagg, SegIndex idx,
                                                             PathConsts* consts, bool with_z, bool need_invS,
                                                             int* status) {
  __shared__ xf s_w[kRThreads / 32];
  __shared__ xf s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long spb = (long long)kRThreads * items;  // segments per block
  const long long first = (long long)blockIdx.x * spb;
  // base = sum of tile aggregates [0, first/8): each round issues four
  // independent loads per thread before adding (one memory round trip per
  // 4*blockDim aggregates)
  const long long ntile = first / kWWarps;
  xf acc = lb_zero<xf>();
#pragma unroll 1
  for (long long t0 = 0; t0 < ntile; t0 += 4 * kRThreads) {
    const long long t = t0 + tid;
    const xf a0 = t < ntile ? tagg[t] : lb_zero<xf>();
    const xf a1 = t + kRThreads < ntile ? tagg[t + kRThreads] : lb_zero<xf>();
    const xf a2 = t + 2 * kRThreads < ntile ? tagg[t + 2 * kRThreads] : lb_zero<xf>();
    const xf a3 = t + 3 * kRThreads < ntile ? tagg[t + 3 * kRThreads] : lb_zero<xf>();
    acc = xf_add(acc, xf_add(xf_add(a0, a1), xf_add(a2, a3)));
  }
  xf part = acc;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const xf x = shfl_down_v(part, o);
    part = xf_add(part, x);
  }
  if (lane == 0) s_w[warp] = part;
  __syncthreads();
  if (warp == 0) {
    xf a = lane < kRThreads / 32 ? s_w[lane] : lb_zero<xf>();
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const xf x = shfl_down_v(a, o);
      if (lane + o < kRThreads / 32) a = xf_add(a, x);
    }
    if (lane == 0) s_base = a;
  }
  __syncthreads();
  // this thread's run of `items` segments
  const long long s0 = first + (long long)tid * items;
  xf run = lb_zero<xf>();
#pragma unroll 1
  for (int q = 0; q < items; ++q) {
    const long long s = s0 + q;
    if (s < nseg) run = xf_add(run, xf_from_u64(__ldcg(&seg[s].F), (long long)__ldcg(&seg[s].E) - kBS));
  }
  const xf incl = warp_incl_scan_v(run, lane);
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const xf wv = lane < kRThreads / 32 ? s_w[lane] : lb_zero<xf>();
    const xf wi = warp_incl_scan_v(wv, lane);
    xf we = shfl_up_v(wi, 1);
    if (lane == 0) we = lb_zero<xf>();
    if (lane < kRThreads / 32) s_w[lane] = xf_add(s_base, we);
  }
  __syncthreads();
  xf le = shfl_up_v(incl, 1);
  if (lane == 0) le = lb_zero<xf>();
  xf P = xf_add(s_w[warp], le);
#pragma unroll 1
  for (int q = 0; q < items; ++q) {
    const long long s = s0 + q;
    if (s >= nseg) break;
    write_seg_prefix(seg, idx, s, P);
    P = xf_add(P, xf_from_u64(__ldcg(&seg[s].F), (long long)__ldcg(&seg[s].E) - kBS));
    if (s == nseg - 1) write_consts(consts, P, with_z, need_invS, status);
  }
}

template <int kBS>
__global__ void __launch_bounds__(kPThreads) k_seg_prefix(long long nseg, SegRec* __restrict__ seg, SegIndex idx,
                                                         TileDesc<xf>* desc, unsigned* ctr, PathConsts* consts,
                                                         bool with_z, bool need_invS, int* status, int spin_limit,
                                                         bool withhold_first) {
  __shared__ xf s_wsum[kPThreads / 32];
  __shared__ xf s_woff[kPThreads / 32];
  __shared__ unsigned s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s = tile * kPTile + threadIdx.x;
  const xf v = (s < nseg) ? xf_from_u64(__ldcg(&seg[s].F), (long long)__ldcg(&seg[s].E) - kBS) : lb_zero<xf>();
  const xf incl = warp_incl_scan_v(v, lane);
  xf lane_off = shfl_up_v(incl, 1);
  if (lane == 0) lane_off = lb_zero<xf>();
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const xf wv = lane < kPThreads / 32 ? s_wsum[lane] : lb_zero<xf>();
    const xf wi = warp_incl_scan_v(wv, lane);
    const xf agg = shfl_v(wi, kPThreads / 32 - 1);
    xf excl = lb_zero<xf>();
    if (tile == 0) {
      if (lane == 0 && !withhold_first) lb_publish(desc, 0, agg, true);
    } else {
      if (lane == 0) lb_publish(desc, tile, agg, false);
      excl = lb_exclusive(desc, tile, lane, spin_limit, status);
      if (lane == 0) lb_publish_inc(desc, tile, xf_add(excl, agg));
    }
    xf wex = shfl_up_v(wi, 1);
    if (lane == 0) wex = lb_zero<xf>();
    if (lane < kPThreads / 32) s_woff[lane] = xf_add(excl, wex);
  }
  __syncthreads();
  if (s >= nseg) return;
  const xf P = xf_add(s_woff[warp], lane_off);
  write_seg_prefix(seg, idx, s, P);
  if (s == nseg - 1) write_consts(consts, xf_add(P, v), with_z, need_invS, status);
}

// ---- write: W_j ------------------------------------------------------------
// W_j = X_j / S with X_j = P_s + F_j * unit_s: per segment A = P_s/S and
// B = unit_s/S (128-bit mantissas), per element W_j = A + F_j * B rounded to
// binary64 by integer operations; clamped to the next segment's start so that
// W is non-decreasing, and the last element of the last segment is exactly 1.
// Head segments use exact per-element prefixes instead of the segment grid.
template <typename T, bool kVec>
__global__ void __launch_bounds__(256) k_w_write(const T* __restrict__ w, long long M, long long nseg,
                                                 const SegRec* __restrict__ seg, const PathConsts* __restrict__ consts,
                                                 double* __restrict__ W) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  constexpr int kBS = Tr::kBias + Tr::kShift;
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const xf invS = ld_xf(consts->invS);
  for (long long s = gw; s < nseg; s += nw) {
    const SegRec r = seg[s];
    const xf P = seg_P_xf(r);
    const xf A = xf_mul(P, invS);
    const xf B = xf_mul(xf_from_u64(1, r.E - kBS), invS);
    const long long an_bits =
        (s + 1 < nseg) ? (long long)xf_to_f64_bits(xf_mul(seg_P_xf(seg[s + 1]), invS)) : 0x3FF0000000000000LL;
    const bool head = sizeof(T) == 8 && head_segment(P, r.E, kBS);
    const long long base = s * kSeg;
    Bits bits[kSegV];
    load_seg_blocked<T, kVec>(w, base, M, lane, bits);
    if (head) {
      xf run = lb_zero<xf>();
#pragma unroll
      for (int i = 0; i < kSegV; ++i)
        if (Tr::valid_top(bits[i])) run = xf_add(run, xf_from_f64_bits((uint64_t)bits[i]));
      const xf incl = warp_incl_scan_v(run, lane);
      xf x = xf_add(P, shfl_up_v(incl, 1));
      if (lane == 0) x = P;
#pragma unroll
      for (int i = 0; i < kSegV; ++i) {
        if (Tr::valid_top(bits[i])) x = xf_add(x, xf_from_f64_bits((uint64_t)bits[i]));
        const long long j = base + (long long)lane * kSegV + i;
        if (j < M) {
          long long wb = (long long)xf_to_f64_bits(xf_mul(x, invS));
          if (wb > an_bits || j == base + r.len - 1) wb = an_bits;
          W[j] = __longlong_as_double(wb);
        }
      }
      continue;
    }
    uint64_t f[kSegV];
    uint64_t run = 0;
#pragma unroll
    for (int i = 0; i < kSegV; ++i) {
      run += Tr::fixed(bits[i], (uint32_t)r.E);
      f[i] = run;
    }
    const uint64_t off = warp_incl_scan_u64(run, lane) - run;
#pragma unroll
    for (int i = 0; i < kSegV; ++i) {
      const long long j = base + (long long)lane * kSegV + i;
      if (j < M) {
        long long wb = (long long)xf_to_f64_bits(xf_add(A, xf_mul_u64(B, off + f[i])));
        if (wb > an_bits || j == base + r.len - 1) wb = an_bits;
        W[j] = __longlong_as_double(wb);
      }
    }
  }
}

// ---- launchers -------------------------------------------------------------
template <typename T, bool kVec>
static cudaError_t reduce_t(const void* w, long long M, SegRec* seg, void* tagg, int* status, cudaStream_t st) {
  const long long nseg = (M + kSeg - 1) / kSeg;
  const long long blocks = (nseg + kWWarps - 1) / kWWarps;
  k_w_reduce<T, kVec><<<(unsigned)blocks, kWThreads, 0, st>>>((const T*)w, M, nseg, seg, (xf*)tagg, status);
  return cudaGetLastError();
}

cudaError_t launch_w_reduce(bool f32, bool vec, const void* w, long long M, SegRec* seg, void* tagg, int* status,
                            cudaStream_t st) {
  if (f32) return vec ? reduce_t<float, true>(w, M, seg, tagg, status, st)
                      : reduce_t<float, false>(w, M, seg, tagg, status, st);
  return vec ? reduce_t<double, true>(w, M, seg, tagg, status, st) : reduce_t<double, false>(w, M, seg, tagg, status, st);
}

cudaError_t launch_seg_prefix(bool f32, long long M, SegRec* seg, const void* tagg, const SegIndex& idx, void* desc,
                              unsigned* ctr, PathConsts* consts, bool with_z, bool need_invS, int* status,
                              int spin_limit, bool withhold_first, cudaStream_t st) {
  constexpr int kBS64 = FixedTraits<double>::kBias + FixedTraits<double>::kShift;
  constexpr int kBS32 = FixedTraits<float>::kBias + FixedTraits<float>::kShift;
  const long long nseg = (M + kSeg - 1) / kSeg;
  // smallest power-of-two run per thread that keeps the grid within kRedMaxBlocks
  int items = 1;
  while (items < kRedMaxItems && (nseg + (long long)kRThreads * items - 1) / ((long long)kRThreads * items) > kRedMaxBlocks)
    items *= 2;
  const long long rblocks = (nseg + (long long)kRThreads * items - 1) / ((long long)kRThreads * items);
  if (rblocks <= kRedMaxBlocks && !withhold_first) {
    if (f32)
      k_seg_prefix_red<kBS32><<<(unsigned)rblocks, kRThreads, 0, st>>>(nseg, items, seg, (const xf*)tagg, idx, consts,
                                                                       with_z, need_invS, status);
    else
      k_seg_prefix_red<kBS64><<<(unsigned)rblocks, kRThreads, 0, st>>>(nseg, items, seg, (const xf*)tagg, idx, consts,
                                                                       with_z, need_invS, status);
    return cudaGetLastError();
  }
  // very large M (or the look-back test hook): blocks of 256 segments chained
  // by decoupled look-back
  const long long tiles = (nseg + kPTile - 1) / kPTile;
  if (f32)
    k_seg_prefix<kBS32><<<(unsigned)tiles, kPThreads, 0, st>>>(nseg, seg, idx, (TileDesc<xf>*)desc, ctr, consts,
                                                               with_z, need_invS, status, spin_limit, withhold_first);
  else
    k_seg_prefix<kBS64><<<(unsigned)tiles, kPThreads, 0, st>>>(nseg, seg, idx, (TileDesc<xf>*)desc, ctr, consts,
                                                               with_z, need_invS, status, spin_limit, withhold_first);
  return cudaGetLastError();
}

template <typename T, bool kVec>
static cudaError_t write_t(const void* w, long long M, const SegRec* seg, const PathConsts* consts, double* W,
                           cudaStream_t st) {
  const long long nseg = (M + kSeg - 1) / kSeg;
  long long blocks = (nseg + 7) / 8;
  const long long cap = (long long)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_w_write<T, kVec><<<(unsigned)blocks, 256, 0, st>>>((const T*)w, M, nseg, seg, consts, W);
  return cudaGetLastError();
}

cudaError_t launch_w_write(bool f32, bool vec, const void* w, long long M, const SegRec* seg,
                           const PathConsts* consts, double* W, cudaStream_t st) {
  if (f32) return vec ? write_t<float, true>(w, M, seg, consts, W, st) : write_t<float, false>(w, M, seg, consts, W, st);
  return vec ? write_t<double, true>(w, M, seg, consts, W, st) : write_t<double, false>(w, M, seg, consts, W, st);
}

}  // namespace gbr
