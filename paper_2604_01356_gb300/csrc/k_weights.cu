// Cumulative weights (Eq. 3 of arXiv 2604.01356): W_j = sum_{k<=j} w_k / S,
// S = sum_k w_k.  The paper only notes that W can be formed alongside the
// normalisation; this file is that step.
//
// GB300 form (two passes, no binary64 work per weight):
//  pass 1  one warp per 512-element segment reads its weights with 16-byte
//          loads, picks the segment's largest exponent E (one warp max) and
//          sums the weights EXACTLY as integers on the segment grid
//          2^(E - bias - shift).  Tiles of 8 segments chain their sums
//          (binary64 pairs) by decoupled look-back.  Output: one SegRec per
//          segment (exclusive prefix P, exact sum F, E) plus a search index
//          over P, and the total S.
//  write   (only when W itself is requested) one warp per segment re-reads
//          the weights, forms exact within-segment prefixes and writes
//          W_j = a_s + F_j * b_s with a_s = P_s/S, b_s = unit_s/S (one FMA per
//          element), clamped so that W is non-decreasing and W_M = 1.
#include "common.cuh"
#include "internal.h"

namespace gbr {

constexpr int kWThreads = 256;
constexpr int kWWarps = kWThreads / kWarp;
static_assert(kWWarps * kSeg == kWTile, "weights tile");

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

template <typename T, bool kVec>
__global__ void __launch_bounds__(kWThreads) k_w_pass1(const T* __restrict__ w, long long M, long long nseg,
                                                      SegRec* __restrict__ seg, SegIndex idx, TileDesc<dd>* desc,
                                                      unsigned* ctr, dd* total, int* status, int spin_limit,
                                                      bool withhold_first) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  __shared__ dd s_val[kWWarps];
  __shared__ unsigned s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(ctr, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s = tile * kWWarps + warp;
  const long long base = s * kSeg;

  Bits b[kSegV];
  load_seg_striped<T, kVec>(w, base, M, lane, b);
  int emax = 0;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < kSegV; ++i) {
    emax = max(emax, seg_expo<T>(b[i]));
    bad |= Tr::bad(b[i]);
  }
  emax = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)emax);
  const int E = emax > 1 ? emax : 1;
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) raise_status(status, ST_ENONFINITE);
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kSegV; ++i) sum += to_fixed<T>(b[i], E);
  sum = warp_sum_u64(sum);
  if (lane == 0) {
    dd v = {0.0, 0.0};
    if (s < nseg) {
      v = u64_scaled_dd(sum, E - Tr::kBias - Tr::kShift);
      seg[s].F = sum;
      seg[s].E = E;
      const long long rem = M - base;
      seg[s].len = (int)(rem < kSeg ? rem : kSeg);
    }
    s_val[warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
    const dd v = lane < kWWarps ? s_val[lane] : dd{0.0, 0.0};
    dd incl = v;
#pragma unroll
    for (int o = 1; o < kWWarps; o <<= 1) {
      const dd t = shfl_up_v(incl, o);
      if (lane >= o) incl = dd_add(t, incl);
    }
    const dd agg = shfl_v(incl, kWWarps - 1);
    dd excl = {0.0, 0.0};
    if (tile == 0) {
      if (lane == 0 && !withhold_first) lb_publish(desc, 0, agg, true);
    } else {
      if (lane == 0) lb_publish(desc, tile, agg, false);
      excl = lb_exclusive(desc, tile, lane, spin_limit, status);
      if (lane == 0) lb_publish_inc(desc, tile, dd_add(excl, agg));
    }
    dd exs = shfl_up_v(incl, 1);
    if (lane == 0) exs = dd{0.0, 0.0};
    const long long sl = tile * kWWarps + lane;
    if (lane < kWWarps && sl < nseg) {
      const dd P = (lane == 0) ? excl : dd_add(excl, exs);
      seg[sl].P_hi = P.hi;
      seg[sl].P_lo = P.lo;
      const unsigned long long key = (unsigned long long)__double_as_longlong(P.hi);
      for (int l = 0; l < idx.nlev; ++l) {
        const long long mask = (1LL << (5 * l)) - 1;
        if (sl & mask) break;
        idx.lvl[l][sl >> (5 * l)] = key;
      }
      if (sl == nseg - 1) {
        const dd S = dd_add(P, v);
        *total = S;
        if (S.hi == 0.0) raise_status(status, ST_EZEROSUM);
      }
    }
  }
}

// W_j = a_s + F_j b_s, with a_s = P_s/S, b_s = 2^(E - bias - shift)/S per
// segment; clamped to a_{s+1} (the next segment's start, 1 for the last) so
// that W is non-decreasing and the last element of the last segment is 1.
template <typename T, bool kVec>
__global__ void __launch_bounds__(256) k_w_write(const T* __restrict__ w, long long M, long long nseg,
                                                 const SegRec* __restrict__ seg, const dd* __restrict__ total,
                                                 double* __restrict__ W) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const dd S = *total;
  for (long long s = gw; s < nseg; s += nw) {
    const SegRec r = seg[s];
    double a = 0.0, b = 0.0, anext = 1.0;
    bool head = false;
    if (lane == 0) {
      a = dd_div(dd{r.P_hi, r.P_lo}, S).hi;
      b = ldexp2(1.0, r.E - Tr::kBias - Tr::kShift) / S.hi;
      if (s + 1 < nseg) anext = dd_div(dd{seg[s + 1].P_hi, seg[s + 1].P_lo}, S).hi;
      head = sizeof(T) == 8 && head_segment(r.P_hi, r.E, Tr::kBias + Tr::kShift);
    }
    a = __shfl_sync(0xFFFFFFFFu, a, 0);
    b = __shfl_sync(0xFFFFFFFFu, b, 0);
    anext = __shfl_sync(0xFFFFFFFFu, anext, 0);
    head = __shfl_sync(0xFFFFFFFFu, head, 0);
    const long long base = s * kSeg;
    const long long an_bits = __double_as_longlong(anext);
    Bits bits[kSegV];
    load_seg_blocked<T, kVec>(w, base, M, lane, bits);
    if (head) {
      // binary64-pair prefixes: W_j = (P_s + sum_{k<=j in segment} w_k) / S
      dd run = {0.0, 0.0};
      dd loc[kSegV];
#pragma unroll
      for (int i = 0; i < kSegV; ++i) {
        const double x = Tr::bad(bits[i]) ? 0.0 : __longlong_as_double((long long)bits[i]);
        run = dd_add_d(run, x);
        loc[i] = run;
      }
      dd off = warp_incl_scan_v(run, lane);
      off = dd_add(off, dd{-run.hi, -run.lo});
      off = dd_add(off, dd{r.P_hi, r.P_lo});
#pragma unroll
      for (int i = 0; i < kSegV; ++i) {
        const long long j = base + (long long)lane * kSegV + i;
        if (j < M) {
          long long wb = __double_as_longlong(dd_div(dd_add(off, loc[i]), S).hi);
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
      run += to_fixed<T>(bits[i], r.E);
      f[i] = run;
    }
    const uint64_t incl = warp_incl_scan_u64(run, lane);
    const uint64_t off = incl - run;
#pragma unroll
    for (int i = 0; i < kSegV; ++i) {
      const long long j = base + (long long)lane * kSegV + i;
      if (j < M) {
        long long wb = __double_as_longlong(__fma_rn(__ull2double_rn(off + f[i]), b, a));
        if (wb > an_bits || j == base + r.len - 1) wb = an_bits;
        W[j] = __longlong_as_double(wb);
      }
    }
  }
}

template <typename T, bool kVec>
static cudaError_t pass1_t(const void* w, long long M, SegRec* seg, const SegIndex& idx, void* desc, unsigned* ctr,
                           void* total, int* status, int spin_limit, bool wf, cudaStream_t st) {
  const long long nseg = (M + kSeg - 1) / kSeg;
  const long long tiles = (nseg + kWWarps - 1) / kWWarps;
  k_w_pass1<T, kVec><<<(unsigned)tiles, kWThreads, 0, st>>>((const T*)w, M, nseg, seg, idx, (TileDesc<dd>*)desc, ctr,
                                                           (dd*)total, status, spin_limit, wf);
  return cudaGetLastError();
}

cudaError_t launch_w_pass1(bool f32, bool vec, const void* w, long long M, SegRec* seg, const SegIndex& idx,
                           void* desc, unsigned* ctr, void* total, int* status, int spin_limit, bool wf,
                           cudaStream_t st) {
  if (f32) return vec ? pass1_t<float, true>(w, M, seg, idx, desc, ctr, total, status, spin_limit, wf, st)
                      : pass1_t<float, false>(w, M, seg, idx, desc, ctr, total, status, spin_limit, wf, st);
  return vec ? pass1_t<double, true>(w, M, seg, idx, desc, ctr, total, status, spin_limit, wf, st)
             : pass1_t<double, false>(w, M, seg, idx, desc, ctr, total, status, spin_limit, wf, st);
}

template <typename T, bool kVec>
static cudaError_t write_t(const void* w, long long M, const SegRec* seg, const void* total, double* W,
                           cudaStream_t st) {
  const long long nseg = (M + kSeg - 1) / kSeg;
  long long blocks = (nseg + 7) / 8;
  const long long cap = (long long)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_w_write<T, kVec><<<(unsigned)blocks, 256, 0, st>>>((const T*)w, M, nseg, seg, (const dd*)total, W);
  return cudaGetLastError();
}

cudaError_t launch_w_write(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const void* total,
                           double* W, int* status, cudaStream_t st) {
  (void)status;
  if (f32) return vec ? write_t<float, true>(w, M, seg, total, W, st) : write_t<float, false>(w, M, seg, total, W, st);
  return vec ? write_t<double, true>(w, M, seg, total, W, st) : write_t<double, false>(w, M, seg, total, W, st);
}

}  // namespace gbr
