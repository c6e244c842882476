// Cumulative weights (Eq. 3 of arXiv 2604.01356): W_j = sum_{k<=j} w_k / S,
// S = sum_k w_k.  The paper only notes that W can be formed alongside the
// normalisation; this file is that step.
//
// GB300 form (no binary64 arithmetic per weight or per segment):
//  reduce   one warp per 512-element segment reads its weights with 16-byte
//           coalesced loads, takes the segment's largest exponent E (one warp
//           max) and sums the weights EXACTLY as integers on the segment grid
//           2^(E - bias - shift).  Pure streaming: no inter-block waits.  Each
//           block of 8 segments (a tile) also records its largest exponent.
//  prefix   every segment sum is moved onto one global grid (2^-41 of the
//           largest segment's unit) and scanned exactly as unsigned 128-bit
//           integers; blocks of 256 tiles chain by decoupled look-back.
//           Writes each segment's exclusive prefix, a search index over them
//           and the per-call constants (S, S / Z_{N+1}, and 1/S when W is
//           written).
//  write    (only when W itself is requested) one warp per segment re-reads
//           the weights and writes W_j = (P_s + F_j unit_s) / S rounded to
//           binary64 by integer operations, clamped so that W is
//           non-decreasing and W_M = 1.
#include "seg_common.cuh"

namespace gbr {

constexpr int kWThreads = 256;
constexpr int kWWarps = kWThreads / kWarp;
static_assert(kWWarps == kSegsPerTile, "a reduce block is one tile of segments");
static_assert(kSegsPerTile == 8, "tile size");

// ---- reduce: exact segment sums ------------------------------------------
// One warp per segment; each block of 8 warps also records the largest
// segment exponent it saw (for the global grid of the prefix pass).
template <typename T, bool kVec>
__global__ void __launch_bounds__(kWThreads, 4) k_w_reduce(const T* __restrict__ w, long long M, long long nseg,
                                                          SegRec* __restrict__ seg, int* __restrict__ emax_blk,
                                                          int* status) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  __shared__ int s_e[kWWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long s = ((long long)blockIdx.x * kWThreads + threadIdx.x) >> 5;
  uint32_t E = 0;
  if (s < nseg) {
    const long long base = s * kSeg;
    uint64_t sum;
    seg_sum<T, kVec>(w, base, M, lane, status, sum, E);
    if (lane == 0) {
      const long long rem = M - base;
      SegRec r;
      r.F = sum;
      r.E = (int)E;
      r.len = (int)(rem < kSeg ? rem : kSeg);
      seg[s] = r;
    }
  }
  if (lane == 0) s_e[warp] = (int)E;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
#pragma unroll
    for (int i = 0; i < kWWarps; ++i) m = max(m, s_e[i]);
    emax_blk[blockIdx.x] = m;
  }
}

// ---- prefix: segment prefixes on the global grid --------------------------
// The per-call constants, written by the thread that owns the last segment:
// S and the grid exponent, c = S * (1/Z_{N+1}) (integer product; the
// reciprocal comes from the spacing scan) and, only when W itself is written,
// 1/S (binary64-pair division, out of line).
__device__ __noinline__ void write_consts(PathConsts* consts, u128 S, long long ge, int Emax, bool with_z,
                                          bool need_invS, int* status) {
  consts->S[0] = S.lo;
  consts->S[1] = S.hi;
  consts->ge = ge;
  consts->Emax = Emax;
  if (u128_is_zero(S)) {
    raise_status(status, ST_EZEROSUM);
    st_xf(consts->invS, lb_zero<xf>());
    st_xf(consts->c, lb_zero<xf>());
    return;
  }
  const xf Sx = xf_make(S.hi, S.lo, 0);
  if (need_invS) st_xf(consts->invS, xf_div(xf_from_u64(1, 0), Sx));
  st_xf(consts->c, with_z ? xf_mul(Sx, ld_xf(consts->invZ)) : lb_zero<xf>());
}

// Blocks of 256 threads, one tile of 8 segments per thread: the block finds
// Emax from the reduce pass's per-block maxima (all loads issued up front),
// converts its segments to the grid, scans them exactly as 128-bit integers
// and chains blocks by decoupled look-back (exact, so the prefixes do not
// depend on timing).  With kXf (W is written) the block also scans the
// segment sums as xf values in a fixed order and stores the in-block exclusive
// prefixes and the block total; the writer combines them for the segments
// whose prefix is below the grid's resolution.
__device__ __forceinline__ void st_segx(SegX* p, const xf& v) {
  SegX r;
  r.lo = v.lo;
  r.hi = v.hi;
  r.e = v.e;
  r.pad = 0;
  *p = r;
}
__device__ __forceinline__ xf ld_segx(const SegX* p) {
  return {__ldcg(&p->lo), __ldcg(&p->hi), (long long)__ldcg((const unsigned long long*)&p->e)};
}

template <bool kXf>
__global__ void __launch_bounds__(kPrefixTilesPerBlock) k_seg_prefix(long long nseg, int kBS,
                                                                    const SegRec* __restrict__ seg,
                                                                    const int* __restrict__ emax_blk,
                                                                    SegPre* __restrict__ pre, SegX* __restrict__ xin,
                                                                    SegX* __restrict__ xagg, SegIndex idx,
                                                                    TileDesc<u128>* desc, unsigned* ctr,
                                                                    PathConsts* consts, bool with_z, bool need_invS,
                                                                    int* status, int spin_limit,
                                                                    bool withhold_first) {
  constexpr int kT = kPrefixTilesPerBlock;
  __shared__ u128 s_w[kT / 32];
  __shared__ xf s_x[kT / 32];
  __shared__ int s_emax[kT / 32];
  __shared__ unsigned s_blk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_blk = atomicAdd(ctr, 1u);
  const long long ntile = (nseg + kSegsPerTile - 1) / kSegsPerTile;
  // Emax over all reduce blocks (one per tile): 16-byte loads, 4 in flight
  int em = 0;
  const long long nq = (ntile + 3) / 4;
  const int4* e4 = reinterpret_cast<const int4*>(emax_blk);
#pragma unroll 1
  for (long long q0 = tid; q0 < nq; q0 += 4LL * kT) {
    int4 a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long q = q0 + (long long)u * kT;
      a[u] = q < nq ? __ldcg(e4 + q) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long b4 = (q0 + (long long)u * kT) * 4;  // ignore the padding past ntile
      em = max(em, b4 < ntile ? a[u].x : 0);
      em = max(em, b4 + 1 < ntile ? a[u].y : 0);
      em = max(em, b4 + 2 < ntile ? a[u].z : 0);
      em = max(em, b4 + 3 < ntile ? a[u].w : 0);
    }
  }
  em = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)em);
  if (lane == 0) s_emax[warp] = em;
  __syncthreads();
  int Emax = 0;
#pragma unroll
  for (int i = 0; i < kT / 32; ++i) Emax = max(Emax, s_emax[i]);
  const long long blk = s_blk;
  // this thread's tile
  const long long t = blk * kT + tid;
  u128 v[kSegsPerTile];
  u128 run = {0ULL, 0ULL};
  xf xrun = lb_zero<xf>();
#pragma unroll
  for (int q = 0; q < kSegsPerTile; ++q) {
    const long long sidx = t * kSegsPerTile + q;
    v[q] = u128{0ULL, 0ULL};
    if (sidx < nseg) {
      const SegRec r = seg[sidx];
      v[q] = grid_value(r.F, r.E, Emax);
      if (kXf) xrun = xf_add(xrun, xf_from_u64(r.F, (long long)r.E - kBS));
    }
    run = u128_add(run, v[q]);
  }
  const u128 incl = warp_incl_scan_v(run, lane);
  if (lane == 31) s_w[warp] = incl;
  xf xexcl = lb_zero<xf>();
  if (kXf) {
    const xf xi = warp_incl_scan_v(xrun, lane);
    xexcl = shfl_up_v(xi, 1);
    if (lane == 0) xexcl = lb_zero<xf>();
    if (lane == 31) s_x[warp] = xi;
  }
  __syncthreads();
  if (warp == 0) {
    const u128 wv = lane < kT / 32 ? s_w[lane] : u128{0ULL, 0ULL};
    const u128 wi = warp_incl_scan_v(wv, lane);
    const u128 agg = shfl_v(wi, kT / 32 - 1);
    u128 excl = {0ULL, 0ULL};
    if (blk == 0) {
      if (lane == 0 && !withhold_first) lb_publish(desc, 0, agg, true);
    } else {
      if (lane == 0) lb_publish(desc, blk, agg, false);
      excl = lb_exclusive(desc, blk, lane, spin_limit, status);
      if (lane == 0) lb_publish_inc(desc, blk, u128_add(excl, agg));
    }
    if (kXf) {
      const xf xv = lane < kT / 32 ? s_x[lane] : lb_zero<xf>();
      const xf xi = warp_incl_scan_v(xv, lane);
      xf xe = shfl_up_v(xi, 1);
      if (lane == 0) xe = lb_zero<xf>();
      if (lane == kT / 32 - 1) st_segx(xagg + blk, xi);
      __syncwarp();
      if (lane < kT / 32) s_x[lane] = xe;
    }
    if (lane < kT / 32) s_w[lane] = u128_add(excl, u128_sub(wi, wv));
  }
  __syncthreads();
  u128 P = u128_add(s_w[warp], u128_sub(incl, run));
  xf X = lb_zero<xf>();
  if (kXf) X = xf_add(s_x[warp], xexcl);
  const long long ge = (long long)Emax - kBS - kGridHead;
#pragma unroll
  for (int q = 0; q < kSegsPerTile; ++q) {
    const long long sidx = t * kSegsPerTile + q;
    if (sidx >= nseg) break;
    SegPre r;
    r.lo = P.lo;
    r.hi = P.hi;
    pre[sidx] = r;
    if (kXf) {
      st_segx(xin + sidx, X);
      const SegRec sr = seg[sidx];
      X = xf_add(X, xf_from_u64(sr.F, (long long)sr.E - kBS));
    }
    const unsigned long long key = u128_key(P);
#pragma unroll 1
    for (int l = 0; l < idx.nlev; ++l) {
      const long long mask = (1LL << (5 * l)) - 1;
      if (sidx & mask) break;
      idx.lvl[l][sidx >> (5 * l)] = key;
    }
    P = u128_add(P, v[q]);
  }
  if (t * kSegsPerTile <= nseg - 1 && nseg - 1 < (t + 1) * kSegsPerTile)
    write_consts(consts, P, ge, Emax, with_z, need_invS, status);
}

// ---- write: W_j ------------------------------------------------------------
// W_j = X_j / S with X_j = P_s + F_j * 2^sh in grid units (sh = E - Emax +
// kGridHead): per element an integer 128-bit value times the 128-bit-mantissa
// reciprocal of S, rounded to binary64 by integer operations; clamped to the
// next segment's start so that W is non-decreasing and W_M = 1.  Head segments
// (prefix below 2^50 segment units) use exact per-element sums instead.
__device__ __forceinline__ u128 grid_shift(uint64_t f, int sh) {
  uint64_t hi = 0, lo = f;
  if (sh >= 0) shl128(hi, lo, sh);
  else shr128(hi, lo, -sh);
  return u128{lo, hi};
}

// Exact (xf) prefix of segment s: the block totals before its prefix-scan
// block, lane-strided then reduced by a butterfly (the same value on every
// lane, independent of timing), plus its in-block exclusive prefix.
__device__ xf exact_prefix(const SegX* __restrict__ xin, const SegX* __restrict__ xagg, long long s, int lane) {
  const long long b = s / ((long long)kPrefixTilesPerBlock * kSegsPerTile);
  xf acc = lb_zero<xf>();
  for (long long t = lane; t < b; t += 32) acc = xf_add(acc, ld_segx(xagg + t));
#pragma unroll
  for (int o = 16; o; o >>= 1) acc = xf_add(acc, shfl_v(acc, lane ^ o));
  return xf_add(acc, ld_segx(xin + s));
}
// A binary64 segment is written from exact prefixes when the grid cannot give
// its elements 2^-53 relative accuracy: its prefix is below 2^82 grid units
// (the grid's absolute error is at most one unit per segment, < 2^22 units) or
// below 2^50 units of its own segment grid.
__device__ __forceinline__ bool write_head(const u128& P, int sh) {
  const xf Px = xf_make(P.hi, P.lo, 0);
  const long long lim = sh + 50 > 82 ? (long long)sh + 50 : 82;
  return xf_zero(Px) || Px.e + kXfTop < lim;
}

template <typename T, bool kVec>
__global__ void __launch_bounds__(256) k_w_write(const T* __restrict__ w, long long M, long long nseg,
                                                 const SegRec* __restrict__ seg, const SegPre* __restrict__ pre,
                                                 const SegX* __restrict__ xin, const SegX* __restrict__ xagg,
                                                 const PathConsts* __restrict__ consts, double* __restrict__ W) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const xf invS = ld_xf(consts->invS);      // 1 / S_grid
  const long long ge = consts->ge;
  const int Emax = (int)consts->Emax;
  xf invS_val = invS;                        // 1 / (S_grid 2^ge)
  invS_val.e -= ge;
  for (long long s = gw; s < nseg; s += nw) {
    const SegRec r = seg[s];
    const u128 P = u128{pre[s].lo, pre[s].hi};
    const int sh = r.E - Emax + kGridHead;
    const bool head = sizeof(T) == 8 && write_head(P, sh);
    // W at the next segment's start, computed as that segment computes it:
    // the clamp keeps W non-decreasing across the boundary and makes W_M = 1
    long long an_bits = 0x3FF0000000000000LL;
    if (s + 1 < nseg) {
      const u128 Pn = u128{pre[s + 1].lo, pre[s + 1].hi};
      if (sizeof(T) == 8 && write_head(Pn, seg[s + 1].E - Emax + kGridHead))
        an_bits = (long long)xf_to_f64_bits(xf_mul(exact_prefix(xin, xagg, s + 1, lane), invS_val));
      else
        an_bits = (long long)xf_to_f64_bits(xf_mul(xf_make(Pn.hi, Pn.lo, 0), invS));
    }
    const long long base = s * kSeg;
    Bits bits[kSegV];
    load_seg_blocked<T, kVec>(w, base, M, lane, bits);
    if (head) {
      const xf Pv = exact_prefix(xin, xagg, s, lane);
      xf run = lb_zero<xf>();
#pragma unroll
      for (int i = 0; i < kSegV; ++i)
        if (Tr::valid_top(bits[i])) run = xf_add(run, xf_from_f64_bits((uint64_t)bits[i]));
      const xf incl = warp_incl_scan_v(run, lane);
      xf x = xf_add(Pv, shfl_up_v(incl, 1));
      if (lane == 0) x = Pv;
#pragma unroll
      for (int i = 0; i < kSegV; ++i) {
        if (Tr::valid_top(bits[i])) x = xf_add(x, xf_from_f64_bits((uint64_t)bits[i]));
        const long long j = base + (long long)lane * kSegV + i;
        if (j < M) {
          long long wb = (long long)xf_to_f64_bits(xf_mul(x, invS_val));
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
        const u128 X = u128_add(P, grid_shift(off + f[i], sh));
        long long wb = (long long)xf_to_f64_bits(xf_mul(xf_make(X.hi, X.lo, 0), invS));
        if (wb > an_bits || j == base + r.len - 1) wb = an_bits;
        W[j] = __longlong_as_double(wb);
      }
    }
  }
}

// ---- launchers -------------------------------------------------------------
template <typename T, bool kVec>
static cudaError_t reduce_t(const void* w, long long M, SegRec* seg, int* emax_blk, int* status, cudaStream_t st) {
  const long long nseg = (M + kSeg - 1) / kSeg;
  const long long blocks = (nseg + kWWarps - 1) / kWWarps;
  k_w_reduce<T, kVec><<<(unsigned)blocks, kWThreads, 0, st>>>((const T*)w, M, nseg, seg, emax_blk, status);
  return cudaGetLastError();
}

cudaError_t launch_w_reduce(bool f32, bool vec, const void* w, long long M, SegRec* seg, int* emax_blk, int* status,
                            cudaStream_t st) {
  if (f32) return vec ? reduce_t<float, true>(w, M, seg, emax_blk, status, st)
                      : reduce_t<float, false>(w, M, seg, emax_blk, status, st);
  return vec ? reduce_t<double, true>(w, M, seg, emax_blk, status, st)
             : reduce_t<double, false>(w, M, seg, emax_blk, status, st);
}

cudaError_t launch_seg_prefix(bool f32, long long M, const SegRec* seg, const int* emax_blk, SegPre* pre,
                              SegX* xin, SegX* xagg, const SegIndex& idx, void* desc, unsigned* ctr,
                              PathConsts* consts, bool with_z, bool need_invS, int* status, int spin_limit,
                              bool withhold_first, cudaStream_t st) {
  const int kBS = f32 ? FixedTraits<float>::kBias + FixedTraits<float>::kShift
                      : FixedTraits<double>::kBias + FixedTraits<double>::kShift;
  const long long nseg = (M + kSeg - 1) / kSeg;
  const long long ntile = (nseg + kSegsPerTile - 1) / kSegsPerTile;
  const long long blocks = (ntile + kPrefixTilesPerBlock - 1) / kPrefixTilesPerBlock;
  if (xin && xagg)
    k_seg_prefix<true><<<(unsigned)blocks, kPrefixTilesPerBlock, 0, st>>>(
        nseg, kBS, seg, emax_blk, pre, xin, xagg, idx, (TileDesc<u128>*)desc, ctr, consts, with_z, need_invS, status,
        spin_limit, withhold_first);
  else
    k_seg_prefix<false><<<(unsigned)blocks, kPrefixTilesPerBlock, 0, st>>>(
        nseg, kBS, seg, emax_blk, pre, nullptr, nullptr, idx, (TileDesc<u128>*)desc, ctr, consts, with_z, need_invS,
        status, spin_limit, withhold_first);
  return cudaGetLastError();
}

template <typename T, bool kVec>
static cudaError_t write_t(const void* w, long long M, const SegRec* seg, const SegPre* pre, const SegX* xin,
                           const SegX* xagg, const PathConsts* consts, double* W, cudaStream_t st) {
  const long long nseg = (M + kSeg - 1) / kSeg;
  long long blocks = (nseg + 7) / 8;
  const long long cap = (long long)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_w_write<T, kVec><<<(unsigned)blocks, 256, 0, st>>>((const T*)w, M, nseg, seg, pre, xin, xagg, consts, W);
  return cudaGetLastError();
}
cudaError_t launch_w_write(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const SegPre* pre,
                           const SegX* xin, const SegX* xagg, const PathConsts* consts, double* W, cudaStream_t st) {
  if (f32) return vec ? write_t<float, true>(w, M, seg, pre, xin, xagg, consts, W, st)
                      : write_t<float, false>(w, M, seg, pre, xin, xagg, consts, W, st);
  return vec ? write_t<double, true>(w, M, seg, pre, xin, xagg, consts, W, st)
             : write_t<double, false>(w, M, seg, pre, xin, xagg, consts, W, st);
}

}  // namespace gbr
