// The map from weights (Eq. 2 through the segment records and prefixes of
// the weights pass): device code shared by the standalone map kernel and the
// fused single-instance kernel.
#pragma once
#include "seg_common.cuh"

namespace gbr {

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

constexpr int kMapWarps = 8;       // warps per block of the map from weights
constexpr int kLeafCount = 4;      // a segment with at most this many samples of a round is counted, not searched
constexpr int kMapTopMax = 6144;   // index entries staged in shared memory (48 KB)

// Per warp, U is processed in rounds of 32 consecutive samples, one per lane:
// every lane computes its key; the round's first sample keeps the segment of
// the previous round or locates its own (index descent); when the round
// spans several segments, the lanes find theirs among the next 32 segment
// prefixes (staged in shared memory), or - when the round spans more than 32
// segments - each with a warp-wide index descent.  Lanes that share a
// segment are then resolved together from the segment's exact prefixes: a
// warp-wide count per sample for a few samples, else the prefixes are staged
// in shared memory and every lane binary-searches its own (the leaf choice of
// Algorithm 5: linear walk for small leaves, binary search for large ones).
struct MapCtx {
  const unsigned long long* s_top;  // level 1 of the index in shared memory (ntop entries)
  int ntop;
  unsigned long long* s_pref;       // kMapWarps x 512 staged prefixes
  u128* s_win;                      // kMapWarps x 32 segment prefixes
  xf c;                             // S / Z_{N+1} (grid units per spacing unit)
  u128 S;                           // total on the grid
  long long ge;                     // grid exponent
  int Emax;                         // largest segment exponent
};

// The segment a warp currently holds: its prefix bounds on the global grid,
// its record and its exact in-segment prefixes (registers, and staged in
// shared memory once a round needs the per-lane search).
struct SegCache {
  long long cur;
  bool staged;
  u128 Ps, Pn;
  int sh, len;
  bool head;
  unsigned long long F;
  uint64_t pref[kSegV];
};
__device__ __forceinline__ void seg_cache_init(SegCache& c) {
  c.cur = -1;
  c.staged = false;
  c.Ps = c.Pn = u128{0ULL, 0ULL};
  c.sh = c.len = 0;
  c.head = false;
  c.F = 0;
#pragma unroll
  for (int q = 0; q < kSegV; ++q) c.pref[q] = 0;
}
// Makes segment sc (whose exclusive prefix is Ps, weights b lane-major) the
// cached one.
template <typename T>
__device__ __forceinline__ void seg_cache_fill(SegCache& c, const typename FixedTraits<T>::Bits (&b)[kSegV],
                                               const SegRec* __restrict__ seg, long long sc, const u128& Ps, int Emax,
                                               int lane) {
  const unsigned long long F = __ldcg(&seg[sc].F);
  const int E = __ldcg(&seg[sc].E);
  c.len = __ldcg(&seg[sc].len);
  c.F = F;
  c.Ps = Ps;
  c.Pn = u128_add(Ps, grid_value(F, E, Emax));
  c.sh = E - Emax + kGridHead;
  const xf Px = xf_make(Ps.hi, Ps.lo, 0);
  c.head = sizeof(T) == 8 && (xf_zero(Px) || Px.e + kXfTop < (long long)c.sh + 50);
  seg_prefixes<T>(b, (uint32_t)E, lane, c.pref);
  c.cur = sc;
  c.staged = false;
}
template <typename T, bool kVec>
__device__ __forceinline__ void seg_cache_load(SegCache& c, const T* __restrict__ w, long long M,
                                               const SegRec* __restrict__ seg, long long sc, const u128& Ps,
                                               int Emax, int lane) {
  if (sc == c.cur) return;
  typename FixedTraits<T>::Bits b[kSegV];
  load_seg_blocked<T, kVec>(w, sc * kSeg, M, lane, b);
  seg_cache_fill<T>(c, b, seg, sc, Ps, Emax, lane);
}

// Asynchronous copy of the calling lane's 16 weights of a full segment into
// shared memory (16-byte pieces; the segment must start 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <typename T>
__device__ __forceinline__ void seg_prefetch(const T* __restrict__ w, long long sc, int lane,
                                             typename FixedTraits<T>::Bits* buf) {
  const char* src = reinterpret_cast<const char*>(w + sc * kSeg + (long long)lane * kSegV);
  char* dst = reinterpret_cast<char*>(buf + lane * kSegV);
#pragma unroll
  for (int q = 0; q < (int)(kSegV * sizeof(T) / 16); ++q) cp_async16(dst + 16 * q, src + 16 * q);
  cp_async_commit();
}

// Resolves the samples of the lanes in grp, all in the cached segment, and
// writes out[i] for them.
template <typename T, bool kVec>
__device__ __forceinline__ void seg_cache_resolve(SegCache& c, const T* __restrict__ w, long long M, unsigned grp,
                                                  const u128& key, long long i, long long ge,
                                                  unsigned long long* my_pref, int lane, int* __restrict__ out) {
  const long long sc = c.cur;
  const bool mine = (grp >> lane) & 1u;
  const u128 rem = (mine && u128_lt(c.Ps, key)) ? u128_sub(key, c.Ps) : u128{0ULL, 0ULL};
  int cnt = 0;
  // In a head segment a key less than 2^50 segment units past its start may
  // need exact per-element sums; any other key is decided by the
  // segment-grid prefixes to 2^-41 relative.
  bool small = false;
  if (c.head && mine) {
    const xf rx = xf_make(rem.hi, rem.lo, 0);
    small = xf_zero(rx) || rx.e + kXfTop < (long long)c.sh + 50;
  }
  // first element whose exact prefix reaches K = ceil(rem / unit_s)
  const unsigned long long K = ceil_units(rem, c.sh, c.F);
  const unsigned gn = grp;
  {
    const bool mn = (gn >> lane) & 1u;
    if (__popc(gn) <= kLeafCount) {
      unsigned gg = gn;
      while (gg) {
        const int jl = __ffs(gg) - 1;
        gg &= gg - 1;
        const unsigned long long Kj = __shfl_sync(0xFFFFFFFFu, K, jl);
        int cj = 0;
#pragma unroll
        for (int q = 0; q < kSegV; ++q) cj += c.pref[q] < Kj ? 1 : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) cj += __shfl_xor_sync(0xFFFFFFFFu, cj, o);
        if (lane == jl) cnt = cj;
      }
    } else {
      if (!c.staged) {
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kSegV; ++q) my_pref[lane * kSegV + q] = c.pref[q];
        c.staged = true;
      }
      __syncwarp();
      if (mn) {  // prefixes below K (non-decreasing)
        int lo = 0, hi = kSeg;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (my_pref[mid] < K) lo = mid + 1;
          else hi = mid;
        }
        cnt = lo;
      }
    }
  }
  if (__any_sync(0xFFFFFFFFu, small)) {
    // Every element is truncated by less than one unit on the segment grid,
    // so its exact prefix lies in [pref, pref + len): the grid count is the
    // exact count unless some grid prefix lies in [K - len, K), or K was
    // clamped at the segment total.  Only such keys take the exact sums.
    const long long len = c.len;
    bool amb = false;
    if (small) {
      if (K >= c.F) amb = true;
      else if ((long long)K <= len) amb = cnt > 0;
    }
    unsigned chk = __ballot_sync(0xFFFFFFFFu, small && K < c.F && (long long)K > len);
    int cnt2 = -1;
    while (chk) {
      const int jl = __ffs(chk) - 1;
      chk &= chk - 1;
      const unsigned long long K2 = __shfl_sync(0xFFFFFFFFu, K, jl) - (unsigned long long)len;
      int cj = 0;
#pragma unroll
      for (int q = 0; q < kSegV; ++q) cj += c.pref[q] < K2 ? 1 : 0;
#pragma unroll
      for (int o = 16; o; o >>= 1) cj += __shfl_xor_sync(0xFFFFFFFFu, cj, o);
      if (lane == jl) cnt2 = cj;
    }
    if (cnt2 >= 0) amb = cnt2 != cnt;
    unsigned gx = __ballot_sync(0xFFFFFFFFu, small && amb);
    while (gx) {
      const int jl = __ffs(gx) - 1;
      gx &= gx - 1;
      const u128 rj = shfl_v(rem, jl);
      const int cj = head_count<kVec>(w, sc * kSeg, M, xf_make(rj.hi, rj.lo, ge), lane);
      if (lane == jl) cnt = cj;
    }
  }
  if (mine) {
    const long long j = cnt < c.len ? cnt : c.len - 1;
    long long rr = sc * kSeg + j;
    if (rr > M - 1) rr = M - 1;
    out[i] = (int)rr;
  }
}
// Resolves one round: every valid lane has its segment s_me and that
// segment's exclusive prefix P_me; lanes sharing a segment are contiguous.
template <typename T, bool kVec>
__device__ __forceinline__ void resolve_round(SegCache& c, const T* __restrict__ w, long long M,
                                              const SegRec* __restrict__ seg, bool valid, long long s_me,
                                              const u128& P_me, const u128& key, long long i, const MapCtx& cx,
                                              unsigned long long* my_pref, int lane, int* __restrict__ out,
                                              typename FixedTraits<T>::Bits* my_buf = nullptr) {
  using Bits = typename FixedTraits<T>::Bits;
  unsigned pend = __ballot_sync(0xFFFFFFFFu, valid);
  long long pf = -1;  // segment whose weights are being copied to my_buf
  while (pend) {
    const int l0 = __ffs(pend) - 1;
    const long long sc = __shfl_sync(0xFFFFFFFFu, s_me, l0);
    const u128 Psc = shfl_v(P_me, l0);
    const unsigned grp = __ballot_sync(0xFFFFFFFFu, valid && s_me == sc) & pend;
    const unsigned rest = pend & ~grp;
    // the next distinct segment's weights travel while this one is resolved
    if (kVec && my_buf && rest && pf < 0) {
      const long long sn = __shfl_sync(0xFFFFFFFFu, s_me, __ffs(rest) - 1);
      if (sn != c.cur && (sn + 1) * kSeg <= M) {
        seg_prefetch<T>(w, sn, lane, my_buf);
        pf = sn;
      }
    }
    if (sc != c.cur) {
      if (sc == pf) {
        cp_async_wait_all();
        Bits b[kSegV];
#pragma unroll
        for (int q = 0; q < kSegV; ++q) b[q] = my_buf[lane * kSegV + q];
        pf = -1;
        seg_cache_fill<T>(c, b, seg, sc, Psc, cx.Emax, lane);
      } else {
        seg_cache_load<T, kVec>(c, w, M, seg, sc, Psc, cx.Emax, lane);
      }
    }
    seg_cache_resolve<T, kVec>(c, w, M, grp, key, i, cx.ge, my_pref, lane, out);
    pend = rest;
  }
  if (pf >= 0) cp_async_wait_all();  // nothing in flight when the buffer is next used
}

// Processes the sample groups g_first, g_first + g_stride, ... (G samples
// each) with the calling warp, locating segments through the global segment
// prefixes and their search index.
template <typename T, bool kVec>
__device__ __forceinline__ void map_groups(const T* __restrict__ w, long long M, const SegRec* __restrict__ seg,
                                           const SegPre* __restrict__ pre, const SegIndex& idx,
                                           const u128* __restrict__ Z, long long N, int G, const MapCtx& cx,
                                           long long g_first, long long g_stride, int* __restrict__ out) {
  const unsigned long long* s_top = cx.s_top;
  const int ntop = cx.ntop;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* my_pref = cx.s_pref + warp * kSeg;
  u128* my_win = cx.s_win + warp * 32;
  const long long nseg = idx.n;
  const u128 kInf = {~0ULL, ~0ULL};
  for (long long g = g_first; g * (long long)G < N; g += g_stride) {
    const long long i0 = g * (long long)G;
    const long long i1 = (i0 + G < N) ? i0 + G : N;
    SegCache c;
    seg_cache_init(c);
    for (long long r0 = i0; r0 < i1; r0 += 32) {
      const long long i = r0 + lane;
      const bool valid = i < i1;
      const int last = (int)((i1 - 1 - r0) < 31 ? (i1 - 1 - r0) : 31);
      u128 key = {0ULL, 0ULL};
      if (valid) key = map_key(cx.c, u128{__ldcg(&Z[i].lo), __ldcg(&Z[i].hi)});  // ceil(U_i * S) in grid units
      const u128 kf = shfl_v(key, 0), kl = shfl_v(key, last);
      // the first sample's segment: the last s with P_s < key
      long long sf = c.cur;
      u128 Pf = c.Ps, Pf1 = c.Pn;
      if (!(c.cur >= 0 && u128_lt(c.Ps, kf) && !u128_lt(c.Pn, kf))) {
        const unsigned long long kb = u128_key(kf);
        sf = ntop > 0 ? locate_seg_smem(pre, idx, s_top, ntop, kb, kf, lane) : locate_seg(pre, idx, kb, kf, lane);
        Pf = seg_pre(pre, sf);
        Pf1 = sf + 1 < nseg ? seg_pre(pre, sf + 1) : cx.S;
      }
      long long s_me = sf;
      u128 P_me = Pf;
      if (u128_lt(Pf1, kl)) {
        // the round spans several segments: try the next 32 prefixes
        const long long j = sf + 1 + lane;
        const u128 Pj = j < nseg ? seg_pre(pre, j) : kInf;
        my_win[lane] = Pj;
        __syncwarp();
        const u128 P32 = shfl_v(Pj, 31);
        if (!u128_lt(P32, kl)) {
          if (valid) {  // number of window prefixes below the key
            int lo = 0, hi = 32;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (u128_lt(my_win[mid], key)) lo = mid + 1;
              else hi = mid;
            }
            s_me = sf + lo;
            if (lo > 0) P_me = my_win[lo - 1];
          }
        } else {
          // sparse round: the first unresolved sample descends the index with
          // the warp; every later sample up to that segment's end shares it
          unsigned todo = __ballot_sync(0xFFFFFFFFu, valid && u128_lt(Pf1, key));
          while (todo) {
            const int jl = __ffs(todo) - 1;
            const u128 kj = shfl_v(key, jl);
            const unsigned long long kb = u128_key(kj);
            const long long sj =
                ntop > 0 ? locate_seg_smem(pre, idx, s_top, ntop, kb, kj, lane) : locate_seg(pre, idx, kb, kj, lane);
            const u128 Ps_j = seg_pre(pre, sj);
            const u128 Pe = sj + 1 < nseg ? seg_pre(pre, sj + 1) : cx.S;
            // (the last segment also takes keys above S, from rounding)
            const unsigned take =
                (__ballot_sync(0xFFFFFFFFu, !u128_lt(Pe, key) || sj == nseg - 1) & todo) | (1u << jl);
            if ((take >> lane) & 1u) {
              s_me = sj;
              P_me = Ps_j;
            }
            todo &= ~take;
          }
        }
        __syncwarp();
      }
      resolve_round<T, kVec>(c, w, M, seg, valid, s_me, P_me, key, i, cx, my_pref, lane, out);
    }
  }
}

}  // namespace gbr
