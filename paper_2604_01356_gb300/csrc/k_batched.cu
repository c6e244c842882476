// Batched resampling: K independent instances (the many-filter setting that
// motivates the paper, Sec. I) in ONE persistent launch.
//
// Each CTA takes instances from an atomic work queue (instances ordered by
// M_k, largest first, so that the big ones do not end up in the tail) and
// runs the whole path for one instance by itself, with no inter-CTA
// communication:
//   A  segment sums   one warp per 512-weight segment, exact fixed-point sums
//                     (Eq. 3 at the segment level), kept in shared memory;
//   B  prefixes       the instance's segment sums on its global grid, scanned
//                     exactly as 128-bit integers (shared memory);
//   C  spacings       all N+1 spacings of Algorithm 1 (or of the strata
//                     points) once, scanned exactly into Z_i (shared memory)
//                     and Z_{N+1}; then key_i = ceil(Z_i S / Z_{N+1});
//   D  map            segment-major: warp w takes a contiguous range of
//                     segments and the samples whose keys fall in them (the
//                     keys are sorted: one ballot over the next 32 keys finds
//                     where a segment's samples end); each segment with samples is loaded
//                     once, the next one travelling meanwhile, and its samples
//                     are resolved from its exact prefixes - by a warp-wide
//                     count when few samples fall in it, else by per-lane
//                     binary search over the prefixes staged in shared memory
//                     (the leaf threshold).
// Every step uses the single-instance path's arithmetic (same segment sums,
// grid, spacings, keys and in-segment decisions), so the indices equal those
// of rs_resample_w on each instance bit for bit.
//
// Instances with more than kBMaxSeg segments or kBMaxN samples are not
// processed here (the host sends them through the single-instance path).
#include <cstddef>

#include "cluster.cuh"
#include "map_common.cuh"

// Phase timestamps (profiling builds only, -DGBR_PHASE_STAMPS): %globaltimer
// at the phase ends of the first instance each CTA takes, 8 slots per CTA,
// in a buffer set by rs_dbg_set_batch_stamps.
#ifdef GBR_PHASE_STAMPS
namespace gbr {
__device__ unsigned long long* g_bstamps = nullptr;
}
extern "C" int rs_dbg_set_batch_stamps(void* p) { return (int)cudaMemcpyToSymbol(gbr::g_bstamps, &p, sizeof(p)); }
#define GBR_BSTAMP(first, k)                                               \
  do {                                                                     \
    if ((first) && threadIdx.x == 0 && gbr::g_bstamps) {                   \
      unsigned long long t_;                                               \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));               \
      gbr::g_bstamps[blockIdx.x * 8 + (k)] = t_;                           \
    }                                                                      \
  } while (0)
#else
#define GBR_BSTAMP(first, k) \
  do {                       \
  } while (0)
#endif

namespace gbr {

namespace {

template <int kWarps>
struct BatchSmem {
  u128 pre[kBMaxSeg + 1];         // exclusive grid prefixes; pre[nseg] = S
  unsigned long long F[kBMaxSeg];  // segment sums on their own grids
  int E[kBMaxSeg];                 // segment exponents
  unsigned long long pref[kWarps][kSeg];  // staged in-segment prefixes (leaf search)
  u128 key[kBMaxN];                 // Z_i, then the keys ceil(Z_i S / Z_{N+1})
  u128 wsum[kWarps];
  xf c;
  int emax_w[kWarps];
  int item;
  LogTab tab;  // logarithm table of the spacings
};

// Exclusive block scan of one u128 per thread; also returns the total.
template <int kWarps>
__device__ __forceinline__ u128 block_excl_scan(u128 v, u128* wsum, u128& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u128 incl = warp_incl_scan_v(v, lane);
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  u128 off = {0ULL, 0ULL}, tot = {0ULL, 0ULL};
#pragma unroll
  for (int i = 0; i < kWarps; ++i) {
    const u128 t = wsum[i];
    if (i < warp) off = u128_add(off, t);
    tot = u128_add(tot, t);
  }
  __syncthreads();
  total = tot;
  return u128_add(off, u128_sub(incl, v));
}

// The striped layout (load_seg_striped) gives each lane runs of kRun
// consecutive weights: run j of lane l starts at element 32 kRun j + kRun l.
// From the lanes' run sums g (seg_sum_bits_groups), lane L returns the
// inclusive prefix of block L (elements 16 L .. 16 L + 15): the runs of one
// block sit in 16 / kRun neighbouring lanes of one row.
template <int kRun>
__device__ __forceinline__ unsigned long long striped_block_prefix(uint64_t (&g)[kSegV / kRun], int lane) {
  constexpr int kLanesPerBlock = 16 / kRun;
  constexpr int kBlocksPerRow = 32 / kLanesPerBlock;
  constexpr int kRows = kSegV / kRun;
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
#pragma unroll
    for (int o = 1; o < kLanesPerBlock; o <<= 1) g[j] += __shfl_xor_sync(0xFFFFFFFFu, g[j], o);
  }
  const int src = (lane % kBlocksPerRow) * kLanesPerBlock;
  uint64_t v = 0;
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const uint64_t t = __shfl_sync(0xFFFFFFFFu, g[j], src);
    if (lane / kBlocksPerRow == j) v = t;
  }
  return warp_incl_scan_u64(v, lane);
}

// Number of a segment's 512 exact prefixes below X, from its 32 inclusive
// lane prefixes lp (lane l: elements 16 l .. 16 l + 15, in shared memory) and
// the 16 weights of the one lane block where X is reached: the blocks before
// it lie entirely below X, those after it entirely at or above, and inside
// it the prefixes are rebuilt exactly.  Equals count_below over the full
// prefixes (512 when every prefix is below X).
template <typename T, bool kVec>
__device__ __forceinline__ int block_count(const unsigned long long* lp, const T* __restrict__ w, long long base,
                                           long long M, uint32_t E, unsigned long long X) {
  int lo = 0, hi = 32;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lp[mid] < X) lo = mid + 1;
    else hi = mid;
  }
  if (lo >= 32) return kSeg;
  typename FixedTraits<T>::Bits b[kSegV];
  load_seg_blocked<T, kVec>(w, base, M, lo, b);
  unsigned long long run = lo ? lp[lo - 1] : 0ULL;
  int c = 0;
#pragma unroll
  for (int q = 0; q < kSegV; ++q) {
    run += FixedTraits<T>::fixed(b[q], E);
    c += run < X ? 1 : 0;
  }
  return lo * kSegV + c;
}

// Number of the 512 non-decreasing entries p[0..511] below X: nine fixed
// halving steps and a last compare, no branch.
__device__ __forceinline__ int count_below(const unsigned long long* p, unsigned long long X) {
  static_assert(kSeg == 512, "nine steps");
  int pos = 0;
#pragma unroll
  for (int step = kSeg / 2; step > 0; step >>= 1) pos += p[pos + step - 1] < X ? step : 0;
  return pos + (p[pos] < X ? 1 : 0);
}

__device__ __noinline__ void compute_c(xf* dst, u128 S, u128 Ztot) {
  *dst = xf_mul(xf_make(S.hi, S.lo, 0), recip_total(Ztot));
}

}  // namespace

// T: the weight type (binary32 weights with binary32 draws, or binary64 with
// binary64 draws).  With w_off == nullptr the batch is the single instance
// (M0, N0); with queue == nullptr CTA b takes instance b only (no queue to
// clear); order == nullptr is the identity order.  Instance k draws from the
// Philox stream (seed, inst_base + k).
template <typename T, int kThreads>
__global__ void __launch_bounds__(kThreads) k_batched(const T* __restrict__ w, const long long* __restrict__ w_off,
                                                      const long long* __restrict__ r_off,
                                                      const int* __restrict__ order, int K, unsigned long long seed,
                                                      unsigned long long inst_base, long long M0, long long N0,
                                                      int leaf_T, int* __restrict__ out, unsigned* queue,
                                                      int* status, int scheme, const LogTab* __restrict__ tab,
                                                      unsigned long long* __restrict__ lpref) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int kWarps = kThreads / 32;
  constexpr int kChunk = kThreads * 4;  // draws per block per chunk (4 per thread)
  constexpr int kRun = 16 / (int)sizeof(T);  // consecutive weights a lane holds in the striped layout
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem<kWarps>& sm = *reinterpret_cast<BatchSmem<kWarps>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < 129; i += kThreads) {
    sm.tab.nlogc[i] = tab->nlogc[i];
    sm.tab.invc[i] = tab->invc[i];
  }
  bool first = true;
  int taken = 0;  // instances this CTA has taken (without a queue: one)
  GBR_BSTAMP(true, 0);
  while (true) {
    __syncthreads();  // the previous instance is done with shared memory
    if (queue) {
      if (tid == 0) sm.item = (int)atomicAdd(queue, 1u);
    } else if (tid == 0) {
      sm.item = taken ? K : (int)blockIdx.x;
    }
    ++taken;
    __syncthreads();
    const int item = sm.item;
    if (item >= K) break;
    const int k = order ? order[item] : item;
    const long long wb = w_off ? w_off[k] : 0;
    const long long Mk = w_off ? w_off[k + 1] - wb : M0;
    const long long rb = r_off ? r_off[k] : 0;
    const long long Nk = r_off ? r_off[k + 1] - rb : N0;
    if (Nk <= 0 || Mk <= 0) continue;
    const long long nseg = (Mk + kSeg - 1) / kSeg;
    if (nseg > kBMaxSeg || Nk > kBMaxN) continue;  // left to the single-instance path
    const unsigned long long inst = inst_base + (unsigned long long)k;
    const T* wk = w + wb;
    const bool vec = (reinterpret_cast<uintptr_t>(wk) & 15) == 0;
    int* outk = out + rb;

    GBR_BSTAMP(first, 1);
    // ---- A: exact segment sums, two segments in flight per warp --------------
    // Besides each segment's sum, the inclusive prefixes of its 32 blocks of
    // 16 consecutive weights (exact, on the segment grid) go to lpb for the
    // map; the striped (coalesced) loads give them through a few shuffles.
    unsigned long long* lpb = lpref + (long long)blockIdx.x * kBMaxSeg * 32;
    int em = 0;
    for (int s0 = warp; s0 < nseg; s0 += 2 * kWarps) {
      const int s1 = s0 + kWarps;
      Bits b0[kSegV], b1[kSegV];
      if (vec) {
        load_seg_striped<T, true>(wk, (long long)s0 * kSeg, Mk, lane, b0);
        if (s1 < nseg) load_seg_striped<T, true>(wk, (long long)s1 * kSeg, Mk, lane, b1);
      } else {
        load_seg_striped<T, false>(wk, (long long)s0 * kSeg, Mk, lane, b0);
        if (s1 < nseg) load_seg_striped<T, false>(wk, (long long)s1 * kSeg, Mk, lane, b1);
      }
      uint64_t F;
      uint32_t E;
      uint64_t g[kSegV / kRun];
      seg_sum_bits_groups<T, kRun>(b0, lane, status, F, E, g);
      lpb[(long long)s0 * 32 + lane] = striped_block_prefix<kRun>(g, lane);
      if (lane == 0) {
        sm.F[s0] = F;
        sm.E[s0] = (int)E;
      }
      em = max(em, (int)E);
      if (s1 < nseg) {
        seg_sum_bits_groups<T, kRun>(b1, lane, status, F, E, g);
        lpb[(long long)s1 * 32 + lane] = striped_block_prefix<kRun>(g, lane);
        if (lane == 0) {
          sm.F[s1] = F;
          sm.E[s1] = (int)E;
        }
        em = max(em, (int)E);
      }
    }
    if (lane == 0) sm.emax_w[warp] = em;
    __syncthreads();
    int Emax = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) Emax = max(Emax, sm.emax_w[i]);
    const long long ge = (long long)Emax - Tr::kBias - Tr::kShift - kGridHead;  // grid exponent

    GBR_BSTAMP(first, 2);
    // ---- B: grid prefixes (consecutive segments per thread) -----------------
    constexpr int kPer = (kBMaxSeg + kThreads - 1) / kThreads;
    u128 v[kPer];
    u128 run = {0ULL, 0ULL};
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int s = tid * kPer + q;
      v[q] = s < nseg ? grid_value(sm.F[s], sm.E[s], Emax) : u128{0ULL, 0ULL};
      run = u128_add(run, v[q]);
    }
    u128 S;
    u128 P = block_excl_scan<kWarps>(run, sm.wsum, S);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int s = tid * kPer + q;
      if (s < nseg) sm.pre[s] = P;
      P = u128_add(P, v[q]);
    }
    if (tid == 0) sm.pre[nseg] = S;
    if (u128_is_zero(S)) {
      if (tid == 0) raise_status(status, ST_EZEROSUM);
      for (long long i = tid; i < Nk; i += kThreads) outk[i] = 0;
      continue;
    }

    GBR_BSTAMP(first, 3);
    // ---- C: all N+1 spacings once, their exact prefixes Z_i kept -------------
    const long long ndraw = Nk + 1;
    u128 carry = {0ULL, 0ULL};
#pragma unroll 1
    for (long long d0 = 0; d0 < ndraw; d0 += kChunk) {
      const long long k0 = d0 + 4LL * tid;  // one Philox block per thread
      uint64_t wd[4];
      philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, seed, inst, wd);
      u128 f[4];
      block_spacings<F32>(scheme, k0, ndraw, seed, inst, wd, &sm.tab, f);
      u128 run = {0ULL, 0ULL}, inc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        run = u128_add(run, f[q]);
        inc[q] = run;
      }
      u128 ctot;
      const u128 off = u128_add(carry, block_excl_scan<kWarps>(run, sm.wsum, ctot));
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (k0 + q < Nk) sm.key[k0 + q] = u128_add(off, inc[q]);
      carry = u128_add(carry, ctot);
    }
    if (tid == 0) compute_c(&sm.c, S, carry);  // carry = Z_{N+1}
    __syncthreads();
    const xf c = sm.c;
    GBR_BSTAMP(first, 4);
    for (long long i = tid; i < Nk; i += kThreads) sm.key[i] = map_key(c, sm.key[i]);
    __syncthreads();

    // ---- D: the map, segment-major -------------------------------------------
    // Warp w takes segments [a, b); a sample belongs to segment s when
    // P_s < key <= P_{s+1} (the last segment also takes keys above S).  Each
    // segment with samples is loaded once (the next one travels meanwhile),
    // its exact prefixes are staged in shared memory and every sample of it
    // is resolved by a binary search over them.
    {
      const int sa = (int)(nseg * warp / kWarps), sb = (int)(nseg * (warp + 1) / kWarps);
      // first sample of segment sa: keys are sorted
      long long i = 0;
      {
        long long lo = 0, hi = Nk;
        const u128 Pa = sm.pre[sa];
        while (lo < hi) {
          const long long mid = (lo + hi) >> 1;
          if (!u128_lt(Pa, sm.key[mid])) lo = mid + 1;
          else hi = mid;
        }
        i = lo;
      }
      unsigned long long* sp = sm.pref[warp];
      Bits bn[kSegV];
      int pf = -1;
      // the lane prefixes of the next segment travel while one is resolved
      unsigned long long lp_next = sa < sb ? __ldcg(lpb + (long long)sa * 32 + lane) : 0ULL;
#pragma unroll 1
      for (int sc = sa; sc < sb && i < Nk; ++sc) {
        const unsigned long long lp_this = lp_next;
        if (sc + 1 < sb) lp_next = __ldcg(lpb + (long long)(sc + 1) * 32 + lane);
        const bool last = sc == (int)nseg - 1;
        const u128 Pn = sm.pre[sc + 1];
        // samples [i, ie) fall in segment sc: the first key above P_{sc+1}
        // among the next 32 (one ballot; keys are sorted), a binary search
        // beyond them only when more than 32 samples fall in the segment
        const long long jl = i + lane;
        u128 kl = {0ULL, 0ULL};  // key of sample i + lane, reused by the leaf
        if (jl < Nk) kl = sm.key[jl];
        long long ie = Nk;
        if (!last) {
          const unsigned above = __ballot_sync(0xFFFFFFFFu, jl >= Nk || u128_lt(Pn, kl));
          if (above) {
            ie = i + __ffs(above) - 1;
            if (ie > Nk) ie = Nk;
          } else {
            long long lo = i + 32, hi = Nk;
            while (lo < hi) {
              const long long mid = (lo + hi) >> 1;
              if (!u128_lt(Pn, sm.key[mid])) lo = mid + 1;
              else hi = mid;
            }
            ie = lo;
          }
        }
        if (ie == i) continue;
        const uint32_t E = (uint32_t)sm.E[sc];
        const unsigned long long Fs = sm.F[sc];
        const u128 Ps = sm.pre[sc];
        const int sh = (int)E - Emax + kGridHead;
        const long long rem_len = Mk - (long long)sc * kSeg;
        const int len = (int)(rem_len < kSeg ? rem_len : kSeg);
        // a head segment (binary64 weights): the prefix before it is too
        // small for the segment grid to decide every key exactly; a key that
        // lies within the grid's truncation of a prefix is decided by exact
        // per-element sums scaled to the key (as on the single-instance path)
        bool head = false;
        if (!F32) {
          const xf Px = xf_make(Ps.hi, Ps.lo, 0);
          head = xf_zero(Px) || Px.e + kXfTop < (long long)sh + 50;
        }
        if (ie - i <= leaf_T) {
          // few samples (the leaf threshold): each sample is decided from
          // the segment's 32 exact lane prefixes (phase A) and the 16
          // weights of the one lane block its target falls in, without
          // decoding the whole segment
          __syncwarp();
          sp[lane] = lp_this;
          __syncwarp();
#pragma unroll 1
          for (long long j0 = i; j0 < ie; j0 += 32) {
            const long long j = j0 + lane;
            const bool mine = j < ie;
            u128 rem = {0ULL, 0ULL};
            unsigned long long Kq = 1;
            int cnt = 0;
            if (mine) {
              const u128 key = j0 == i ? kl : sm.key[j];
              rem = u128_lt(Ps, key) ? u128_sub(key, Ps) : u128{0ULL, 0ULL};
              Kq = ceil_units(rem, sh, Fs);
              cnt = vec ? block_count<T, true>(sp, wk, (long long)sc * kSeg, Mk, E, Kq)
                        : block_count<T, false>(sp, wk, (long long)sc * kSeg, Mk, E, Kq);
            }
            if (head) {  // warp-uniform branch; the ambiguous keys one by one
              bool amb = false;
              if (mine) {
                const xf rx = xf_make(rem.hi, rem.lo, 0);
                if (xf_zero(rx) || rx.e + kXfTop < (long long)sh + 50) {
                  if (Kq >= Fs) amb = true;
                  else if ((long long)Kq <= len) amb = cnt > 0;
                  else
                    amb = (vec ? block_count<T, true>(sp, wk, (long long)sc * kSeg, Mk, E, Kq - (unsigned long long)len)
                               : block_count<T, false>(sp, wk, (long long)sc * kSeg, Mk, E,
                                                       Kq - (unsigned long long)len)) != cnt;
                }
              }
              unsigned gx = __ballot_sync(0xFFFFFFFFu, amb);
#pragma unroll 1
              while (gx) {
                const int jl = __ffs(gx) - 1;
                gx &= gx - 1;
                const u128 rj = shfl_v(rem, jl);
                const int cj = vec ? head_count<true>(reinterpret_cast<const double*>(wk), (long long)sc * kSeg, Mk,
                                                      xf_make(rj.hi, rj.lo, ge), lane)
                                   : head_count<false>(reinterpret_cast<const double*>(wk), (long long)sc * kSeg, Mk,
                                                       xf_make(rj.hi, rj.lo, ge), lane);
                if (lane == jl) cnt = cj;
              }
            }
            if (mine) {
              const int jj = cnt < len ? cnt : len - 1;
              long long idx = (long long)sc * kSeg + jj;
              if (idx > Mk - 1) idx = Mk - 1;
              outk[j] = (int)idx;
            }
          }
          __syncwarp();
        } else {
          // many samples: the whole segment's exact prefixes, staged in
          // shared memory, and a binary search over them per sample
          Bits b[kSegV];
          if (pf == sc) {
#pragma unroll
            for (int q = 0; q < kSegV; ++q) b[q] = bn[q];
          } else if (vec) {
            load_seg_blocked<T, true>(wk, (long long)sc * kSeg, Mk, lane, b);
          } else {
            load_seg_blocked<T, false>(wk, (long long)sc * kSeg, Mk, lane, b);
          }
          pf = -1;
          if (F32 && sc + 1 < sb) {  // the next segment's weights travel while this one is resolved
            if (vec) load_seg_blocked<T, true>(wk, (long long)(sc + 1) * kSeg, Mk, lane, bn);
            else load_seg_blocked<T, false>(wk, (long long)(sc + 1) * kSeg, Mk, lane, bn);
            pf = sc + 1;
          }
          uint64_t pref[kSegV];
          seg_prefixes<T>(b, E, lane, pref);
          // the binary-search leaf over prefixes staged in shared memory
          __syncwarp();
#pragma unroll
          for (int q = 0; q < kSegV; ++q) sp[lane * kSegV + q] = pref[q];
          __syncwarp();
#pragma unroll 1
          for (long long j0 = i; j0 < ie; j0 += 32) {
            const long long j = j0 + lane;
            const bool mine = j < ie;
            u128 rem = {0ULL, 0ULL};
            unsigned long long Kq = 1;
            int cnt = 0;
            if (mine) {
              const u128 key = j0 == i ? kl : sm.key[j];
              rem = u128_lt(Ps, key) ? u128_sub(key, Ps) : u128{0ULL, 0ULL};
              Kq = ceil_units(rem, sh, Fs);
              cnt = count_below(sp, Kq);
            }
            if (head) {  // warp-uniform branch; the ambiguous keys one by one
              bool amb = false;
              if (mine) {
                const xf rx = xf_make(rem.hi, rem.lo, 0);
                if (xf_zero(rx) || rx.e + kXfTop < (long long)sh + 50) {
                  if (Kq >= Fs) amb = true;
                  else if ((long long)Kq <= len) amb = cnt > 0;
                  else amb = count_below(sp, Kq - (unsigned long long)len) != cnt;
                }
              }
              unsigned gx = __ballot_sync(0xFFFFFFFFu, amb);
#pragma unroll 1
              while (gx) {
                const int jl = __ffs(gx) - 1;
                gx &= gx - 1;
                const u128 rj = shfl_v(rem, jl);
                const int cj = vec ? head_count<true>(reinterpret_cast<const double*>(wk), (long long)sc * kSeg, Mk,
                                                      xf_make(rj.hi, rj.lo, ge), lane)
                                   : head_count<false>(reinterpret_cast<const double*>(wk), (long long)sc * kSeg, Mk,
                                                       xf_make(rj.hi, rj.lo, ge), lane);
                if (lane == jl) cnt = cj;
              }
            }
            if (mine) {
              const int jj = cnt < len ? cnt : len - 1;
              long long idx = (long long)sc * kSeg + jj;
              if (idx > Mk - 1) idx = Mk - 1;
              outk[j] = (int)idx;
            }
          }
          __syncwarp();
        }
        i = ie;
      }
    }
    GBR_BSTAMP(first, 5);
    first = false;
  }
}

// ---- the whole path of a small instance on one CTA, weights in shared memory
// (at most 12,288 weights, N <= 2047).  Latency is what counts here, so the
// two independent chains overlap and nothing is done twice:
//   - the weights travel to shared memory by asynchronous copies while the
//     draws are made (all N + 1 in one tile over the 512 threads);
//   - then warp 15 computes 1 / Z_{N+1} while warps 0-14 take one segment
//     each: its exact sum (Eq. 3 at the segment level) and its exact
//     in-segment prefixes, written once to shared memory (in place of
//     binary64 weights);
//   - the grid prefixes, c, the keys, and the map: warp w takes samples
//     [N w / 16, N (w+1) / 16) in rounds of 32, finds each sample's segment
//     by a binary search over the grid prefixes (keys are sorted) and the
//     element by a binary search over that segment's staged prefixes, as the
//     persistent kernel's search leaf does; so the indices are identical.
template <typename T>
struct SmallSmem {
  static constexpr int kMaxSeg = kSmallMaxM / kSeg;
  u128 key[kSmallMaxN + 1];                    // Z_i, then the keys
  alignas(16) unsigned long long P[kSmallMaxM];  // binary64 weights, then every segment's exact prefixes
  alignas(16) uint32_t w32[sizeof(T) == 4 ? kSmallMaxM : 4];  // binary32 weights
  u128 pre[kMaxSeg + 1];
  unsigned long long F[kMaxSeg];
  int E[kMaxSeg];
  u128 wsum[kSmThreads / 32];
  alignas(16) u128 part;  // this CTA's spacing total, read by the other CTAs of a cluster (16-byte loads)
  xf c, invZ;
  int emax_w[kSmThreads / 32];
  LogTab tab;
};


static_assert(offsetof(SmallSmem<double>, part) % 16 == 0 && offsetof(SmallSmem<float>, part) % 16 == 0,
              "16-byte cluster loads of part");

// Shared-memory position of entry e of an array of 8-byte (kPer = 2) or
// 4-byte (kPer = 4) entries: 16-byte chunks are swizzled within each
// 128-byte row (chunk c at c ^ ((c >> 3) & 7)), so that lane-major 16-byte
// reads (lane l: entries 16 l ..) are free of bank conflicts.
__device__ __forceinline__ long long sm_chunk(long long c) { return c ^ ((c >> 3) & 7); }
template <int kPer>
__device__ __forceinline__ long long sm_word(long long e) {
  return sm_chunk(e / kPer) * kPer + e % kPer;
}
// count_below over the 512 staged prefixes of segment s (swizzled).
__device__ __forceinline__ int count_below_sw(const unsigned long long* P, long long s, unsigned long long X) {
  const long long base = s * kSeg;
  int pos = 0;
#pragma unroll
  for (int step = kSeg / 2; step > 0; step >>= 1) pos += P[sm_word<2>(base + pos + step - 1)] < X ? step : 0;
  return pos + (P[sm_word<2>(base + pos)] < X ? 1 : 0);
}

// kG > 1: a cluster of kG CTAs shares the instance.  CTA r makes the draws
// [k_a, k_b) (Philox blocks split evenly) and maps those samples; the kG
// spacing totals are exchanged once through distributed shared memory (the
// offset of this CTA's prefixes and Z_{N+1}); every CTA stages all the
// weights and decodes every segment itself, so nothing else crosses CTAs and
// the arithmetic is that of kG = 1.
template <typename T, int kG>
__global__ void __launch_bounds__(kSmThreads, 1) k_small(const T* __restrict__ w, long long M, long long N,
                                                         unsigned long long seed, unsigned long long inst,
                                                         int* __restrict__ out, int* status, int scheme,
                                                         const LogTab* __restrict__ tab) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int kWarps = kSmThreads / 32;
  constexpr int kPer = 16 / (int)sizeof(T);  // weights per 16-byte chunk
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallSmem<T>& sm = *reinterpret_cast<SmallSmem<T>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  GBR_BSTAMP(true, 7);
  Bits* ws = F32 ? reinterpret_cast<Bits*>(sm.w32) : reinterpret_cast<Bits*>(sm.P);  // staged weights

  // the weights: 16-byte asynchronous copies by warps 0-14 (warp 15 computes
  // 1 / Z_{N+1} while they take the segments), in flight during the draws
  constexpr int kSegThreads = kSmThreads - 32;
  const bool vec = (reinterpret_cast<uintptr_t>(w) & 15) == 0;
  const long long nchunk = vec ? M * (long long)sizeof(T) / 16 : 0;
  if (tid < kSegThreads) {
    for (long long q = tid; q < nchunk; q += kSegThreads)
      cp_async16(reinterpret_cast<char*>(ws) + 16 * sm_chunk(q), reinterpret_cast<const char*>(w) + 16 * q);
    cp_async_commit();
  }
  for (int i = tid; i < 129; i += kSmThreads) {
    sm.tab.nlogc[i] = tab->nlogc[i];
    sm.tab.invc[i] = tab->invc[i];
  }
  __syncthreads();
  GBR_BSTAMP(true, 0);

  // ---- Algorithm 1: this CTA's spacings in one tile, exact prefixes --------
  // Multinomial draws: two per thread when the CTA holds at most 1024 (one
  // Philox block serves two threads), else four (one block per thread).
  const long long ndraw = N + 1;
  const int rank = kG > 1 ? (int)cluster_rank() : 0;
  const long long nblk = (ndraw + 3) / 4;
  const long long ka = 4 * (nblk * rank / kG);
  const long long kb = rank == kG - 1 ? ndraw : 4 * (nblk * (rank + 1) / kG);
  const long long ns = (kb < N ? kb : N) - ka;  // this CTA's samples [ka, ka + ns)
  u128 zoff = {0ULL, 0ULL};                     // spacings of the CTAs before this one
  {
    const int dpt = (scheme == kSchemeMultinomial && kb - ka <= 2 * kSmThreads) ? 2 : 4;
    const long long k0 = ka + (long long)dpt * tid;
    uint64_t wd[4] = {0ULL, 0ULL, 0ULL, 0ULL};
    if (k0 < kb) philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, seed, inst, wd);
    u128 f[4];
    if (dpt == 2) {
      const int o = (int)(k0 & 3);  // 0 or 2
      f[0] = k0 < kb ? spacing_fixed<F32>(o ? wd[2] : wd[0], &sm.tab) : u128{0ULL, 0ULL};
      f[1] = k0 + 1 < kb ? spacing_fixed<F32>(o ? wd[3] : wd[1], &sm.tab) : u128{0ULL, 0ULL};
      f[2] = f[3] = u128{0ULL, 0ULL};
    } else {
      block_spacings<F32>(scheme, k0, ndraw, seed, inst, wd, &sm.tab, f);
      if (k0 >= kb) f[0] = f[1] = f[2] = f[3] = u128{0ULL, 0ULL};  // another CTA's draws
    }
    u128 run = {0ULL, 0ULL}, inc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      run = u128_add(run, f[q]);
      inc[q] = run;
    }
    // the block scan; wsum is not used again, so one barrier suffices
    const u128 incl = warp_incl_scan_v(run, lane);
    if (lane == 31) sm.wsum[warp] = incl;
    __syncthreads();
    u128 off = {0ULL, 0ULL}, tot = {0ULL, 0ULL};
#pragma unroll
    for (int j = 0; j < kWarps; ++j) {
      const u128 t = sm.wsum[j];
      if (j < warp) off = u128_add(off, t);
      tot = u128_add(tot, t);
    }
    off = u128_add(off, u128_sub(incl, run));
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < dpt && k0 + q < ka + ns) sm.key[k0 + q - ka] = u128_add(off, inc[q]);
    if (kG > 1) {
      // the CTAs' spacing totals: this CTA's offset and Z_{N+1}
      if (tid == 0) sm.part = tot;
      cluster_sync_all();
      tot = u128{0ULL, 0ULL};
#pragma unroll
      for (int r = 0; r < kG; ++r) {
        const u128 v = ld_cluster_u128(&sm.part, (unsigned)r);
        if (r < rank) zoff = u128_add(zoff, v);
        tot = u128_add(tot, v);
      }
    }
    // 1 / Z_{N+1} on warp 15 from here on, while warps 0-14 take the segments
    if (tid == kSegThreads) sm.invZ = recip_total(tot);
  }
  GBR_BSTAMP(true, 1);
  const int nseg = (int)((M + kSeg - 1) / kSeg);
  if (warp < kWarps - 1) {
    cp_async_wait_all();
    // what the 16-byte copies left (an unaligned start, a ragged end), and
    // +0 up to the end of the last segment
    for (long long e = nchunk * kPer + tid; e < (long long)nseg * kSeg; e += kSegThreads) {
      Bits v = (Bits)0;
      if (e < M) {
        if (F32) v = (Bits)__ldg(reinterpret_cast<const unsigned*>(w + e));
        else v = (Bits)__ldg(reinterpret_cast<const unsigned long long*>(w + e));
      }
      ws[sm_word<kPer>(e)] = v;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kSegThreads) : "memory");  // warps 0-14 only
  }
  GBR_BSTAMP(true, 2);

  // ---- segments (warps 0-14): exact sums and prefixes -----------------------
  {
    int em = 0;
    if (warp < kWarps - 1) {
#pragma unroll 1
      for (int s = warp; s < nseg; s += kWarps - 1) {
        Bits b[kSegV];  // lane-major: elements 16 lane .. 16 lane + 15
        const long long c0 = ((long long)s * kSeg + lane * kSegV) / kPer;
#pragma unroll
        for (int j = 0; j < kSegV / kPer; ++j) {
          const uint4 v = *reinterpret_cast<const uint4*>(ws + sm_chunk(c0 + j) * kPer);
          if (F32) {
            b[4 * j] = (Bits)v.x;
            b[4 * j + 1] = (Bits)v.y;
            b[4 * j + 2] = (Bits)v.z;
            b[4 * j + 3] = (Bits)v.w;
          } else {
            b[2 * j] = (Bits)(((unsigned long long)v.y << 32) | v.x);
            b[2 * j + 1] = (Bits)(((unsigned long long)v.w << 32) | v.z);
          }
        }
        uint64_t F;
        uint32_t E;
        seg_sum_bits<T>(b, lane, status, F, E);
        uint64_t pref[kSegV];
        seg_prefixes<T>(b, E, lane, pref);
        // the prefixes replace the segment's weights (each lane its own entries)
        const long long p0 = ((long long)s * kSeg + lane * kSegV) / 2;
#pragma unroll
        for (int j = 0; j < kSegV / 2; ++j)
          *reinterpret_cast<ulonglong2*>(sm.P + sm_chunk(p0 + j) * 2) = make_ulonglong2(pref[2 * j], pref[2 * j + 1]);
        if (lane == 0) {
          sm.F[s] = F;
          sm.E[s] = (int)E;
        }
        em = max(em, (int)E);
      }
    }
    if (lane == 0) sm.emax_w[warp] = em;
  }
  __syncthreads();
  GBR_BSTAMP(true, 3);
  int Emax = 0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) Emax = max(Emax, sm.emax_w[i]);
  const long long ge = (long long)Emax - Tr::kBias - Tr::kShift - kGridHead;  // grid exponent

  // ---- grid prefixes (one warp) and c = S / Z_{N+1} --------------------------
  static_assert(SmallSmem<T>::kMaxSeg <= 32, "one segment a lane");
  if (warp == 0) {
    const u128 v = lane < nseg ? grid_value(sm.F[lane], sm.E[lane], Emax) : u128{0ULL, 0ULL};
    const u128 incl = warp_incl_scan_v(v, lane);
    if (lane < nseg) sm.pre[lane] = u128_sub(incl, v);
    if (lane == 31) {
      sm.pre[nseg] = incl;  // S
      sm.c = u128_is_zero(incl) ? lb_zero<xf>() : xf_mul(xf_make(incl.hi, incl.lo, 0), sm.invZ);
    }
  }
  __syncthreads();
  GBR_BSTAMP(true, 4);
  if (u128_is_zero(sm.pre[nseg])) {
    if (tid == 0 && rank == 0) raise_status(status, ST_EZEROSUM);
    for (long long i = tid; i < ns; i += kSmThreads) out[ka + i] = 0;
    if (kG > 1) cluster_sync_all();  // no CTA leaves while another may read its shared memory
    return;
  }
  const xf c = sm.c;
  for (long long i = tid; i < ns; i += kSmThreads) sm.key[i] = map_key(c, u128_add(zoff, sm.key[i]));
  __syncthreads();
  GBR_BSTAMP(true, 5);

  // ---- the map (Eq. 2 by Algorithm 5's split argument) of this CTA's samples -
  const long long i0 = ns * warp / kWarps, i1 = ns * (warp + 1) / kWarps;
#pragma unroll 1
  for (long long r0 = i0; r0 < i1; r0 += 32) {
    const long long i = r0 + lane;
    const bool valid = i < i1;
    const u128 key = valid ? sm.key[i] : u128{0ULL, 0ULL};
    // the segment: how many of the prefixes P_1 .. P_{nseg-1} lie below the key
    int s_me = 0;
    if (valid) {
      int lo = 1, hi = nseg;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u128_lt(sm.pre[mid], key)) lo = mid + 1;
        else hi = mid;
      }
      s_me = lo - 1;
    }
    const u128 Ps = sm.pre[s_me];
    const uint32_t E = (uint32_t)sm.E[s_me];
    const unsigned long long Fs = sm.F[s_me];
    const int sh = (int)E - Emax + kGridHead;
    const long long rem_len = M - (long long)s_me * kSeg;
    const int len = (int)(rem_len < kSeg ? rem_len : kSeg);
    const u128 rem = u128_lt(Ps, key) ? u128_sub(key, Ps) : u128{0ULL, 0ULL};
    const unsigned long long Kq = ceil_units(rem, sh, Fs);
    int cnt = valid ? count_below_sw(sm.P, s_me, Kq) : 0;
    if (!F32) {
      // a head segment: the prefix before it is too small for the segment
      // grid to decide every key exactly; the ambiguous keys are decided by
      // exact per-element sums (as on every other path)
      bool amb = false;
      if (valid) {
        const xf Px = xf_make(Ps.hi, Ps.lo, 0);
        const xf rx = xf_make(rem.hi, rem.lo, 0);
        if ((xf_zero(Px) || Px.e + kXfTop < (long long)sh + 50) && (xf_zero(rx) || rx.e + kXfTop < (long long)sh + 50)) {
          if (Kq >= Fs) amb = true;
          else if ((long long)Kq <= len) amb = cnt > 0;
          else amb = count_below_sw(sm.P, s_me, Kq - (unsigned long long)len) != cnt;
        }
      }
      unsigned gx = __ballot_sync(0xFFFFFFFFu, amb);
#pragma unroll 1
      while (gx) {
        const int jl = __ffs(gx) - 1;
        gx &= gx - 1;
        const u128 rj = shfl_v(rem, jl);
        const long long sj = __shfl_sync(0xFFFFFFFFu, s_me, jl);
        const int cj = vec ? head_count<true>(reinterpret_cast<const double*>(w), sj * kSeg, M,
                                              xf_make(rj.hi, rj.lo, ge), lane)
                           : head_count<false>(reinterpret_cast<const double*>(w), sj * kSeg, M,
                                               xf_make(rj.hi, rj.lo, ge), lane);
        if (lane == jl) cnt = cj;
      }
    }
    if (valid) {
      const int jj = cnt < len ? cnt : len - 1;
      long long idx = (long long)s_me * kSeg + jj;
      if (idx > M - 1) idx = M - 1;
      out[ka + i] = (int)idx;
    }
  }
#ifdef GBR_PHASE_STAMPS
  __syncthreads();
  GBR_BSTAMP(true, 6);
#endif
  if (kG > 1) cluster_sync_all();  // no CTA leaves while another may read its shared memory
}

// CTAs of a batched launch: K without a queue, else every CTA the device
// holds at once (at most K).
template <typename T, int kThreads>
static cudaError_t batched_blocks(int K, bool queue, long long& blocks) {
  const size_t smem = sizeof(BatchSmem<kThreads / 32>);
  cudaError_t e = cudaFuncSetAttribute(k_batched<T, kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  blocks = K;
  if (queue) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<T, kThreads>, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    blocks = (long long)num_sms() * per_sm;
    if (blocks > K) blocks = K;
  }
  if (blocks < 1) blocks = 1;
  return cudaSuccess;
}

template <typename T, int kThreads>
static cudaError_t batched_t(const T* w, const long long* w_off, const long long* r_off, const int* order, int K,
                             unsigned long long seed, unsigned long long inst_base, long long M0, long long N0,
                             int leaf_T, int* out, unsigned* queue, int* status, cudaStream_t st, int scheme,
                             const LogTab* tab, unsigned long long* lpref) {
  long long blocks = 0;
  cudaError_t e = batched_blocks<T, kThreads>(K, queue != nullptr, blocks);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(BatchSmem<kThreads / 32>);
  k_batched<T, kThreads><<<(unsigned)blocks, kThreads, smem, st>>>(w, w_off, r_off, order, K, seed, inst_base, M0, N0,
                                                                    leaf_T, out, queue, status, scheme, tab, lpref);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t batched_dispatch(const T* w, const long long* w_off, const long long* r_off, const int* order, int K,
                                    unsigned long long seed, unsigned long long inst_base, long long M0, long long N0,
                                    int threads, int leaf_T, int* out, unsigned* queue, int* status, cudaStream_t st,
                                    int scheme, const LogTab* tab, unsigned long long* lpref) {
  switch (threads) {
    case 128:
      return batched_t<T, 128>(w, w_off, r_off, order, K, seed, inst_base, M0, N0, leaf_T, out, queue, status, st,
                               scheme, tab, lpref);
    case 512:
      return batched_t<T, 512>(w, w_off, r_off, order, K, seed, inst_base, M0, N0, leaf_T, out, queue, status, st,
                               scheme, tab, lpref);
    default:
      return batched_t<T, 256>(w, w_off, r_off, order, K, seed, inst_base, M0, N0, leaf_T, out, queue, status, st,
                               scheme, tab, lpref);
  }
}

size_t batched_scratch_bytes(bool f32, int threads, int K, bool queue) {
  long long blocks = 0;
  cudaError_t e;
  if (f32) {
    e = threads == 128 ? batched_blocks<float, 128>(K, queue, blocks)
        : threads == 512 ? batched_blocks<float, 512>(K, queue, blocks) : batched_blocks<float, 256>(K, queue, blocks);
  } else {
    e = threads == 128 ? batched_blocks<double, 128>(K, queue, blocks)
        : threads == 512 ? batched_blocks<double, 512>(K, queue, blocks) : batched_blocks<double, 256>(K, queue, blocks);
  }
  if (e != cudaSuccess) return 0;
  return (size_t)blocks * kBMaxSeg * 32 * sizeof(unsigned long long);
}

cudaError_t launch_batched(bool f32, const void* w, const long long* w_off, const long long* r_off, const int* order,
                           int K, unsigned long long seed, unsigned long long inst_base, long long M0, long long N0,
                           int threads, int leaf_T, int* out, unsigned* queue, int* status, cudaStream_t st, int scheme,
                           const LogTab* tab, unsigned long long* lpref) {
  if (K <= 0) return cudaSuccess;
  if (f32)
    return batched_dispatch<float>(static_cast<const float*>(w), w_off, r_off, order, K, seed, inst_base, M0, N0,
                                   threads, leaf_T, out, queue, status, st, scheme, tab, lpref);
  return batched_dispatch<double>(static_cast<const double*>(w), w_off, r_off, order, K, seed, inst_base, M0, N0,
                                  threads, leaf_T, out, queue, status, st, scheme, tab, lpref);
}


template <typename T, int kG>
static cudaError_t small_t(const T* w, long long M, long long N, unsigned long long seed, unsigned long long inst,
                           int* out, int* status, cudaStream_t st, int scheme, const LogTab* tab) {
  const size_t smem = sizeof(SmallSmem<T>);
  cudaError_t e = cudaFuncSetAttribute(k_small<T, kG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (kG == 1) {
    k_small<T, 1><<<1, kSmThreads, smem, st>>>(w, M, N, seed, inst, out, status, scheme, tab);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kG, 1, 1);
  cfg.blockDim = dim3(kSmThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kG;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_small<T, kG>, w, M, N, seed, inst, out, status, scheme, tab);
  if (e == cudaSuccess) return e;
  // a device that cannot place the cluster: the one-CTA form (same indices)
  (void)cudaGetLastError();
  return small_t<T, 1>(w, M, N, seed, inst, out, status, st, scheme, tab);
}

cudaError_t launch_small(bool f32, const void* w, long long M, long long N, unsigned long long seed,
                         unsigned long long inst, int* out, int* status, cudaStream_t st, int scheme, const LogTab* tab,
                         int cluster) {
  if (N <= 0 || M <= 0) return cudaSuccess;
  if (N > kSmallMaxN || M > kSmallMaxM) return cudaErrorInvalidValue;
  if (f32) {
    if (cluster == 4)
      return small_t<float, 4>(static_cast<const float*>(w), M, N, seed, inst, out, status, st, scheme, tab);
    return small_t<float, 1>(static_cast<const float*>(w), M, N, seed, inst, out, status, st, scheme, tab);
  }
  if (cluster == 4)
    return small_t<double, 4>(static_cast<const double*>(w), M, N, seed, inst, out, status, st, scheme, tab);
  return small_t<double, 1>(static_cast<const double*>(w), M, N, seed, inst, out, status, st, scheme, tab);
}

// ---- work order: instances by M_k descending (ties by index) ----------------
// One block bitonic-sorts (M_k, k) keys in shared memory when K <= kSortMax;
// larger batches keep the identity order.
__global__ void __launch_bounds__(1024) k_batched_order(const long long* __restrict__ w_off, int K, int n2,
                                                        int* __restrict__ order) {
  extern __shared__ unsigned long long keys[];
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    unsigned long long key = ~0ULL;  // padding sorts last
    if (i < K) {
      long long m = w_off[i + 1] - w_off[i];
      if (m < 0) m = 0;
      if (m > 0x7FFFFFFFLL) m = 0x7FFFFFFFLL;
      // ascending key order = M_k descending, then k ascending
      key = ((unsigned long long)(0x7FFFFFFFLL - m) << 32) | (unsigned)i;
    }
    keys[i] = key;
  }
  __syncthreads();
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const unsigned long long a = keys[i], b = keys[j];
          if ((a > b) == up) {
            keys[i] = b;
            keys[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < K; i += blockDim.x) order[i] = (int)(keys[i] & 0xFFFFFFFFu);
}

__global__ void k_iota(int K, int* __restrict__ order) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < K; i += (long long)gridDim.x * blockDim.x)
    order[i] = (int)i;
}

cudaError_t launch_batched_order(const long long* w_off, int K, int* order, cudaStream_t st) {
  if (K <= 0) return cudaSuccess;
  if (K <= kSortMax) {
    int n2 = 1;
    while (n2 < K) n2 <<= 1;
    const size_t smem = (size_t)n2 * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(k_batched_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_batched_order<<<1, 1024, smem, st>>>(w_off, K, n2, order);
  } else {
    long long blocks = (K + 255) / 256;
    const long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    k_iota<<<(unsigned)blocks, 256, 0, st>>>(K, order);
  }
  return cudaGetLastError();
}

}  // namespace gbr
