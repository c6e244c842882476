// The whole single-instance path of rs_resample_w (Eq. 3, Algorithm 1 and
// the segmented map of Eq. 2) in ONE cooperative launch, one CTA per SM.
//
// Every CTA owns a contiguous, balanced range of the 512-weight segments and
// a contiguous range of the N+1 draws (and of the N samples):
//
//   phase 1  the CTA's draws: Philox, spacings -log v on the 2^-88 grid and
//            their exact inclusive prefixes (Algorithm 1), each warp over
//            the draws of the samples it maps later, plus the warps'
//            offsets; the CTA's segments: streamed into shared memory by bulk
//            async copies (TMA engine, a ring of stages completed on
//            mbarriers), exact segment sums (one warp per segment).
//   exchange 1  every CTA publishes its largest segment exponent and its
//            spacing total; every CTA reads all of them (tagged words,
//            bounded waits): Emax, Z_{N+1} and the CTA's own spacing offset
//            follow.
//   phase 2  the CTA's segment sums on the global grid (unit fixed by
//            Emax), exact prefixes relative to the CTA range, the CTA total.
//   exchange 2  every CTA publishes its total and reads all of them
//            (release and acquire fences around it: the range prefixes and
//            segment records of other CTAs are read next): the CTA prefixes
//            and S.
//   phase 3  the map of the CTA's own samples: key ceil(U_i S), the owner
//            CTA of the key by binary search over the CTA prefixes and a
//            coarse index in shared memory, the segment among 32 prefixes,
//            the element from the segment's exact prefixes.
//
// There is no grid barrier and no per-call clearing: exchange flags carry a
// per-call epoch kept in device memory (advanced by CTA 0 once every CTA has
// published its total), so CUDA-graph replays work unchanged.  Every wait is
// bounded; a wait that runs out latches RS_ETIMEOUT and the kernel finishes
// (results are then unspecified).  The arithmetic is that of the multi-kernel
// path (same segment sums, exact integer prefixes, keys and in-segment
// decisions), so the indices are identical to it.
#include "map_common.cuh"

// Phase timestamps (profiling builds only, -DGBR_PHASE_STAMPS): %globaltimer
// of thread 0 (or of lane 0 of warp 0 inside the map) at the phase ends of
// every CTA, 32 slots per CTA, in a buffer set by rs_dbg_set_stamps.
#ifdef GBR_PHASE_STAMPS
namespace gbr {
__device__ unsigned long long* g_stamps = nullptr;
}
extern "C" int rs_dbg_set_stamps(void* p) { return (int)cudaMemcpyToSymbol(gbr::g_stamps, &p, sizeof(p)); }
#define GBR_STAMP_IF(cond, k)                                              \
  do {                                                                     \
    if ((cond) && gbr::g_stamps) {                                         \
      unsigned long long t_;                                               \
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));               \
      gbr::g_stamps[blockIdx.x * 32 + (k)] = t_;                           \
    }                                                                      \
  } while (0)
#else
#define GBR_STAMP_IF(cond, k) \
  do {                        \
    (void)(cond);             \
  } while (0)
#endif
#define GBR_STAMP(k) GBR_STAMP_IF(threadIdx.x == 0, k)

namespace gbr {

namespace {

constexpr int kFThreads = 512;
constexpr int kFWarps = kFThreads / 32;
constexpr int kStages = 3;                 // TMA ring stages
constexpr int kStageBytes = 64 * 1024;     // 16 binary64 or 32 binary32 segments
static_assert(kStageBytes < (1 << 20), "an mbarrier phase counts fewer than 2^20 bytes");
constexpr int kCoarseMax = 1024;           // coarse-index entries in shared memory
constexpr int kTmaSpin = 1 << 20;          // safety bound of the copy-completion waits
constexpr unsigned kFull = 0xFFFFFFFFu;

struct FusedArgs {
  const void* w;
  long long M, nseg, nfull, N, ndraw;
  unsigned long long seed, inst;
  SegRec* seg;        // [nseg]
  SegPre* rel;        // [nseg] prefix of each segment relative to its CTA range
  SegPre* crel;       // [ncoarse] the same for every stride-th segment
  long long ncoarse;
  int lgstride;
  u128* Z;            // [N] inclusive spacing prefixes relative to the owning CTA's draws
  unsigned* xch;      // epoch word + exchange slots (kFusedXchBytes)
  int* status;
  int spin;
  bool withhold_first;
  const LogTab* tab;  // logarithm table of the spacings
  bool few;           // one warp makes the draws while fifteen stream
  int kBS;
  int* out;
  int scheme;         // uniforms: Algorithm 1, stratified or systematic points
};

// Exchange slots: a published value of up to 144 bits travels in three
// 64-bit words, each carrying the call's 16-bit tag in its low bits.  Aligned
// 64-bit accesses are single-copy atomic, so a reader that sees the tag in all
// three words has the whole value in one round trip, without a flag.
constexpr int kLocalSegs = 1024;  // segment records a CTA keeps in shared memory
constexpr int kXSlotWords = 16;   // one 128-byte line per slot
static_assert(kFusedMaxCtas * 2 * kXSlotWords * 8 + 256 <= kFusedXchBytes, "exchange area");
static_assert(kFusedMaxCtas <= kFThreads - 32, "the last warp reads no exchange slot");
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void xput(unsigned long long* slot, unsigned tag, u128 v, unsigned extra) {
  const unsigned long long p0 = v.lo & 0xFFFFFFFFFFFFULL;
  const unsigned long long p1 = (v.lo >> 48) | ((v.hi & 0xFFFFFFFFULL) << 16);
  const unsigned long long p2 = (v.hi >> 32) | ((unsigned long long)(extra & 0xFFFFu) << 32);
  st_relaxed_u64(slot, (p0 << 16) | tag);
  st_relaxed_u64(slot + 1, (p1 << 16) | tag);
  st_relaxed_u64(slot + 2, (p2 << 16) | tag);
}
// Waits (at most `spin` polls) until all three words carry the tag.
__device__ __forceinline__ bool xget(const unsigned long long* slot, unsigned tag, int spin, u128& v,
                                     unsigned& extra) {
  unsigned long long a0, a1, a2;
  int spins = 0;
  while (true) {
    a0 = ld_relaxed_u64(slot);
    a1 = ld_relaxed_u64(slot + 1);
    a2 = ld_relaxed_u64(slot + 2);
    if ((a0 & 0xFFFFu) == tag && (a1 & 0xFFFFu) == tag && (a2 & 0xFFFFu) == tag) break;
    if (++spins > spin) return false;
    // every CTA polls every slot: back off so that the slot's own store is
    // not queued behind the polls
    __nanosleep(128);
  }
  a0 >>= 16;
  a1 >>= 16;
  a2 >>= 16;
  v.lo = a0 | (a1 << 48);
  v.hi = (a1 >> 16) | ((a2 & 0xFFFFFFFFULL) << 32);
  extra = (unsigned)(a2 >> 32);
  return true;
}

// Release / acquire fence at GPU scope (lighter than the sequentially
// consistent __threadfence).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release_flag(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- mbarrier / bulk-copy helpers (CTA-local) ---------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Waits for the phase with the given parity to complete; false after `spin`
// unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, int spin) {
  const unsigned a = smem_u32(b);
  for (int i = 0; i < spin; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// Bulk copy global -> shared completing on an mbarrier; the weights stream
// through L2 with evict-first priority (they are read once), so the segment
// records, prefixes and code of the later phases stay cached.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                         unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// One spacing -log v on the 2^-88 grid, out of line (one copy for the four
// draws of a Philox block).
template <bool F32>
static __device__ __noinline__ u128 spacing_ool(uint64_t word, const LogTab* tab) {
  return spacing_fixed<F32>(word, tab);
}

// The exact segment sum of seg_sum_bits for a segment staged in shared memory
// (lane l's elements in the 16-byte pieces at 16 l + 512 q), in two passes
// over shared memory (largest exponent field, then the fixed-point sum) so
// that the segment is never held in registers; the rare segment with a sign
// bit or a non-finite weight takes the register path.  The sum is an exact
// integer sum, so the result is that of seg_sum_bits.
template <typename T>
__device__ __forceinline__ void seg_sum_smem(const unsigned char* src, int lane, int* status, uint64_t& F,
                                             uint32_t& E) {
  using Tr = FixedTraits<T>;
  using Bits = typename Tr::Bits;
  constexpr int kPer = 16 / (int)sizeof(T);  // elements per 16-byte piece
  uint32_t tmax = 0;
#pragma unroll
  for (int q = 0; q < kSegV / kPer; ++q) {
    const uint4 v = *reinterpret_cast<const uint4*>(src + 16 * lane + 512 * q);
    if (sizeof(T) == 4) tmax = max(tmax, max(max(v.x >> 23, v.y >> 23), max(v.z >> 23, v.w >> 23)));
    else tmax = max(tmax, max(v.y >> 20, v.w >> 20));  // sign and exponent fields
  }
  tmax = __reduce_max_sync(kFull, tmax);
  constexpr uint32_t kTopInf = sizeof(T) == 8 ? 0x7FFu : 0xFFu;
  if (tmax < kTopInf) {
    E = tmax > 1u ? tmax : 1u;
    uint64_t sum = 0;
#pragma unroll
    for (int q = 0; q < kSegV / kPer; ++q) {
      const uint4 v = *reinterpret_cast<const uint4*>(src + 16 * lane + 512 * q);
      if (sizeof(T) == 4) {
        sum += Tr::fixed((Bits)v.x, E) + Tr::fixed((Bits)v.y, E) + Tr::fixed((Bits)v.z, E) + Tr::fixed((Bits)v.w, E);
      } else {
        sum += fixed64_valid(((uint64_t)v.y << 32) | v.x, E) + fixed64_valid(((uint64_t)v.w << 32) | v.z, E);
      }
    }
    F = warp_sum_u64(sum);
  } else {
    Bits b[kSegV];
#pragma unroll
    for (int q = 0; q < kSegV / kPer; ++q) {
      const uint4 v = *reinterpret_cast<const uint4*>(src + 16 * lane + 512 * q);
      if (sizeof(T) == 4) {
        b[4 * q] = (Bits)v.x;
        b[4 * q + 1] = (Bits)v.y;
        b[4 * q + 2] = (Bits)v.z;
        b[4 * q + 3] = (Bits)v.w;
      } else {
        b[2 * q] = (Bits)(((uint64_t)v.y << 32) | v.x);
        b[2 * q + 1] = (Bits)(((uint64_t)v.w << 32) | v.z);
      }
    }
    seg_sum_bits<T>(b, lane, status, F, E);
  }
}

// The draws [g0, g1) of the stream by one warp (Algorithm 1's spacings, or
// the strata spacings): their exact inclusive prefixes relative to g0 are
// stored as Z[k] for k < N.  Returns the warp's total (every lane).
template <bool F32>
__device__ __forceinline__ u128 draw_range(const FusedArgs& a, long long g0, long long g1, const LogTab* tab,
                                           int lane) {
  u128 wrun = {0ULL, 0ULL};
  const long long base = g0 & ~3LL;
#pragma unroll 1
  for (long long t0 = base; t0 < g1; t0 += 128) {
    const long long k0 = t0 + 4LL * lane;
    u128 pre[4];
    u128 run = {0ULL, 0ULL};
    const bool mine = k0 < g1 && k0 + 3 >= g0;
    if (a.scheme == kSchemeMultinomial) {
      if (mine) {
        uint64_t words[4];
        philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, a.seed, a.inst, words);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const long long k = k0 + q;
          if (k >= g0 && k < g1) run = u128_add(run, spacing_ool<F32>(words[q], tab));
          pre[q] = run;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) pre[q] = run;
      }
    } else {
      // strata points: every lane of the warp takes part (neighbour words)
      uint64_t words[4];
      philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, a.seed, a.inst, words);
      u128 f[4];
      block_spacings<F32>(a.scheme, k0, a.ndraw, a.seed, a.inst, words, tab, f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long k = k0 + q;
        if (k >= g0 && k < g1) run = u128_add(run, f[q]);
        pre[q] = run;
      }
    }
    const u128 incl = warp_incl_scan_v(run, lane);
    const u128 excl = u128_add(wrun, u128_sub(incl, run));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long k = k0 + q;
      if (k >= g0 && k < g1 && k < a.N) a.Z[k] = u128_add(excl, pre[q]);
    }
    wrun = u128_add(wrun, shfl_v(incl, 31));
  }
  return wrun;
}

// Owner CTA of segment t under the balanced split floor(nseg c / B).
__device__ __forceinline__ int seg_owner(long long t, long long nseg, int B) {
  return (int)(((unsigned long long)(t + 1) * (unsigned)B - 1ULL) / (unsigned long long)nseg);
}

// Block-wide exclusive prefix of v (over lower thread indices) and total.
struct BlockScan {
  u128 excl, tot;
};
static __device__ __noinline__ BlockScan block_scan(u128 v, u128* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u128 incl = warp_incl_scan_v(v, lane);
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  u128 before = {0ULL, 0ULL}, t = {0ULL, 0ULL};
#pragma unroll
  for (int i = 0; i < kFWarps; ++i) {
    const u128 x = s_w[i];
    if (i < warp) before = u128_add(before, x);
    t = u128_add(t, x);
  }
  __syncthreads();  // s_w may be reused
  return BlockScan{u128_add(before, u128_sub(incl, v)), t};
}

// ---- the in-segment step of the map, kept small ----------------------------
// The map after the weights pass is latency-bound and runs once per call, so
// its code is fetched cold: every step below exists once (no duplicated
// paths), loops stay rolled, and the segment's exact prefixes are staged in
// shared memory (slot q*32 + lane holds the prefix of element 16 lane + q)
// and binary-searched.  Decisions are those of seg_cache_resolve.
struct LeanSeg {
  long long cur;
  u128 Ps, Pn;
  int sh, len;
  bool head;
  unsigned long long F;
};

__device__ __forceinline__ unsigned long long lean_pref(const unsigned long long* p, int j) {
  return p[(j & 15) * 32 + (j >> 4)];
}
// Number of elements whose exact prefix is below X (the prefixes are
// non-decreasing): nine fixed halving steps, no branch.
__device__ __forceinline__ int lean_count(const unsigned long long* p, unsigned long long X) {
  static_assert(kSeg == 512, "nine steps");
  int pos = 0;
#pragma unroll
  for (int step = kSeg / 2; step > 0; step >>= 1) pos += lean_pref(p, pos + step - 1) < X ? step : 0;
  return pos + (lean_pref(p, pos) < X ? 1 : 0);
}
template <bool kVec>
static __device__ __noinline__ int head_count_ool(const double* w, long long base, long long M, xf rem, int lane) {
  return head_count<kVec>(w, base, M, rem, lane);
}
template <bool kVec>
static __device__ __noinline__ int head_count_ool(const float*, long long, long long, xf, int) {
  return 0;
}

// Makes segment sc (weights b, lane-major; record F, E, len; exclusive
// prefix Ps) the warp's current one: exact in-segment prefixes to shared
// memory and the segment's bounds on the global grid.
template <typename T>
__device__ __forceinline__ void lean_fill(LeanSeg& c, const typename FixedTraits<T>::Bits (&b)[kSegV],
                                          unsigned long long F, int E, int len, long long sc, const u128& Ps,
                                          int Emax, unsigned long long* my_pref, int lane) {
  uint64_t pref[kSegV];
  seg_prefixes<T>(b, (uint32_t)E, lane, pref);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < kSegV; ++q) my_pref[q * 32 + lane] = pref[q];
  __syncwarp();
  c.cur = sc;
  c.F = F;
  c.len = len;
  c.Ps = Ps;
  c.Pn = u128_add(Ps, grid_value(F, E, Emax));
  c.sh = E - Emax + kGridHead;
  const xf Px = xf_make(Ps.hi, Ps.lo, 0);
  c.head = sizeof(T) == 8 && (xf_zero(Px) || Px.e + kXfTop < (long long)c.sh + 50);
}

// Resolves one round: every valid lane has its segment s_me and that
// segment's exclusive prefix P_me; lanes sharing a segment are contiguous.
// The next distinct segment's weights are copied to my_buf (asynchronously)
// while the current one is resolved.
template <typename T, bool kVec>
__device__ __forceinline__ void lean_round(LeanSeg& c, const T* __restrict__ w, long long M,
                                           const SegRec* __restrict__ seg, bool valid, long long s_me, const u128& P_me,
                                           const u128& key, long long i, int Emax, long long ge,
                                           unsigned long long* my_pref, typename FixedTraits<T>::Bits* my_buf, int lane,
                                           int* __restrict__ out) {
  using Bits = typename FixedTraits<T>::Bits;
  unsigned pend = __ballot_sync(0xFFFFFFFFu, valid);
  long long pf = -1;  // segment being copied to my_buf
  unsigned long long pfF = 0;
  int pfE = 0, pfL = 0;
#pragma unroll 1
  while (pend) {
    const int l0 = __ffs(pend) - 1;
    const long long sc = __shfl_sync(0xFFFFFFFFu, s_me, l0);
    const u128 Psc = shfl_v(P_me, l0);
    const unsigned grp = __ballot_sync(0xFFFFFFFFu, valid && s_me == sc) & pend;
    const unsigned rest = pend & ~grp;
    if (sc != c.cur) {
      Bits b[kSegV];
      unsigned long long F;
      int E, len;
      if (sc == pf) {
        cp_async_wait_all();
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kSegV; ++q) b[q] = my_buf[lane * kSegV + q];
        F = pfF;
        E = pfE;
        len = pfL;
        pf = -1;
        __syncwarp();  // my_buf is free again
      } else {
        F = __ldcg(&seg[sc].F);
        E = __ldcg(&seg[sc].E);
        len = __ldcg(&seg[sc].len);
        load_seg_blocked<T, kVec>(w, sc * kSeg, M, lane, b);
      }
      if (kVec && rest) {
        const long long sn = __shfl_sync(0xFFFFFFFFu, s_me, __ffs(rest) - 1);
        if ((sn + 1) * kSeg <= M) {
          seg_prefetch<T>(w, sn, lane, my_buf);
          pf = sn;
          pfF = __ldcg(&seg[sn].F);
          pfE = __ldcg(&seg[sn].E);
          pfL = __ldcg(&seg[sn].len);
        }
      }
      lean_fill<T>(c, b, F, E, len, sc, Psc, Emax, my_pref, lane);
    }
    // the element: first whose exact prefix reaches K = ceil(rem / unit_s)
    const bool mine = (grp >> lane) & 1u;
    const u128 rem = (mine && u128_lt(c.Ps, key)) ? u128_sub(key, c.Ps) : u128{0ULL, 0ULL};
    bool small = false;
    if (c.head && mine) {
      const xf rx = xf_make(rem.hi, rem.lo, 0);
      small = xf_zero(rx) || rx.e + kXfTop < (long long)c.sh + 50;
    }
    const unsigned long long K = ceil_units(rem, c.sh, c.F);
    int cnt = mine ? lean_count(my_pref, K) : 0;
    if (__any_sync(0xFFFFFFFFu, small)) {
      // head segment: the grid count is exact unless a grid prefix lies in
      // [K - len, K) or K was clamped at the segment total
      bool amb = false;
      if (small) {
        if (K >= c.F) amb = true;
        else if ((long long)K <= c.len) amb = cnt > 0;
        else amb = lean_count(my_pref, K - (unsigned long long)c.len) != cnt;
      }
      unsigned gx = __ballot_sync(0xFFFFFFFFu, small && amb);
#pragma unroll 1
      while (gx) {
        const int jl = __ffs(gx) - 1;
        gx &= gx - 1;
        const u128 rj = shfl_v(rem, jl);
        const int cj = head_count_ool<kVec>(w, sc * kSeg, M, xf_make(rj.hi, rj.lo, ge), lane);
        if (lane == jl) cnt = cj;
      }
    }
    if (mine) {
      const long long j = cnt < c.len ? cnt : c.len - 1;
      long long rr = sc * kSeg + j;
      if (rr > M - 1) rr = M - 1;
      out[i] = (int)rr;
    }
    pend = rest;
  }
  if (pf >= 0) cp_async_wait_all();  // nothing in flight when the buffer is next used
}

// The map of the CTA's own samples [i0, i1) by one warp, in rounds of 32:
// keys, the segment among the prefixes P_t = (CTA prefix of t's owner) + rel_t,
// located through the coarse index, then the in-segment decision.
template <typename T, bool kVec>
__device__ __forceinline__ void map_own(const T* __restrict__ w, long long M, const SegRec* __restrict__ seg,
                                        const SegPre* __restrict__ rel, long long nseg, const u128* __restrict__ Z,
                                        u128 zoff, u128 z_first, long long i0, long long i1, const MapCtx& cx,
                                        const u128* s_cp,
                                        const u128* s_coarse, long long ncoarse, int lgstride, int B,
                                        typename FixedTraits<T>::Bits* my_buf, int* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* my_pref = cx.s_pref + warp * kSeg;
  u128* my_win = cx.s_win + warp * 32;
  const u128 kInf = {~0ULL, ~0ULL};
  const long long stride = 1LL << lgstride;
  LeanSeg c;
  c.cur = -1;
  c.Ps = c.Pn = u128{0ULL, 0ULL};
  c.sh = c.len = 0;
  c.head = false;
  c.F = 0;
  u128 z_cur = z_first;
#pragma unroll 1
  for (long long r0 = i0; r0 < i1; r0 += 32) {
    const long long i = r0 + lane;
    const bool valid = i < i1;
    const bool w0 = threadIdx.x == 0 && r0 == i0;
    GBR_STAMP_IF(w0, 10);
    // the next round's spacing prefixes travel while this round is mapped
    u128 z_next = {0ULL, 0ULL};
    if (i + 32 < i1) z_next = u128{__ldcg(&Z[i + 32].lo), __ldcg(&Z[i + 32].hi)};
    u128 key = {0ULL, 0ULL};
    if (valid) key = map_key(cx.c, u128_add(zoff, z_cur));
    z_cur = z_next;
    GBR_STAMP_IF(w0, 11);
    const bool in_cur = valid && c.cur >= 0 && u128_lt(c.Ps, key) && !u128_lt(c.Pn, key);
    long long s_me = c.cur;
    u128 P_me = c.Ps;
    unsigned need = __ballot_sync(0xFFFFFFFFu, valid && !in_cur);
    if (!need && !c.head) {
      // every sample of the round lies in the current (non-head) segment:
      // the in-segment decision directly, without the grouping below
      if (valid) {
        const u128 rem = u128_lt(c.Ps, key) ? u128_sub(key, c.Ps) : u128{0ULL, 0ULL};
        const int cnt = lean_count(cx.s_pref + warp * kSeg, ceil_units(rem, c.sh, c.F));
        long long rr = c.cur * kSeg + (cnt < c.len ? cnt : c.len - 1);
        if (rr > M - 1) rr = M - 1;
        out[i] = (int)rr;
      }
      continue;
    }
    if (need) {
      // coarse block: the last j with coarse_j < key (coarse_0 = 0 < key)
      long long j_me = 0;
      if ((need >> lane) & 1u) {
        long long lo = 0, hi = ncoarse;
        while (lo < hi) {
          const long long mid = (lo + hi) >> 1;
          if (u128_lt(s_coarse[mid], key)) lo = mid + 1;
          else hi = mid;
        }
        j_me = lo > 0 ? lo - 1 : 0;
      }
      while (need) {
        const long long jj = __shfl_sync(0xFFFFFFFFu, j_me, __ffs(need) - 1);
        const unsigned grp = __ballot_sync(0xFFFFFFFFu, ((need >> lane) & 1u) && j_me == jj) & need;
        const long long blo = jj * stride;
        const long long bhi = blo + stride < nseg ? blo + stride : nseg;
        unsigned unres = grp;
        u128 prevP = kInf;  // prefix of segment c0 - 1
        for (long long c0 = blo; c0 < bhi && unres; c0 += 32) {
          const long long t = c0 + lane;
          u128 Pt = kInf;
          if (t < bhi) Pt = u128_add(s_cp[seg_owner(t, nseg, B)], u128{__ldcg(&rel[t].lo), __ldcg(&rel[t].hi)});
          my_win[lane] = Pt;
          __syncwarp();
          // a sample is resolved in the batch holding the first prefix that
          // reaches its key; the block's last batch also takes keys above
          // every prefix (the block's end, or S plus rounding)
          const bool last_batch = c0 + 32 >= bhi;
          bool here = false;
          if ((unres >> lane) & 1u) {
            int l2 = 0, h2 = 32;
            while (l2 < h2) {
              const int mid = (l2 + h2) >> 1;
              if (u128_lt(my_win[mid], key)) l2 = mid + 1;
              else h2 = mid;
            }
            here = l2 < 32 || last_batch;
            if (here) {
              if (l2 > 0) {
                s_me = c0 + l2 - 1;
                P_me = my_win[l2 - 1];
              } else {  // the batch's first prefix already reaches the key
                s_me = c0 - 1;
                P_me = prevP;
              }
            }
          }
          unres &= ~__ballot_sync(0xFFFFFFFFu, here);
          prevP = my_win[31];
          __syncwarp();
        }
        need &= ~grp;
      }
      if (s_me < 0) {  // only a zero key (all weights zero): the first segment
        s_me = 0;
        P_me = u128{0ULL, 0ULL};
      }
    }
    GBR_STAMP_IF(w0, 12);
    lean_round<T, kVec>(c, w, M, seg, valid, s_me, P_me, key, i, cx.Emax, cx.ge, my_pref,
                        my_buf + (long long)warp * kSeg, lane, out);
    GBR_STAMP_IF(w0, 13);
  }
}

}  // namespace

template <typename T, bool kVec>
__global__ void __launch_bounds__(kFThreads, 1) k_fused(FusedArgs a) {
  constexpr bool F32 = sizeof(T) == 4;
  using Bits = typename FixedTraits<T>::Bits;
  constexpr int kSegBytes = kSeg * (int)sizeof(T);
  constexpr int kSegsPerWarp = kStageBytes / kSegBytes / kFWarps;  // stage segments per streaming warp
  extern __shared__ __align__(128) unsigned char s_dyn[];
  __shared__ LogTab tab;
  __shared__ u128 s_w[kFWarps];
  __shared__ unsigned long long s_full[kStages], s_empty[kStages];
  __shared__ int s_e[kFWarps], s_x[kFWarps];
  __shared__ xf s_c, s_invZ;
  __shared__ u128 s_S, s_zoff;
  __shared__ u128 s_woff[kFWarps];  // spacing totals of the CTA's warps before each
  __shared__ u128 s_wz[kFWarps];    // the warps' spacing totals
  __shared__ int s_Emax, s_abort;
  __shared__ unsigned s_target;
  __shared__ unsigned long long s_lF[kLocalSegs];  // the CTA's segment records, when they fit
  __shared__ int s_lE[kLocalSegs];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B = gridDim.x, cta = blockIdx.x;
  const T* w = static_cast<const T*>(a.w);
  unsigned long long* x1 = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(a.xch) + 256);
  unsigned long long* x2 = x1 + kXSlotWords * kFusedMaxCtas;

  // ranges of this CTA; with few draws warp 15 makes them all while the
  // other fifteen stream the weights
  const int nSW = a.few ? kFWarps - 1 : kFWarps;  // streaming warps
  const long long kStageSegs = (long long)nSW * kSegsPerWarp;
  const long long s0 = a.nseg * cta / B, s1 = a.nseg * (cta + 1) / B;
  const long long d0 = a.ndraw * cta / B, d1 = a.ndraw * (cta + 1) / B;
  const long long tma_end = s1 < a.nfull ? s1 : (s0 > a.nfull ? s0 : a.nfull);  // full segments [s0, tma_end)
  const long long n_it = kVec ? (tma_end - s0 + kStageSegs - 1) / kStageSegs : 0;
  const bool local = s1 - s0 <= kLocalSegs;

  unsigned long long pol = 0;
  if (kVec) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  long long issued = 0;  // stages issued so far (thread 0)
  // stage it of the ring: segments [s0 + it*kStageSegs, ...) of the CTA range
  auto issue = [&](long long it) {
    const int st = (int)(it % kStages);
    const long long sa = s0 + it * kStageSegs;
    const long long sb = sa + kStageSegs < tma_end ? sa + kStageSegs : tma_end;
    const unsigned bytes = (unsigned)((sb - sa) * kSegBytes);
    mbar_expect_tx(&s_full[st], bytes);
    bulk_g2s(s_dyn + (size_t)st * kStageBytes, w + sa * kSeg, bytes, &s_full[st], pol);  // one copy per stage
    issued = it + 1;
  };
  if (tid == 0) {
    // the first stages travel before anything else is done
    if (kVec) {
      for (int s = 0; s < kStages; ++s) {
        mbar_init(&s_full[s], 1);
        mbar_init(&s_empty[s], (unsigned)nSW);
      }
      asm volatile("fence.mbarrier_init.release.cluster;\n fence.proxy.async.shared::cta;" ::: "memory");
      for (long long it = 0; it < n_it && it < kStages; ++it) issue(it);
    }
    s_abort = 0;
  }
  if (tid == 32) s_target = __ldcg(a.xch) + 1u;  // this call's epoch
  if (tid < kFWarps) s_wz[tid] = u128{0ULL, 0ULL};
  for (int i = tid; i < 129; i += kFThreads) {
    tab.nlogc[i] = a.tab->nlogc[i];
    tab.invc[i] = a.tab->invc[i];
  }
  __syncthreads();
  const unsigned target = s_target;
  const unsigned tag = target % 65535u + 1u;  // never 0 (a slot never written), differs between calls
  GBR_STAMP(0);
  GBR_STAMP(14);
  if (tid == kFThreads - 32) {
    // fetch the code of the once-per-call scalar steps (reciprocal, product)
    // into the instruction caches while the first copies are in flight
    const xf r = recip_total(u128{(unsigned long long)a.M | 1ULL, 0ULL});
    if (r.lo == 0x5A5A5A5AULL && r.hi == (unsigned long long)a.N) s_c = r;  // never true; keeps the call
  }

  // ---- phase 1a: the CTA's draws (Algorithm 1) -------------------------------
  // Many draws: warp w < nW draws exactly the samples it maps below, [m0 +
  // nsm w / nW, m0 + nsm (w+1) / nW), warp nW - 1 also the final draw N when
  // this CTA holds it, each warp with its own exact running prefix (warp
  // scans, no block barrier per tile); the warp totals are scanned once after
  // the stream, and the map adds the warp's offset.  With at most 2048 draws
  // the last warp takes none (it fetches the code of the scalar steps
  // meanwhile).  Few draws (a.few): warp 15 makes all of them during the
  // stream (below), every warp maps a sixteenth of the samples.
  const long long m0 = d0, m1 = d1 < a.N ? d1 : a.N;
  const long long nsm = m1 > m0 ? m1 - m0 : 0;
  const int nW = a.few || d1 - d0 > 4LL * kFThreads ? kFWarps : kFWarps - 1;
  const long long g0 = warp < nW ? m0 + nsm * warp / nW : 0;  // [0, 0): no draws
  const long long g1 = warp < nW - 1 ? m0 + nsm * (warp + 1) / nW : (warp < nW ? d1 : 0);
  const long long i1 = warp < nW ? m0 + nsm * (warp + 1) / nW : m1;
  if (!a.few) {
    const u128 t = draw_range<F32>(a, g0, g1, &tab, lane);
    if (lane == 0) s_wz[warp] = t;
  }
  GBR_STAMP(1);

  // ---- phase 1b: the CTA's segments (with few draws, warp 15's draws) ------
  int emax = 0;
  if (a.few && warp == kFWarps - 1) {
    const u128 t = draw_range<F32>(a, d0, d1, &tab, lane);
    if (lane == 0) s_wz[warp] = t;
  } else {
    if (kVec) {
#pragma unroll 1
      for (long long it = 0; it < n_it; ++it) {
        const int st = (int)(it % kStages);
        const unsigned par = (unsigned)((it / kStages) & 1);
        if (*(volatile int*)&s_abort) break;
        if (!mbar_wait(&s_full[st], par, kTmaSpin)) {
          // a copy that did not complete: no further stage is issued, and
          // the stages already issued are drained before the ring is reused
          if (lane == 0) {
            raise_status(a.status, ST_ETIMEOUT);
            *(volatile int*)&s_abort = 1;
          }
          break;
        }
        const long long sa = s0 + it * kStageSegs;
#pragma unroll
        for (int r = 0; r < kSegsPerWarp; ++r) {
          const int j = warp + r * nSW;
          const long long s = sa + j;
          if (s < tma_end) {
            uint64_t F;
            uint32_t E;
            seg_sum_smem<T>(s_dyn + (size_t)st * kStageBytes + (size_t)j * kSegBytes, lane, a.status, F, E);
            if (lane == 0) {
              a.seg[s] = SegRec{F, (int)E, kSeg};
              if (local) {
                s_lF[s - s0] = F;
                s_lE[s - s0] = (int)E;
              }
            }
            emax = max(emax, (int)E);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[st]);
        if (tid == 0 && it + kStages < n_it && !*(volatile int*)&s_abort) {
          // refill this stage once every streaming warp has read it
          if (!mbar_wait(&s_empty[st], par, kTmaSpin)) {
            raise_status(a.status, ST_ETIMEOUT);
            *(volatile int*)&s_abort = 1;
          } else {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(it + kStages);
          }
        }
      }
    }
    // segments not taken by the ring (unaligned weights, the ragged last one)
#pragma unroll 1
    for (long long s = (kVec ? tma_end : s0) + warp; s < s1; s += nSW) {
      Bits b[kSegV];
      load_seg_striped<T, kVec>(w, s * kSeg, a.M, lane, b);
      uint64_t F;
      uint32_t E;
      seg_sum_bits<T>(b, lane, a.status, F, E);
      if (lane == 0) {
        const long long rem = a.M - s * kSeg;
        a.seg[s] = SegRec{F, (int)E, (int)(rem < kSeg ? rem : kSeg)};
        if (local) {
          s_lF[s - s0] = F;
          s_lE[s - s0] = (int)E;
        }
      }
      emax = max(emax, (int)E);
    }
  }
  if (kVec && tid == 0 && *(volatile int*)&s_abort) {
    // drain: the last use of every stage issued completes (bounded) before
    // the shared memory of the ring is reused
    for (long long it = issued > kStages ? issued - kStages : 0; it < issued; ++it)
      mbar_wait(&s_full[it % kStages], (unsigned)((it / kStages) & 1), kTmaSpin);
  }
  if (lane == 0) s_e[warp] = emax;
  __syncthreads();
  GBR_STAMP(2);
  u128 ztot;  // the CTA's spacing total; the warps' offsets for the map
  {
    u128 before = {0ULL, 0ULL}, t = {0ULL, 0ULL};
#pragma unroll
    for (int i = 0; i < kFWarps; ++i) {
      const u128 x = s_wz[i];
      if (i < warp) before = u128_add(before, x);
      t = u128_add(t, x);
    }
    if (lane == 0) s_woff[warp] = before;
    ztot = t;
  }

  // ---- exchange 1: segment exponents and spacing totals ----------------------
  // (nothing else of this CTA is read by others before exchange 2, whose
  // writer fence covers it)
  if (tid == 0) {
    int m = 0;
#pragma unroll
    for (int i = 0; i < kFWarps; ++i) m = max(m, s_e[i]);
    if (!(a.withhold_first && cta == 0)) xput(x1 + kXSlotWords * cta, tag, ztot, (unsigned)m);
    GBR_STAMP(25);
  }
  {
    unsigned e = 0;
    u128 z = {0ULL, 0ULL};
    if (tid < B && !xget(x1 + kXSlotWords * tid, tag, a.spin, z, e)) {
      raise_status(a.status, ST_ETIMEOUT);
      e = 0;
      z = u128{0ULL, 0ULL};
    }
    GBR_STAMP(24);
    const int wm = (int)__reduce_max_sync(0xFFFFFFFFu, e);
    GBR_STAMP(8);
    if (lane == 0) s_x[warp] = wm;
    const BlockScan bs = block_scan(z, s_w);  // (its __syncthreads also publishes s_x)
    const u128 tot = bs.tot;
    if (tid == cta) s_zoff = bs.excl;  // spacing totals of the CTAs before this one
    if (tid == 0) {
      int m = 0;
#pragma unroll
      for (int i = 0; i < kFWarps; ++i) m = max(m, s_x[i]);
      s_Emax = m;
      s_S = tot;  // Z_{N+1}, until the reciprocal is taken
    }
    __syncthreads();
  }
  GBR_STAMP(3);

  // ---- phase 2: the CTA range on the global grid -----------------------------
  const int Emax = s_Emax;
  const long long stride = 1LL << a.lgstride;
  {
    const long long n = s1 - s0;
    const long long t_lo = s0 + n * tid / kFThreads, t_hi = s0 + n * (tid + 1) / kFThreads;
    u128 tsum = {0ULL, 0ULL};
#pragma unroll 1
    for (long long s = t_lo; s < t_hi; ++s) {
      const unsigned long long F = local ? s_lF[s - s0] : __ldcg(&a.seg[s].F);
      const int E = local ? s_lE[s - s0] : __ldcg(&a.seg[s].E);
      tsum = u128_add(tsum, grid_value(F, E, Emax));
    }
    GBR_STAMP(20);
    const BlockScan bs = block_scan(tsum, s_w);
    u128 R = bs.excl;
    const u128 ctot = bs.tot;
    GBR_STAMP(21);
#pragma unroll 1
    for (long long s = t_lo; s < t_hi; ++s) {
      a.rel[s] = SegPre{R.lo, R.hi};
      if ((s & (stride - 1)) == 0) a.crel[s >> a.lgstride] = SegPre{R.lo, R.hi};
      const unsigned long long F = local ? s_lF[s - s0] : __ldcg(&a.seg[s].F);
      const int E = local ? s_lE[s - s0] : __ldcg(&a.seg[s].E);
      R = u128_add(R, grid_value(F, E, Emax));
    }
    __syncthreads();  // rel, crel and the segment records precede the published total
    GBR_STAMP(22);
    if (tid == 0) {
      fence_acq_rel_gpu();  // release: rel, crel and the segment records precede the total
      GBR_STAMP(23);
      xput(x2 + kXSlotWords * cta, tag, ctot, 0u);
      GBR_STAMP(15);
    }
    if (tid == kFThreads - 32) {
      // 1 / Z_{N+1} while the exchange completes (this thread reads no slot)
      const u128 zt = s_S;
      s_invZ = u128_is_zero(zt) ? lb_zero<xf>() : recip_total(zt);
      GBR_STAMP_IF(true, 9);
    }
  }
  GBR_STAMP(4);

  // this warp's samples (the draws it made) and the spacing prefixes of
  // their first round, read before the exchange completes
  const long long i0 = warp < nW ? g0 : m1;
  u128 z_first = {0ULL, 0ULL};
  if (i0 + lane < i1) z_first = u128{__ldcg(&a.Z[i0 + lane].lo), __ldcg(&a.Z[i0 + lane].hi)};

  // ---- exchange 2: CTA totals -> CTA prefixes and S --------------------------
  u128* s_cp = reinterpret_cast<u128*>(s_dyn);          // [B + 1]
  u128* s_coarse = s_cp + (kFusedMaxCtas + 1);          // [ncoarse]
  unsigned long long* s_pref = reinterpret_cast<unsigned long long*>(s_coarse + kCoarseMax);  // kFWarps x 512
  u128* s_win = reinterpret_cast<u128*>(s_pref + kFWarps * kSeg);                           // kFWarps x 32
  Bits* s_buf = reinterpret_cast<Bits*>(s_win + kFWarps * 32);                              // kFWarps x 512
  {
    unsigned e = 0;
    u128 v = {0ULL, 0ULL};
    if (tid < B) {
      if (!xget(x2 + kXSlotWords * tid, tag, a.spin, v, e)) {
        raise_status(a.status, ST_ETIMEOUT);
        v = u128{0ULL, 0ULL};
      }
      GBR_STAMP(16);
      fence_acq_rel_gpu();  // acquire: the publishers' segment data are read below
      GBR_STAMP(17);
    }
    const BlockScan bs = block_scan(v, s_w);
    const u128 tot = bs.tot;
    GBR_STAMP(18);
    if (tid < B) s_cp[tid] = bs.excl;
    if (tid == 0) {
      s_cp[B] = tot;
      s_S = tot;
      if (u128_is_zero(tot)) {
        if (cta == 0) raise_status(a.status, ST_EZEROSUM);
        s_c = lb_zero<xf>();
      } else {
        s_c = xf_mul_ool(xf_make(tot.hi, tot.lo, 0), s_invZ);
      }
      GBR_STAMP(19);
      // every CTA has read this call's epoch (its totals are in): advance it
      if (cta == 0) st_release_flag(a.xch, target);
    }
    __syncthreads();
    GBR_STAMP(5);
#pragma unroll 1
    for (long long j = tid; j < a.ncoarse; j += kFThreads)
      s_coarse[j] = u128_add(s_cp[seg_owner(j << a.lgstride, a.nseg, B)],
                             u128{__ldcg(&a.crel[j].lo), __ldcg(&a.crel[j].hi)});
    __syncthreads();
  }
  GBR_STAMP(6);

  // ---- phase 3: the map of this CTA's samples --------------------------------
  MapCtx cx;
  cx.s_top = nullptr;
  cx.ntop = 0;
  cx.s_pref = s_pref;
  cx.s_win = s_win;
  cx.c = s_c;
  cx.S = s_S;
  cx.ge = (long long)Emax - a.kBS - kGridHead;
  cx.Emax = Emax;
  if (i1 > i0)
    map_own<T, kVec>(w, a.M, a.seg, a.rel, a.nseg, a.Z, u128_add(s_zoff, s_woff[warp]), z_first, i0, i1, cx, s_cp, s_coarse, a.ncoarse,
                     a.lgstride, B, s_buf, a.out);
#ifdef GBR_PHASE_STAMPS
  __syncthreads();
  GBR_STAMP(7);
#endif
}

size_t fused_smem_bytes(bool f32) {
  const size_t seg_bytes = (size_t)kSeg * (f32 ? 4 : 8);
  const size_t map = (size_t)(kFusedMaxCtas + 1) * 16 + (size_t)kCoarseMax * 16 + (size_t)kFWarps * kSeg * 8 +
                     (size_t)kFWarps * 32 * 16 + (size_t)kFWarps * seg_bytes;
  const size_t ring = (size_t)kStages * kStageBytes;
  return map > ring ? map : ring;
}

template <typename T, bool kVec>
static cudaError_t fused_t(const FusedLaunch& L, cudaStream_t st) {
  const size_t smem = fused_smem_bytes(sizeof(T) == 4);
  cudaError_t e = cudaFuncSetAttribute(k_fused<T, kVec>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<T, kVec>, kFThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int blocks = num_sms();
  if (blocks > kFusedMaxCtas) return cudaErrorCooperativeLaunchTooLarge;
  FusedArgs a;
  a.w = L.w;
  a.M = L.M;
  a.nseg = (L.M + kSeg - 1) / kSeg;
  a.nfull = L.M / kSeg;
  a.N = L.N;
  a.ndraw = L.N + 1;
  a.seed = L.seed;
  a.inst = L.inst;
  a.seg = L.seg;
  a.rel = L.rel;
  a.crel = static_cast<SegPre*>(L.crel);
  // coarse blocks of 2^lgstride segments, at most kCoarseMax of them
  a.lgstride = 5;
  while (((a.nseg + (1LL << a.lgstride) - 1) >> a.lgstride) > kCoarseMax) ++a.lgstride;
  a.ncoarse = (a.nseg + (1LL << a.lgstride) - 1) >> a.lgstride;
  a.Z = static_cast<u128*>(L.Z);
  a.xch = L.xch;
  a.status = L.status;
  a.spin = L.spin;
  a.withhold_first = L.withhold_first;
  a.tab = L.tab;
  // one warp makes all of a CTA's draws while the others stream when that
  // takes well under the CTA's share of the stream (about 1 us per 128
  // draws against about 45 GB/s per SM)
  {
    const long long draws_cta = (a.ndraw + blocks - 1) / blocks;
    const long long bytes_cta = L.M * (long long)sizeof(T) / blocks;
    a.few = kVec && draws_cta * 1024 <= bytes_cta;
  }
  a.kBS = sizeof(T) == 4 ? FixedTraits<float>::kBias + FixedTraits<float>::kShift
                         : FixedTraits<double>::kBias + FixedTraits<double>::kShift;
  a.out = L.out;
  a.scheme = L.scheme;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kFThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused<T, kVec>, a);
}

cudaError_t launch_fused(bool f32, bool vec, const FusedLaunch& L, cudaStream_t st) {
  if (f32) return vec ? fused_t<float, true>(L, st) : fused_t<float, false>(L, st);
  return vec ? fused_t<double, true>(L, st) : fused_t<double, false>(L, st);
}

}  // namespace gbr
