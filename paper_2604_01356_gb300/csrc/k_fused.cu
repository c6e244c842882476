// The whole single-instance path of rs_resample_w (Eq. 3, Algorithm 1 and
// the segmented map of Eq. 2) in ONE cooperative launch: every CTA is
// resident, and the phases are separated by grid-wide barriers instead of
// kernel boundaries.
//
//   phase 1  the spacing-scan tiles (Algorithm 1, tiles chained by decoupled
//            look-back, assigned by CTA index), then exact segment sums (one
//            warp per 512 weights): a static share per warp, the rest from a
//            shared queue so that the CTAs that drew spacing tiles take less.
//   barrier
//   phase 2  every CTA owns a contiguous range of segments: grid values on
//            the global grid (needs the largest exponent, known only now),
//            summed exactly; the CTA total is published.
//   barrier
//   phase 3  every CTA scans all CTA totals (the CTA-level prefixes and S)
//            and computes S / Z_{N+1}; then the map: a sample finds its CTA
//            range by binary search over those prefixes, its segment by an
//            exact scan of that range's segment sums (32 at a time, staged
//            in shared memory), and its element as in the standalone map.
//            No global segment prefixes or search index are written.
//
// Every barrier wait is bounded by spin_limit polls, after which the CTA
// latches RS_ETIMEOUT and continues (results are then unspecified, nothing
// hangs).  Arithmetic is that of the multi-kernel path, so the indices are
// identical to it.
#include "map_common.cuh"

namespace gbr {

namespace {

constexpr int kFThreads = 256;
constexpr int kFWarps = kFThreads / 32;
constexpr int kCoarseMax = 1024;         // coarse-index entries in shared memory
constexpr int kMaxCtas = 512;            // CTA prefixes in shared memory
constexpr int kDynChunk = 4;             // segments per dynamic work item of the weights pass
static_assert(kFWarps == kMapWarps, "the map phase uses the map's warp layout");

struct FusedArgs {
  const void* w;
  long long M, nseg, N, ndraw, utiles;
  unsigned long long seed, inst;
  SegRec* seg;
  unsigned* emax_g;   // the largest segment exponent (cleared per call)
  u128* agg;          // [gridDim.x]
  SegPre* rel;        // [nseg] prefix of each segment relative to its CTA range
  SegPre* crel;       // [ncoarse] the same for the first segment of each coarse block
  long long ncoarse, stride;
  int lgstride;
  PathConsts* consts;
  u128* Z;
  u128* Ztot;
  TileDesc<u128>* udesc;
  unsigned* work;     // work-queue counter (cleared per call)
  unsigned* bar;      // barrier counter (cleared per call)
  int* status;
  int spin;
  bool withhold_first;
  const LogTab* tab;  // logarithm table (binary64 draws)
  int G;
  int kBS;
  int* out;
};

__device__ __forceinline__ void grid_sync(unsigned* bar, unsigned& gen, int spin, int* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++gen;
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = gen * gridDim.x;
    int spins = 0;
    while (ld_acquire_u32(bar) < target) {
      if (++spins > spin) {
        raise_status(status, ST_ETIMEOUT);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
}

template <int kWarps>
__device__ __forceinline__ u128 block_sum_u128(u128 v, u128* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v = u128_add(v, shfl_v(v, lane ^ o));
  __syncthreads();
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  u128 t = {0ULL, 0ULL};
#pragma unroll
  for (int i = 0; i < kWarps; ++i) t = u128_add(t, s_w[i]);
  return t;
}

__device__ __noinline__ void fused_consts(PathConsts* consts, u128 S, long long ge, int Emax, int* status) {
  consts->S[0] = S.lo;
  consts->S[1] = S.hi;
  consts->ge = ge;
  consts->Emax = Emax;
  if (u128_is_zero(S)) {
    raise_status(status, ST_EZEROSUM);
    consts->c[0] = consts->c[1] = 0ULL;
    consts->c[2] = (unsigned long long)kXfZeroE;
    return;
  }
  const xf invZ = {__ldcg(consts->invZ), __ldcg(consts->invZ + 1), (long long)__ldcg(consts->invZ + 2)};
  const xf c = xf_mul(xf_make(S.hi, S.lo, 0), invZ);
  consts->c[0] = c.lo;
  consts->c[1] = c.hi;
  consts->c[2] = (unsigned long long)c.e;
}

// The map of the fused kernel: like map_groups, but a sample's segment is
// found from the coarse index in shared memory (the prefix of every
// stride-th segment) and then among that block's prefixes, each the CTA
// prefix plus the segment's prefix relative to its CTA range.
template <typename T, bool kVec>
__device__ __forceinline__ void map_groups_direct(const T* __restrict__ w, long long M,
                                                  const SegRec* __restrict__ seg, const SegPre* __restrict__ rel,
                                                  long long nseg, const u128* __restrict__ Z, long long N, int G,
                                                  const MapCtx& cx, const u128* s_cp, const u128* s_coarse,
                                                  const short* s_ccta, long long ncoarse, long long stride,
                                                  typename FixedTraits<T>::Bits* my_buf, long long g_first,
                                                  long long g_stride, int* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long* my_pref = cx.s_pref + warp * kSeg;
  u128* my_win = cx.s_win + warp * 32;
  const u128 kInf = {~0ULL, ~0ULL};
  for (long long g = g_first; g * (long long)G < N; g += g_stride) {
    const long long i0 = g * (long long)G;
    const long long i1 = (i0 + G < N) ? i0 + G : N;
    SegCache c;
    seg_cache_init(c);
    for (long long r0 = i0; r0 < i1; r0 += 32) {
      const long long i = r0 + lane;
      const bool valid = i < i1;
      u128 key = {0ULL, 0ULL};
      if (valid) key = map_key(cx.c, u128{__ldcg(&Z[i].lo), __ldcg(&Z[i].hi)});  // ceil(U_i * S) in grid units
      const bool in_cur = valid && c.cur >= 0 && u128_lt(c.Ps, key) && !u128_lt(c.Pn, key);
      long long s_me = c.cur;
      u128 P_me = c.Ps;
      unsigned need = __ballot_sync(0xFFFFFFFFu, valid && !in_cur);
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
          const int bcta = s_ccta[jj];
          const u128 cpb = s_cp[bcta];
          const long long blo = jj * stride;
          const long long bhi = blo + stride < nseg ? blo + stride : nseg;
          unsigned unres = grp;
          u128 prevP = kInf;  // prefix of segment c0 - 1
          // the block's prefixes, 32 at a time (one load per lane)
          for (long long c0 = blo; c0 < bhi && unres; c0 += 32) {
            const long long t = c0 + lane;
            u128 Pt = kInf;
            if (t < bhi) Pt = u128_add(cpb, u128{__ldcg(&rel[t].lo), __ldcg(&rel[t].hi)});
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
      }
      resolve_round<T, kVec>(c, w, M, seg, valid, s_me, P_me, key, i, cx, my_pref, lane, out,
                             my_buf + (long long)warp * kSeg);
    }
  }
}

}  // namespace

template <typename T, bool kVec>
__global__ void __launch_bounds__(kFThreads, 2) k_fused(FusedArgs a) {
  constexpr bool F32 = sizeof(T) == 4;
  using Bits = typename FixedTraits<T>::Bits;
  extern __shared__ __align__(16) unsigned long long s_dyn[];  // map staging
  __shared__ LogTab tab;
  __shared__ UniformTileSmem us;
  __shared__ int s_e[kFWarps];
  __shared__ u128 s_w[kFWarps];
  __shared__ xf s_c;
  __shared__ u128 s_S;
  __shared__ long long s_ge;
  __shared__ int s_Emax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* w = static_cast<const T*>(a.w);
  unsigned gen = 0;
  if (!F32)
    for (int i = tid; i < 129; i += kFThreads) {
      tab.nlogc[i] = a.tab->nlogc[i];
      tab.invc[i] = a.tab->invc[i];
    }
  __syncthreads();

  // ---- phase 1: spacing tiles, then segment sums ------------------------------
  // spacing tiles by CTA index: a tile waits only on lower tiles, which every
  // CTA processes in increasing order, so every wait ends
  const int B = gridDim.x;
  for (long long t = blockIdx.x; t < a.utiles; t += B)
    uniform_tile<F32>(t, a.ndraw, a.seed, a.inst, a.Z, a.Ztot, a.consts, a.udesc, a.status, a.spin,
                      a.withhold_first, &tab, us);
  // segments: a static round-robin share (half), then chunks of kDynChunk from
  // a shared counter; the next segment's loads are issued before the current
  // one is reduced.  When only some CTAs drew spacing tiles, the static share
  // goes to the others.
  int emax = 0;
  {
    const long long ub = a.utiles < B ? a.utiles : 0;  // CTAs left out of the static share
    const long long W = ((long long)B - ub) * kFWarps;
    const long long gw = ((long long)blockIdx.x - ub) * kFWarps + warp;
    const long long per = (long long)blockIdx.x < ub ? 0 : (a.nseg / 2) / W;
    const long long pool = ((a.nseg / 2) / W) * W;
    long long k = 0, dyn_s = 0, dyn_left = 0;
    auto next_seg = [&]() -> long long {
      if (k < per) return gw + (k++) * W;
      if (dyn_left == 0) {
        unsigned c = 0;
        if (lane == 0) c = atomicAdd(a.work, 1u);
        c = __shfl_sync(0xFFFFFFFFu, c, 0);
        dyn_s = pool + (long long)c * kDynChunk;
        dyn_left = kDynChunk;
      }
      --dyn_left;
      return dyn_s++;
    };
    long long cur = next_seg();
    Bits cb[kSegV];
    if (cur < a.nseg) load_seg_striped<T, kVec>(w, cur * kSeg, a.M, lane, cb);
    while (cur < a.nseg) {
      const long long nxt = next_seg();
      Bits nb[kSegV];
      if (nxt < a.nseg) load_seg_striped<T, kVec>(w, nxt * kSeg, a.M, lane, nb);
      uint64_t F;
      uint32_t E;
      seg_sum_bits<T>(cb, lane, a.status, F, E);
      if (lane == 0) {
        const long long rem = a.M - cur * kSeg;
        a.seg[cur] = SegRec{F, (int)E, (int)(rem < kSeg ? rem : kSeg)};
      }
      emax = max(emax, (int)E);
      cur = nxt;
#pragma unroll
      for (int q = 0; q < kSegV; ++q) cb[q] = nb[q];
    }
  }
  if (lane == 0) s_e[warp] = emax;
  __syncthreads();
  if (tid == 0) {
    int m = 0;
#pragma unroll
    for (int i = 0; i < kFWarps; ++i) m = max(m, s_e[i]);
    atomicMax(a.emax_g, (unsigned)m);
  }
  grid_sync(a.bar, gen, a.spin, a.status);

  // ---- phase 2: grid values of this CTA's segment range ----------------------
  const int Emax = (int)__ldcg(a.emax_g);
  {
    // consecutive sub-ranges per thread; exclusive scan inside the CTA gives
    // every segment's prefix relative to the CTA range's start
    // the CTA owns whole coarse blocks: [jlo, jhi) of stride segments each
    const int nc = (int)a.ncoarse;  // <= kCoarseMax: 32-bit division
    const int jlo = nc * (int)blockIdx.x / B, jhi = nc * ((int)blockIdx.x + 1) / B;
    const long long lo = (long long)jlo * a.stride;
    const long long hi = (long long)jhi * a.stride < a.nseg ? (long long)jhi * a.stride : a.nseg;
    const long long t_lo = lo + (hi - lo) * tid / kFThreads, t_hi = lo + (hi - lo) * (tid + 1) / kFThreads;
    u128 tsum = {0ULL, 0ULL};
    for (long long s = t_lo; s < t_hi; ++s)
      tsum = u128_add(tsum, grid_value(__ldcg(&a.seg[s].F), __ldcg(&a.seg[s].E), Emax));
    const u128 incl = warp_incl_scan_v(tsum, lane);
    __syncthreads();
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    u128 R = u128_sub(incl, tsum), ctot = {0ULL, 0ULL};
#pragma unroll
    for (int i = 0; i < kFWarps; ++i) {
      if (i < warp) R = u128_add(R, s_w[i]);
      ctot = u128_add(ctot, s_w[i]);
    }
    for (long long s = t_lo; s < t_hi; ++s) {
      a.rel[s] = SegPre{R.lo, R.hi};
      if ((s & (a.stride - 1)) == 0) a.crel[s >> a.lgstride] = SegPre{R.lo, R.hi};
      R = u128_add(R, grid_value(__ldcg(&a.seg[s].F), __ldcg(&a.seg[s].E), Emax));
    }
    if (tid == 0) a.agg[blockIdx.x] = ctot;
  }
  grid_sync(a.bar, gen, a.spin, a.status);

  // ---- phase 3: CTA prefixes, S, S / Z_{N+1}; the map -------------------------
  u128* s_cp = reinterpret_cast<u128*>(s_dyn + kMapWarps * kSeg + kMapWarps * 32 * 2);  // [B + 1]
  u128* s_coarse = s_cp + (kMaxCtas + 1);                                                   // [ncoarse]
  short* s_ccta = reinterpret_cast<short*>(s_coarse + kCoarseMax);                          // CTA of each entry
  {
    // the coarse entries' relative prefixes go to shared memory while the CTA
    // totals are scanned; each thread then adds the CTA prefix to the entries
    // of CTAs 2 tid and 2 tid + 1
    const int t0 = 2 * tid;
    for (long long j = tid; j < a.ncoarse; j += kFThreads)
      s_coarse[j] = u128{__ldcg(&a.crel[j].lo), __ldcg(&a.crel[j].hi)};
    const u128 v0 = t0 < B ? u128{__ldcg(&a.agg[t0].lo), __ldcg(&a.agg[t0].hi)} : u128{0ULL, 0ULL};
    const u128 v1 = t0 + 1 < B ? u128{__ldcg(&a.agg[t0 + 1].lo), __ldcg(&a.agg[t0 + 1].hi)} : u128{0ULL, 0ULL};
    xf invZ = lb_zero<xf>();
    if (tid == 0) invZ = xf{__ldcg(a.consts->invZ), __ldcg(a.consts->invZ + 1), (long long)__ldcg(a.consts->invZ + 2)};
    const u128 pair = u128_add(v0, v1);
    const u128 incl = warp_incl_scan_v(pair, lane);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    u128 off = u128_sub(incl, pair), tot = {0ULL, 0ULL};
#pragma unroll
    for (int i = 0; i < kFWarps; ++i) {
      if (i < warp) off = u128_add(off, s_w[i]);
      tot = u128_add(tot, s_w[i]);
    }
    const u128 cpq[2] = {off, u128_add(off, v0)};
    if (tid == 0) {  // S / Z_{N+1} while the others place the coarse entries
      s_S = tot;
      s_c = u128_is_zero(tot) ? lb_zero<xf>() : xf_mul(xf_make(tot.hi, tot.lo, 0), invZ);
    }
    __syncthreads();  // the relative entries are in place
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int b = t0 + q;
      if (b < B) {
        s_cp[b] = cpq[q];
        const int jl = (int)a.ncoarse * b / B, jh = (int)a.ncoarse * (b + 1) / B;
        for (int j = jl; j < jh; ++j) {
          s_coarse[j] = u128_add(cpq[q], s_coarse[j]);
          s_ccta[j] = (short)b;
        }
      }
    }
    if (tid == 0) s_cp[B] = tot;
    if (tid == 32 && blockIdx.x == 0) fused_consts(a.consts, tot, (long long)Emax - a.kBS - kGridHead, Emax, a.status);
    __syncthreads();
  }
  MapCtx cx;
  cx.s_top = nullptr;
  cx.ntop = 0;
  cx.s_pref = s_dyn;
  cx.s_win = reinterpret_cast<u128*>(s_dyn + kMapWarps * kSeg);
  cx.c = s_c;
  cx.S = s_S;
  cx.ge = (long long)Emax - a.kBS - kGridHead;
  cx.Emax = Emax;
  Bits* s_buf = reinterpret_cast<Bits*>(s_ccta + kCoarseMax);  // kMapWarps x 512 prefetched weights
  map_groups_direct<T, kVec>(w, a.M, a.seg, a.rel, a.nseg, a.Z, a.N, a.G, cx, s_cp, s_coarse, s_ccta, a.ncoarse,
                             a.stride, s_buf, (long long)blockIdx.x * kFWarps + warp, (long long)gridDim.x * kFWarps,
                             a.out);
}

template <typename T, bool kVec>
static cudaError_t fused_t(const FusedLaunch& L, cudaStream_t st) {
  const int max_b = 2 * num_sms();
  const size_t smem = (size_t)kMapWarps * kSeg * sizeof(unsigned long long) + (size_t)kMapWarps * 32 * sizeof(u128) +
                      (size_t)(kMaxCtas + 1) * sizeof(u128) + (size_t)kCoarseMax * sizeof(u128) +
                      (size_t)kCoarseMax * sizeof(short) + (size_t)kMapWarps * kSeg * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_fused<T, kVec>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<T, kVec>, kFThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if (per_sm > 2) per_sm = 2;
  const int blocks = num_sms() * per_sm;
  if (blocks > L.max_blocks || blocks > max_b || blocks > kMaxCtas) return cudaErrorCooperativeLaunchTooLarge;
  FusedArgs a;
  a.w = L.w;
  a.M = L.M;
  a.nseg = (L.M + kSeg - 1) / kSeg;
  a.N = L.N;
  a.ndraw = L.N + 1;
  a.utiles = (a.ndraw + kUTile - 1) / kUTile;
  a.seed = L.seed;
  a.inst = L.inst;
  a.seg = L.seg;
  a.emax_g = L.emax_g;
  a.agg = static_cast<u128*>(L.agg);
  a.rel = L.rel;
  a.crel = static_cast<SegPre*>(L.crel);
  // coarse blocks: at most kCoarseMax, and at most 8 per CTA
  const long long cmax = kCoarseMax < 8LL * blocks ? kCoarseMax : 8LL * blocks;
  a.stride = 32;
  a.lgstride = 5;
  while ((a.nseg + a.stride - 1) / a.stride > cmax) {
    a.stride *= 2;
    ++a.lgstride;
  }
  a.ncoarse = (a.nseg + a.stride - 1) / a.stride;
  a.consts = L.consts;
  a.Z = static_cast<u128*>(L.Z);
  a.Ztot = static_cast<u128*>(L.Ztot);
  a.udesc = static_cast<TileDesc<u128>*>(L.udesc);
  a.work = L.work;
  a.bar = L.bar;
  a.status = L.status;
  a.spin = L.spin;
  a.withhold_first = L.withhold_first;
  a.tab = L.tab;
  long long G = (L.N + (long long)blocks * kFWarps - 1) / ((long long)blocks * kFWarps);
  a.G = (int)(G < 1 ? 1 : G);
  a.kBS = sizeof(T) == 4 ? FixedTraits<float>::kBias + FixedTraits<float>::kShift
                         : FixedTraits<double>::kBias + FixedTraits<double>::kShift;
  a.out = L.out;
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
