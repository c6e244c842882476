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
#include <cstddef>

#include "cluster.cuh"
#include "map_common.cuh"

namespace gbr {

__device__ __forceinline__ long long ldkey(const double* __restrict__ p) {
  return ord_key_bits(__ldg(reinterpret_cast<const long long*>(p)));
}

template <typename T, bool kVec>
__global__ void __launch_bounds__(kMapWarps * 32, 2) k_map_seg(const T* __restrict__ w, long long M,
                                                              const SegRec* __restrict__ seg,
                                                              const SegPre* __restrict__ pre, SegIndex idx,
                                                              const PathConsts* __restrict__ consts,
                                                              const u128* __restrict__ Z, long long N, int G, int ntop,
                                                              int* __restrict__ out) {
  extern __shared__ __align__(16) unsigned long long s_dyn[];
  __shared__ xf s_c;
  __shared__ u128 s_S;
  __shared__ long long s_ge;
  __shared__ int s_Emax;
  for (int t = threadIdx.x; t < ntop; t += blockDim.x) s_dyn[t] = __ldcg(idx.lvl[1] + t);
  if (threadIdx.x == 0) {
    s_c = ld_consts_xf(consts->c);
    s_S = u128{__ldcg(consts->S), __ldcg(consts->S + 1)};
    s_ge = (long long)__ldcg((const unsigned long long*)&consts->ge);
    s_Emax = (int)__ldcg((const unsigned long long*)&consts->Emax);
  }
  __syncthreads();
  MapCtx cx;
  cx.s_top = s_dyn;
  cx.ntop = ntop;
  cx.s_pref = s_dyn + ((ntop + 1) & ~1);
  cx.s_win = reinterpret_cast<u128*>(cx.s_pref + kMapWarps * kSeg);
  cx.c = s_c;
  cx.S = s_S;
  cx.ge = s_ge;
  cx.Emax = s_Emax;
  map_groups<T, kVec>(w, M, seg, pre, idx, Z, N, G, cx, ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                      ((long long)gridDim.x * blockDim.x) >> 5, out);
}

template <typename T, bool kVec>
static cudaError_t map_seg_t(const void* w, long long M, const SegRec* seg, const SegPre* pre, const SegIndex& idx,
                             const PathConsts* consts, const void* Z, long long N, int G, int* out, cudaStream_t st) {
  const long long groups = (N + G - 1) / G;
  long long blocks = (groups + kMapWarps - 1) / kMapWarps;
  const long long cap = (long long)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  // stage level 1 of the segment index in shared memory when it is small
  int ntop = 0;
  if (idx.nlev >= 2 && idx.lvl_n[1] <= kMapTopMax) ntop = (int)idx.lvl_n[1];
  const size_t smem = (size_t)((ntop + 1) & ~1) * sizeof(unsigned long long) +
                      (size_t)kMapWarps * kSeg * sizeof(unsigned long long) + (size_t)kMapWarps * 32 * sizeof(u128);
  cudaError_t e = cudaFuncSetAttribute(k_map_seg<T, kVec>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_map_seg<T, kVec><<<(unsigned)blocks, kMapWarps * 32, smem, st>>>((const T*)w, M, seg, pre, idx, consts,
                                                                     (const u128*)Z, N, G, ntop, out);
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

// ---------------------------------------------------------------------------
// The sampling steps of a small instance on one CTA (M <= 12,288, N <= 2047):
// W travels to shared memory while the draws are made; then 1 / Z_{N+1} (warp
// 15), U_i exactly as the one-CTA uniform kernel forms it, and the map named
// by kAlgo over W in shared memory:
//   kMapDac     Algorithm 5: leaves of L samples; each leaf's last sample is
//               located in W[0, M-1], its first in [0, r_last] (the split
//               argument), and the samples between walk forward from there;
//   kMapBinary  Algorithm 3: one lower-bound search of W per sample;
//   kMapLinear  Algorithm 4: thread t owns W[M t / 512, M (t+1) / 512) and the
//               samples whose answers fall there, found by one search of U,
//               and merge-walks them.
// Comparisons are exact (total-order integer keys), so all three equal the
// multi-launch maps bit for bit.
enum : int { kMapDac = 0, kMapBinary = 1, kMapLinear = 2 };
constexpr int kSwThreads = kSmallThreadsW;
struct SmallWSmem {
  long long Wk[kSmallMaxM];  // W's bits, then their total-order keys
  long long Uk[kSmallMaxN];  // the keys of U
  u128 wsum[kSwThreads / 32];
  alignas(16) u128 part;  // this CTA's spacing total, read by the other CTAs of a cluster (16-byte loads)
  xf r;
  LogTab tab;
};
static_assert(offsetof(SmallWSmem, part) % 16 == 0, "16-byte cluster loads of part");
__device__ __forceinline__ long long lower_bound_sm(const long long* Wk, long long a, long long b, long long key) {
  while (a < b) {  // smallest m in [a, b] with Wk[m] >= key, else b
    const long long m = (a + b) >> 1;
    if (Wk[m] < key) a = m + 1;
    else b = m;
  }
  return b;
}

// kG > 1: a cluster of kG CTAs; CTA r makes the draws of its share of the
// Philox blocks, forms U for those samples and maps them against its own copy
// of W; the spacing totals are exchanged once through distributed shared
// memory, so U is exactly that of one CTA.
template <bool F32, int kAlgo, int kG>
__global__ void __launch_bounds__(kSwThreads, 1) k_small_W(const double* __restrict__ W, long long M, long long N,
                                                           unsigned long long seed, unsigned long long inst, int L,
                                                           int* __restrict__ out, int scheme,
                                                           const LogTab* __restrict__ tab) {
  constexpr int kWarps = kSwThreads / 32;
  constexpr int kCopyThreads = kSwThreads - 32;  // warp 15 computes 1 / Z_{N+1} meanwhile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmallWSmem& sm = *reinterpret_cast<SmallWSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool vec = (reinterpret_cast<uintptr_t>(W) & 15) == 0;
  const long long nchunk = vec ? M / 2 : 0;  // 16-byte chunks
  if (tid < kCopyThreads) {
    for (long long q = tid; q < nchunk; q += kCopyThreads)
      cp_async16(sm.Wk + 2 * q, reinterpret_cast<const char*>(W) + 16 * q);
    cp_async_commit();
  }
  // the logarithm table: loaded now, stored to shared memory after the
  // Philox blocks (which do not need it)
  float2 tnl = {0.0f, 0.0f}, tic = {0.0f, 0.0f};
  if (tid < 129) {
    tnl = tab->nlogc[tid];
    tic = tab->invc[tid];
  }

  // ---- Algorithm 1, exactly as the one-CTA uniform kernel ------------------
  // Multinomial draws: one per thread when the CTA holds at most 512, two when
  // at most 1024, else four (one Philox block per thread).
  const long long ndraw = N + 1;
  const int rank = kG > 1 ? (int)cluster_rank() : 0;
  const long long nblk = (ndraw + 3) / 4;
  const long long ka = 4 * (nblk * rank / kG);
  const long long kb = rank == kG - 1 ? ndraw : 4 * (nblk * (rank + 1) / kG);
  const long long ns = (kb < N ? kb : N) - ka;  // this CTA's samples [ka, ka + ns)
  const int dpt = scheme != kSchemeMultinomial ? 4 : kb - ka <= kSwThreads ? 1 : kb - ka <= 2 * kSwThreads ? 2 : 4;
  const long long k0 = ka + (long long)dpt * tid;
  u128 z[4];
  {
    uint64_t wd[4] = {0ULL, 0ULL, 0ULL, 0ULL};
    if (k0 < kb) philox4x64_10((uint64_t)(k0 / 4), 0ULL, 0ULL, 0ULL, seed, inst, wd);
    if (tid < 129) {
      sm.tab.nlogc[tid] = tnl;
      sm.tab.invc[tid] = tic;
    }
    __syncthreads();
    u128 f[4];
    if (dpt == 1) {
      const int o = (int)(k0 & 3);
      const uint64_t x = o == 0 ? wd[0] : o == 1 ? wd[1] : o == 2 ? wd[2] : wd[3];
      f[0] = k0 < kb ? spacing_fixed<F32>(x, &sm.tab) : u128{0ULL, 0ULL};
      f[1] = f[2] = f[3] = u128{0ULL, 0ULL};
    } else if (dpt == 2) {
      const int o = (int)(k0 & 3);
      f[0] = k0 < kb ? spacing_fixed<F32>(o ? wd[2] : wd[0], &sm.tab) : u128{0ULL, 0ULL};
      f[1] = k0 + 1 < kb ? spacing_fixed<F32>(o ? wd[3] : wd[1], &sm.tab) : u128{0ULL, 0ULL};
      f[2] = f[3] = u128{0ULL, 0ULL};
    } else {
      block_spacings<F32>(scheme, k0, ndraw, seed, inst, wd, &sm.tab, f);
      if (k0 >= kb) f[0] = f[1] = f[2] = f[3] = u128{0ULL, 0ULL};  // another CTA's draws
    }
    u128 run = {0ULL, 0ULL};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      run = u128_add(run, f[q]);
      z[q] = run;
    }
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
    if (kG > 1) {
      // the CTAs' spacing totals: this CTA's offset and Z_{N+1}
      if (tid == 0) sm.part = tot;
      cluster_sync_all();
      tot = u128{0ULL, 0ULL};
#pragma unroll
      for (int r = 0; r < kG; ++r) {
        const u128 v = ld_cluster_u128(&sm.part, (unsigned)r);
        if (r < rank) off = u128_add(off, v);
        tot = u128_add(tot, v);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) z[q] = u128_add(off, z[q]);  // Z_{k0+q+1}
    if (tid == kCopyThreads) sm.r = u128_is_zero(tot) ? lb_zero<xf>() : recip_total(tot);
  }
  if (tid < kCopyThreads) {
    cp_async_wait_all();
    for (long long e = 2 * nchunk + tid; e < M; e += kCopyThreads)
      sm.Wk[e] = __ldg(reinterpret_cast<const long long*>(W + e));
    asm volatile("bar.sync 1, %0;" ::"n"(kCopyThreads) : "memory");
    for (long long e = tid; e < M; e += kCopyThreads) sm.Wk[e] = ord_key_bits(sm.Wk[e]);
  }
  __syncthreads();
  {
    const xf r = sm.r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q < dpt && k0 + q < ka + ns) {
        long long ub = (long long)xf_to_f64_bits(xf_mul_u128(r, z[q]));
        if (ub > 0x3FF0000000000000LL) ub = 0x3FF0000000000000LL;
        sm.Uk[k0 + q - ka] = ord_key_bits(ub);
      }
    }
  }
  __syncthreads();

  // ---- the map of this CTA's samples (local index i is sample ka + i) ----------
  const long long* Wk = sm.Wk;
  const long long* Uk = sm.Uk;
  int* outk = out + ka;
  if (kAlgo == kMapBinary) {
    for (long long i = tid; i < ns; i += kSwThreads) outk[i] = (int)lower_bound_sm(Wk, 0, M - 1, Uk[i]);
  } else if (kAlgo == kMapLinear) {
    const long long a = M * tid / kSwThreads, b = M * (tid + 1) / kSwThreads;
    if (a < b) {
      // the slice's samples: W[a-1] < U_i <= W[b-1] (the last slice: all above W[a-1])
      long long i = 0;
      if (a > 0) {
        long long lo = 0, hi = ns;
        while (lo < hi) {
          const long long m = (lo + hi) >> 1;
          if (Uk[m] <= Wk[a - 1]) lo = m + 1;
          else hi = m;
        }
        i = lo;
      }
      const bool last = b == M;
      long long j = a;
      for (; i < ns; ++i) {
        const long long k = Uk[i];
        if (!last && k > Wk[b - 1]) break;
        while (j < M - 1 && Wk[j] < k) ++j;
        outk[i] = (int)j;
      }
    }
  } else {
    const long long nleaf = (ns + L - 1) / L;
    for (long long leaf = tid; leaf < nleaf; leaf += kSwThreads) {
      const long long a = leaf * (long long)L;
      const long long b = (a + L < ns ? a + L : ns) - 1;
      const long long rb = lower_bound_sm(Wk, 0, M - 1, Uk[b]);
      long long j = lower_bound_sm(Wk, 0, rb, Uk[a]);
      outk[a] = (int)j;
      for (long long i = a + 1; i <= b; ++i) {
        const long long k = Uk[i];
        while (j < rb && Wk[j] < k) ++j;
        outk[i] = (int)j;
      }
    }
  }
  if (kG > 1) cluster_sync_all();  // no CTA leaves while another may read its shared memory
}

template <bool F32, int kAlgo, int kG>
static cudaError_t small_W_go(const double* W, long long M, long long N, unsigned long long seed,
                              unsigned long long inst, int L, int* out, cudaStream_t st, int scheme, const LogTab* tab) {
  const size_t smem = sizeof(SmallWSmem);
  cudaError_t e = cudaFuncSetAttribute(k_small_W<F32, kAlgo, kG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (kG == 1) {
    k_small_W<F32, kAlgo, 1><<<1, kSwThreads, smem, st>>>(W, M, N, seed, inst, L, out, scheme, tab);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kG, 1, 1);
  cfg.blockDim = dim3(kSwThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kG;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_small_W<F32, kAlgo, kG>, W, M, N, seed, inst, L, out, scheme, tab);
  if (e == cudaSuccess) return e;
  // a device that cannot place the cluster: the one-CTA form (same indices)
  (void)cudaGetLastError();
  return small_W_go<F32, kAlgo, 1>(W, M, N, seed, inst, L, out, st, scheme, tab);
}

template <bool F32, int kG>
static cudaError_t small_W_t(int algo, const double* W, long long M, long long N, unsigned long long seed,
                             unsigned long long inst, int L, int* out, cudaStream_t st, int scheme, const LogTab* tab) {
  if (algo == kMapBinary) return small_W_go<F32, kMapBinary, kG>(W, M, N, seed, inst, L, out, st, scheme, tab);
  if (algo == kMapLinear) return small_W_go<F32, kMapLinear, kG>(W, M, N, seed, inst, L, out, st, scheme, tab);
  return small_W_go<F32, kMapDac, kG>(W, M, N, seed, inst, L, out, st, scheme, tab);
}

cudaError_t launch_small_W(bool f32, int algo, const double* W, long long M, long long N, unsigned long long seed,
                           unsigned long long inst, int L, int* out, cudaStream_t st, int scheme, const LogTab* tab,
                           int cluster) {
  if (N <= 0 || M <= 0) return cudaSuccess;
  if (N > kSmallMaxN || M > kSmallMaxM || L < 1) return cudaErrorInvalidValue;
  if (cluster == 4)
    return f32 ? small_W_t<true, 4>(algo, W, M, N, seed, inst, L, out, st, scheme, tab)
               : small_W_t<false, 4>(algo, W, M, N, seed, inst, L, out, st, scheme, tab);
  return f32 ? small_W_t<true, 1>(algo, W, M, N, seed, inst, L, out, st, scheme, tab)
             : small_W_t<false, 1>(algo, W, M, N, seed, inst, L, out, st, scheme, tab);
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
