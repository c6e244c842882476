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
//   C  total Z_{N+1}  all N+1 spacings of Algorithm 1 summed exactly;
//   D  map            the spacings again, in chunks of 4 per thread, scanned
//                     into Z_i; key_i = ceil(Z_i S / Z_{N+1}); the segment by
//                     binary search over the shared-memory prefixes; the
//                     element inside the segment from the segment's exact
//                     prefixes - by a warp-wide count when few samples fall
//                     in the segment, else by per-lane binary search over the
//                     prefixes staged in shared memory (the leaf threshold).
// Every step uses the single-instance path's arithmetic (same segment sums,
// grid, spacings, keys and in-segment decisions), so the indices equal those
// of rs_resample_w on each instance bit for bit.
//
// Instances with more than kBMaxSeg segments are not processed here (the host
// sends them through the multi-CTA single-instance path).
#include "seg_common.cuh"

namespace gbr {

namespace {

template <int kWarps>
struct BatchSmem {
  u128 pre[kBMaxSeg + 1];         // exclusive grid prefixes; pre[nseg] = S
  unsigned long long F[kBMaxSeg];  // segment sums on their own grids
  int E[kBMaxSeg];                 // segment exponents
  unsigned long long pref[kWarps][kSeg];  // staged in-segment prefixes (leaf search)
  u128 wsum[kWarps];
  xf c;
  int emax_w[kWarps];
  int item;
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

__device__ __noinline__ void compute_c(xf* dst, u128 S, u128 Ztot) {
  *dst = xf_mul(xf_make(S.hi, S.lo, 0), recip_total(Ztot));
}

}  // namespace

template <int kThreads>
__global__ void __launch_bounds__(kThreads) k_batched_f32(const float* __restrict__ w,
                                                          const long long* __restrict__ w_off,
                                                          const long long* __restrict__ r_off,
                                                          const int* __restrict__ order, int K,
                                                          unsigned long long seed, int leaf_T,
                                                          int* __restrict__ out, unsigned* queue, int* status,
                                                          int scheme) {
  using Tr = FixedTraits<float>;
  using Bits = Tr::Bits;
  constexpr int kWarps = kThreads / 32;
  constexpr int kChunk = kThreads * 4;  // draws per block per chunk (4 per thread)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem<kWarps>& sm = *reinterpret_cast<BatchSmem<kWarps>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  while (true) {
    __syncthreads();  // the previous instance is done with shared memory
    if (tid == 0) sm.item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int item = sm.item;
    if (item >= K) break;
    const int k = order[item];
    const long long wb = w_off[k];
    const long long Mk = w_off[k + 1] - wb;
    const long long rb = r_off[k];
    const long long Nk = r_off[k + 1] - rb;
    if (Nk <= 0 || Mk <= 0) continue;
    const long long nseg = (Mk + kSeg - 1) / kSeg;
    if (nseg > kBMaxSeg) continue;  // left to the single-instance path
    const float* wk = w + wb;
    const bool vec = (reinterpret_cast<uintptr_t>(wk) & 15) == 0;
    int* outk = out + rb;

    // ---- A: exact segment sums, two segments in flight per warp --------------
    int em = 0;
    for (int s0 = warp; s0 < nseg; s0 += 2 * kWarps) {
      const int s1 = s0 + kWarps;
      Bits b0[kSegV], b1[kSegV];
      if (vec) {
        load_seg_striped<float, true>(wk, (long long)s0 * kSeg, Mk, lane, b0);
        if (s1 < nseg) load_seg_striped<float, true>(wk, (long long)s1 * kSeg, Mk, lane, b1);
      } else {
        load_seg_striped<float, false>(wk, (long long)s0 * kSeg, Mk, lane, b0);
        if (s1 < nseg) load_seg_striped<float, false>(wk, (long long)s1 * kSeg, Mk, lane, b1);
      }
      uint64_t F;
      uint32_t E;
      seg_sum_bits<float>(b0, lane, status, F, E);
      if (lane == 0) {
        sm.F[s0] = F;
        sm.E[s0] = (int)E;
      }
      em = max(em, (int)E);
      if (s1 < nseg) {
        seg_sum_bits<float>(b1, lane, status, F, E);
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

    // ---- C: Z_{N+1}, the sum of all N+1 spacings ----------------------------
    const long long ndraw = Nk + 1;
    u128 zsum = {0ULL, 0ULL};
    if (scheme == kSchemeMultinomial)
      for (long long d0 = (long long)tid * 4; d0 < ndraw; d0 += kChunk) {
        uint64_t wd[4];
        philox4x64_10((uint64_t)(d0 / 4), 0ULL, 0ULL, 0ULL, seed, (uint64_t)k, wd);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (d0 + q < ndraw) zsum = u128_add(zsum, spacing_fixed<true>(wd[q], nullptr));
      }
    else if (tid == 0)
      zsum = u128{0ULL, (unsigned long long)Nk << 24};  // the strata spacings telescope to N
    u128 Ztot;
    (void)block_excl_scan<kWarps>(zsum, sm.wsum, Ztot);
    u128 vsys = {0ULL, 0ULL};  // systematic: the one draw v_0
    if (scheme == kSchemeSystematic) {
      uint64_t w0[4];
      philox4x64_10(0ULL, 0ULL, 0ULL, 0ULL, seed, (uint64_t)k, w0);
      vsys = draw_fixed<true>(w0[0]);
    }
    if (tid == 0) compute_c(&sm.c, S, Ztot);
    __syncthreads();
    const xf c = sm.c;

    // ---- D: Z_i, keys and the map, 4 rounds of 32 samples per warp ----------
    u128 carry = {0ULL, 0ULL};
    for (long long cb = 0; cb < Nk; cb += kChunk) {
      const long long wbase = cb + (long long)warp * 128;  // this warp's 128 draws
      uint64_t wd[4];
      philox4x64_10((uint64_t)((wbase + 4 * lane) / 4), 0ULL, 0ULL, 0ULL, seed, (uint64_t)k, wd);
      u128 f[4], inc[4];
      u128 wtot = {0ULL, 0ULL};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int src = 8 * r + (lane >> 2);
        const uint64_t x0 = __shfl_sync(0xFFFFFFFFu, wd[0], src);
        const uint64_t x1 = __shfl_sync(0xFFFFFFFFu, wd[1], src);
        const uint64_t x2 = __shfl_sync(0xFFFFFFFFu, wd[2], src);
        const uint64_t x3 = __shfl_sync(0xFFFFFFFFu, wd[3], src);
        const int wq = lane & 3;
        const uint64_t word = wq == 0 ? x0 : wq == 1 ? x1 : wq == 2 ? x2 : x3;
        const long long d = wbase + 32 * r + lane;
        if (scheme == kSchemeMultinomial) {
          f[r] = d < Nk ? spacing_fixed<true>(word, nullptr) : u128{0ULL, 0ULL};
        } else {
          // word d - 1: the previous word of this block, the last word of the
          // previous lane's block, or (draw 32 r of the chunk) recomputed
          uint64_t wp = __shfl_sync(0xFFFFFFFFu, wd[3], src > 0 ? src - 1 : 0);
          if (wq == 1) wp = x0;
          if (wq == 2) wp = x1;
          if (wq == 3) wp = x2;
          if (wq == 0 && src == 0 && d > 0) {
            uint64_t pw[4];
            philox4x64_10((uint64_t)(d / 4 - 1), 0ULL, 0ULL, 0ULL, seed, (uint64_t)k, pw);
            wp = pw[3];
          }
          const u128 vk = scheme == kSchemeSystematic ? vsys : draw_fixed<true>(word);
          const u128 vp = scheme == kSchemeSystematic ? vsys : draw_fixed<true>(wp);
          f[r] = d < Nk ? strata_spacing(d, Nk, vk, vp) : u128{0ULL, 0ULL};
        }
        inc[r] = warp_incl_scan_v(f[r], lane);
        const u128 t = shfl_v(inc[r], 31);
        inc[r] = u128_add(inc[r], wtot);  // plus the earlier rounds of this warp
        wtot = u128_add(wtot, t);
      }
      u128 ctot;
      const u128 woff = block_excl_scan<kWarps>(lane == 0 ? wtot : u128{0ULL, 0ULL}, sm.wsum, ctot);
      const u128 base = u128_add(carry, shfl_v(woff, 0));
      carry = u128_add(carry, ctot);
#pragma unroll 1
      for (int r = 0; r < 4; ++r) {
        const long long i = wbase + 32 * r + lane;  // sample index (Z_{i+1})
        const bool valid = i < Nk;
        if (!__any_sync(0xFFFFFFFFu, valid)) break;
        const u128 key = map_key(c, u128_add(base, inc[r]));
        // last segment with P_s < key (P_0 = 0 < key)
        int s_me = 0;
        if (valid) {
          int lo = 0, hi = (int)nseg;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (u128_lt(sm.pre[mid], key)) lo = mid + 1;
            else hi = mid;
          }
          s_me = lo > 0 ? lo - 1 : 0;
        }
        unsigned pend = __ballot_sync(0xFFFFFFFFu, valid);
        while (pend) {
          const int sc = __shfl_sync(0xFFFFFFFFu, s_me, __ffs(pend) - 1);
          const unsigned grp = __ballot_sync(0xFFFFFFFFu, valid && s_me == sc) & pend;
          const bool mine = (grp >> lane) & 1u;
          Bits b[kSegV];
          if (vec) load_seg_blocked<float, true>(wk, (long long)sc * kSeg, Mk, lane, b);
          else load_seg_blocked<float, false>(wk, (long long)sc * kSeg, Mk, lane, b);
          const uint32_t E = (uint32_t)sm.E[sc];
          uint64_t pref[kSegV];
          seg_prefixes<float>(b, E, lane, pref);
          unsigned long long Kq = 0;
          if (mine) {
            const u128 Ps = sm.pre[sc];
            const u128 rem = u128_lt(Ps, key) ? u128_sub(key, Ps) : u128{0ULL, 0ULL};
            Kq = ceil_units(rem, (int)E - Emax + kGridHead, sm.F[sc]);
          }
          int cnt = 0;
          if (__popc(grp) <= leaf_T) {
            unsigned g = grp;
            while (g) {
              const int j = __ffs(g) - 1;
              g &= g - 1;
              const unsigned long long Kj = __shfl_sync(0xFFFFFFFFu, Kq, j);
              int cj = 0;
#pragma unroll
              for (int q = 0; q < kSegV; ++q) cj += pref[q] < Kj ? 1 : 0;
#pragma unroll
              for (int o = 16; o; o >>= 1) cj += __shfl_xor_sync(0xFFFFFFFFu, cj, o);
              if (lane == j) cnt = cj;
            }
          } else {
            unsigned long long* sp = sm.pref[warp];
#pragma unroll
            for (int q = 0; q < kSegV; ++q) sp[lane * kSegV + q] = pref[q];
            __syncwarp();
            if (mine) {  // number of prefixes below K (they are non-decreasing)
              int lo = 0, hi = kSeg;
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sp[mid] < Kq) lo = mid + 1;
                else hi = mid;
              }
              cnt = lo;
            }
            __syncwarp();
          }
          if (mine) {
            const long long rem_len = Mk - (long long)sc * kSeg;
            const int len = (int)(rem_len < kSeg ? rem_len : kSeg);
            const int j = cnt < len ? cnt : len - 1;
            long long idx = (long long)sc * kSeg + j;
            if (idx > Mk - 1) idx = Mk - 1;
            outk[i] = (int)idx;
          }
          pend &= ~grp;
        }
      }
    }
  }
}

template <int kThreads>
static cudaError_t batched_t(const float* w, const long long* w_off, const long long* r_off, const int* order, int K,
                             unsigned long long seed, int leaf_T, int* out, unsigned* queue, int* status,
                             cudaStream_t st, int scheme) {
  const size_t smem = sizeof(BatchSmem<kThreads / 32>);
  cudaError_t e = cudaFuncSetAttribute(k_batched_f32<kThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched_f32<kThreads>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  long long blocks = (long long)num_sms() * per_sm;
  if (blocks > K) blocks = K;
  if (blocks < 1) blocks = 1;
  k_batched_f32<kThreads><<<(unsigned)blocks, kThreads, smem, st>>>(w, w_off, r_off, order, K, seed, leaf_T, out,
                                                                     queue, status, scheme);
  return cudaGetLastError();
}

cudaError_t launch_batched_f32(const float* w, const long long* w_off, const long long* r_off, const int* order, int K,
                               unsigned long long seed, int threads, int leaf_T, int* out, unsigned* queue,
                               int* status, cudaStream_t st, int scheme) {
  if (K <= 0) return cudaSuccess;
  switch (threads) {
    case 128: return batched_t<128>(w, w_off, r_off, order, K, seed, leaf_T, out, queue, status, st, scheme);
    case 512: return batched_t<512>(w, w_off, r_off, order, K, seed, leaf_T, out, queue, status, st, scheme);
    default: return batched_t<256>(w, w_off, r_off, order, K, seed, leaf_T, out, queue, status, st, scheme);
  }
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
