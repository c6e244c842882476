// Thread-block cluster helpers (a cluster of CTAs on distinct SMs that
// exchange values through distributed shared memory).
#pragma once
#include "common.cuh"

namespace gbr {

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster; orders the shared-memory
// writes before it against the other CTAs' reads after it.
__device__ __forceinline__ void cluster_sync_all() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The u128 at the same shared-memory offset as p in CTA `rank` of the cluster.
__device__ __forceinline__ u128 ld_cluster_u128(const u128* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  unsigned long long lo, hi;
  asm volatile("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(lo), "=l"(hi) : "r"(ra) : "memory");
  return u128{lo, hi};
}

}  // namespace gbr
