// Helpers of the CTA-pair (cta_group::2) tcgen05 kernels: cluster rank and shared-memory
// mapping, arrivals on the leader CTA's barriers, cluster barriers, TMA loads that signal a
// barrier of either CTA of the pair, and MMA commits multicast to both CTAs.
#pragma once
#include "tcgen05.cuh"

namespace ipc {
namespace tc {

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address of the same shared-memory offset in the cluster's CTA `rank`.
__device__ __forceinline__ uint32_t peer_addr(uint32_t addr, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(addr), "r"(rank));
  return d;
}

// Arrive on a barrier of the leader CTA: local for the leader's own warps, through the cluster
// window for the peer's. The arrive only says that the warp's TMEM columns were read and reset:
// tcgen05.wait::st and tcgen05.fence::before_thread_sync already order those stores, so the
// default (CTA-scope) release suffices and no cluster-wide fence is paid on every drain.
__device__ __forceinline__ void arrive_leader(uint32_t bar, bool leader) {
  if (leader) {
    mbar_arrive(bar);
  } else {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(remote) : "r"(bar));
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
  }
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA tile load into this CTA's shared memory whose completion is counted on `bar`, a barrier
// in either CTA of the pair.
__device__ __forceinline__ void tma_load_pair(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// D (+)= A B on the pair (issued by the leader CTA only); idesc carries M = 256.
__device__ __forceinline__ void umma_pair_desc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(1u)
      : "memory");
}

// Arrives on the barrier at this offset in both CTAs once every MMA issued so far has completed.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          bar),
      "h"(static_cast<uint16_t>(3))
      : "memory");
}

}  // namespace tc
}  // namespace ipc
