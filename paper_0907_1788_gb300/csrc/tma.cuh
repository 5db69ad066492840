// TMA (cp.async.bulk.tensor) and mbarrier helpers, inline PTX for sm_103a.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include <cuda/ptx>

namespace fntrs {

// Upper bound on mbarrier polls before a wait gives up (the kernel then
// reports ST_TIMEOUT instead of spinning forever).
constexpr uint32_t kWaitPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// one arrival without transaction bytes (release: this thread's earlier
// shared-memory writes are seen by whoever completes a wait on the phase)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// OR of `v` over the first N threads of the CTA (named barrier 15, as FirstSync)
template <int N>
__device__ __forceinline__ bool first_sync_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 15, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(N)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// order this thread's earlier shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled TMA load of one box at element coordinates (x, y) into shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Untiled bulk copy global -> shared of `bytes` (a multiple of 16; both
// addresses 16-byte aligned), completing its bytes on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Asynchronous global -> shared copy of BYTES (4, 8 or 16) bytes of which the
// first `valid` are read and the rest zero-filled (cp.async, LDGSTS).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int valid) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src),
               "n"(BYTES), "r"(valid)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// waits for all of this thread's committed copies (a barrier then publishes them)
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Cluster launch control (sm_100 and later).  The TMA kernels are launched
// with one CTA per tile; a running CTA asks the hardware to cancel the launch
// of a CTA of the same grid that has not started yet and then processes that
// CTA's tile itself (prefetching it while it finishes the current one).  Every
// tile is thus processed exactly once, by its own CTA if that CTA is launched
// or else by the CTA whose request cancelled it, and CTAs that start late
// (the SM was busy with another kernel) simply take fewer tiles.  After a
// request that cancelled nothing, no further request is made.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void clc_request(uint4* resp, uint64_t* bar) {
  cuda::ptx::clusterlaunchcontrol_try_cancel(resp, bar);
  mbar_expect_tx(bar, 16);
}

constexpr int kClcNone = -1;     // the request cancelled nothing
constexpr int kClcTimeout = -2;  // the response did not arrive within the bound

// Waits for the outstanding request (phase `phase` of `bar`) and returns the
// x index of the cancelled CTA, kClcNone or kClcTimeout.
__device__ __forceinline__ int clc_take(const uint4* resp, uint64_t* bar, uint32_t& phase) {
  if (!mbar_wait(bar, phase)) return kClcTimeout;
  phase ^= 1u;
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "r"(smem_u32(resp))
               : "memory");
  if (!cuda::ptx::clusterlaunchcontrol_query_cancel_is_canceled(r)) return kClcNone;
  return (int)cuda::ptx::clusterlaunchcontrol_query_cancel_get_first_ctaid_x<uint32_t>(r);
}

// Shared-memory bytes after a TMA kernel's stage: the TMA barrier, the
// cancel barrier, (the decode's stage-empty barrier,) the 16-byte cancel
// response at byte 32.
constexpr int kSchedBytes = 64;

}  // namespace fntrs
