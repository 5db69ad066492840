// The ragged persistent kernel: one launch runs the encode tiles, pattern
// builds and decode tiles of every group with 256 <= n <= 8192 in a
// ragged batch.  CTAs stay resident and take work items in list order from an
// atomic counter; the list puts all encode and pattern items before the
// decode items, so a decode item only ever waits (boundedly) on items that
// running CTAs already hold, and the wait always ends.
#include <cuda_runtime.h>

#include <algorithm>

#include "inst.cuh"
#include "ragged_dev.h"
#include "tma.cuh"

namespace fntrs {
namespace {

template <int L>
using RS = typename SchedFor<L>::type;
constexpr int NT = kRaggedNT;

template <int L>
__device__ __noinline__ void rg_encode(const KArgs& a, int tx) {
  constexpr int W = wt_one(L);
  tile_body<RS<L>, W, NT, false, LoadSrcFold<W>, StoreRows32<W>>(a, tx, 0);
}

template <int L>
__device__ __noinline__ void rg_decode(const KArgs& a, int tx) {
  decode_body<RS<L>, wt_one(L), NT, true>(a, tx);
}

template <int L>
__device__ __noinline__ void rg_decode_split(const KArgs& a, int tx) {
  decode_split_body<RS<L>, wt_two(L), NT, true>(a, tx);
}

template <int L>
__device__ __noinline__ bool rg_plan(const PlanArgs& pa, int t) {
  return plan_body<RS<L>, NT>(pa, t);
}

// k > n/2: the step-6 product is split at h = n/2, so the tables are the
// transforms of the two halves of A mod x^k (as the host-side build does):
// coefficients = n^-1 IFNT(A(r^j)), halves, FNT of both, n^-1 scaling.
template <int L>
__device__ __noinline__ void rg_plan_tail(const RaggedGroupDev& g) {
  constexpr int W = wt_one(L), H = L / 2;
  tile_body<RS<L>, W, NT, true, LoadRows32<W>, StoreRows32<W>>(g.tail_inv, 0, 0);
  __syncthreads();
  const uint32_t* coef = static_cast<const uint32_t*>(g.tail_inv.out);
  const int k = g.dec.k;
  for (int j = threadIdx.x; j < L; j += NT) {
    uint32_t a0 = 0u, a1 = 0u;
    if (k == L) {
      a0 = j == 0 ? kP - 1u : 0u;  // A = x^n - 1, A mod x^n = -1
    } else {
      if (j < H) a0 = coef[j];
      if (j < k - H) a1 = coef[H + j];
    }
    g.halves[2 * j] = a0;
    g.halves[2 * j + 1] = a1;
  }
  __syncthreads();
  tile_body<RS<L>, W, NT, false, LoadRows32<W>, StoreRows32<W>>(g.tail_fwd, 0, 0);
  __syncthreads();
  const uint32_t* E = static_cast<const uint32_t*>(g.tail_fwd.out);
  uint32_t* ahat = const_cast<uint32_t*>(g.dec.ahat);
  uint32_t* ahat2 = const_cast<uint32_t*>(g.dec.ahat2);
  for (int j = threadIdx.x; j < L; j += NT) {
    ahat[j] = p_mul(E[2 * j], g.plan.ninv);
    ahat2[j] = p_mul(E[2 * j + 1], g.plan.ninv);
  }
}

// Bounded wait until *p >= target; false if the bound ran out.
__device__ __forceinline__ bool wait_at_least(const unsigned* p, unsigned target) {
  for (uint32_t i = 0; i < kWaitPolls; ++i) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= target) return true;
    __nanosleep(64);
  }
  return false;
}

#define FNTRS_RAGGED_SWITCH(L, CALL) \
  switch (L) {                       \
    case 256: CALL(256); break;      \
    case 512: CALL(512); break;      \
    case 1024: CALL(1024); break;    \
    case 2048: CALL(2048); break;    \
    case 4096: CALL(4096); break;    \
    case 8192: CALL(8192); break;    \
    default: break;                  \
  }

__global__ void __launch_bounds__(NT, 1) k_ragged(RaggedArgs ra) {
  __shared__ int s_item, s_ok;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(ra.next, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= ra.nitems) return;
    const RaggedItem item = ra.items[it];
    const RaggedGroupDev& g = ra.groups[item.group];
    const int L = g.L;
    if (item.kind == RI_ENC) {
#define FNTRS_CALL(X) rg_encode<X>(g.enc, item.tile)
      FNTRS_RAGGED_SWITCH(L, FNTRS_CALL)
#undef FNTRS_CALL
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(ra.enc_done + item.group, 1u);
    } else if (item.kind == RI_PLAN) {
      bool last = false;
#define FNTRS_CALL(X) last = rg_plan<X>(g.plan, item.tile)
      FNTRS_RAGGED_SWITCH(L, FNTRS_CALL)
#undef FNTRS_CALL
      if (last) {
        if (g.blocked) {
          __syncthreads();
#define FNTRS_CALL(X) rg_plan_tail<X>(g)
          FNTRS_RAGGED_SWITCH(L, FNTRS_CALL)
#undef FNTRS_CALL
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicExch(ra.plan_done + item.group, 1u);
      }
    } else {
      if (threadIdx.x == 0) {
        const bool ok = wait_at_least(ra.enc_done + item.group, (unsigned)g.enc_need) &&
                        (!g.has_plan || wait_at_least(ra.plan_done + item.group, 1u));
        if (!ok) atomicOr(g.dec.status, ST_TIMEOUT);
        __threadfence();
        s_ok = ok;
      }
      __syncthreads();
      if (s_ok) {
        if (g.blocked) {
#define FNTRS_CALL(X) rg_decode_split<X>(g.dec, item.tile)
          FNTRS_RAGGED_SWITCH(L, FNTRS_CALL)
#undef FNTRS_CALL
        } else {
#define FNTRS_CALL(X) rg_decode<X>(g.dec, item.tile)
          FNTRS_RAGGED_SWITCH(L, FNTRS_CALL)
#undef FNTRS_CALL
        }
      }
    }
    __syncthreads();
  }
}

template <int L>
constexpr int body_smem_words() {
  using S = RS<L>;
  const int one = smem_words<S, wt_one(L)>();
  const int two = 2 * smem_words<S, wt_two(L)>();
  const int plan = Lay<S, 1>::WORDS + L;
  return std::max(one, std::max(two, plan));
}

}  // namespace

int ragged_smem_bytes() {
  const int w = std::max({body_smem_words<256>(), body_smem_words<512>(), body_smem_words<1024>(),
                          body_smem_words<2048>(), body_smem_words<4096>(),
                          body_smem_words<8192>()});
  return w * 4;
}

int ragged_wt_enc(int L) {
  switch (L) {
    case 256: return wt_one(256);
    case 512: return wt_one(512);
    case 1024: return wt_one(1024);
    case 2048: return wt_one(2048);
    case 4096: return wt_one(4096);
    case 8192: return wt_one(8192);
    default: return 0;
  }
}

int ragged_wt_dec(int L, bool blocked) {
  if (!blocked) return ragged_wt_enc(L);
  switch (L) {
    case 256: return wt_two(256);
    case 512: return wt_two(512);
    case 1024: return wt_two(1024);
    case 2048: return wt_two(2048);
    case 4096: return wt_two(4096);
    case 8192: return wt_two(8192);
    default: return 0;
  }
}

int launch_ragged(const RaggedArgs& ra, int grid, cudaStream_t st) {
  const int smem = ragged_smem_bytes();
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    if (cudaFuncSetAttribute(k_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return -1;
    done[dev & 63] = true;
  }
  k_ragged<<<grid, NT, smem, st>>>(ra);
  count_launch();
  return 0;
}

}  // namespace fntrs
