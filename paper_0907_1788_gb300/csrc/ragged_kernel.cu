// The ragged persistent kernel: one launch runs the encode tiles, pattern
// builds and decode tiles of every group with n >= 256 in a ragged batch.
// CTAs stay resident and take work items in list order from an atomic
// counter; the list puts the spectrum items first, then all encode and
// pattern items, then the decode items (every spectrum item before the digit
// items that read it), so an item only ever waits (boundedly) on items that
// running CTAs already hold, and every wait ends.  Data written by other CTAs of the same
// launch (encoded rows, pattern tables, spectra) is read through L2 only.
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
using SLoc = SchedFor<kLocalL>::type;
constexpr int WL = kRaggedSplitWT;
static_assert(WL == wt_one(kLocalL), "a split item is one local tile wide");

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

// ---------------------------------------------------------------------------
// Split transforms run by one CTA over the columns of one work item (x.W <=
// WL): the radix-C cross pass into the CTA's scratch x.out2, then the C local
// 4096-point passes, each a tile transform whose output goes where x.mode
// says (kargs.h).  The same arithmetic as the standalone cross and local
// kernels; the global scratch is written and read by this CTA only, between
// CTA barriers.
// ---------------------------------------------------------------------------
// U (i2, column) pairs per thread at a time: the loads of the U groups are
// independent, so a thread keeps U * C loads in flight (one CTA per SM has to
// cover the memory latency of the whole pass by itself).
template <int C, bool INV, int LOADM>
__device__ __noinline__ void cta_cross(const KArgs& x) {
  constexpr int U = C <= 8 ? 4 : 2;
  uint32_t bad = 0u;
  const int total = x.L * x.W;
  int t = threadIdx.x;
  for (; t + (U - 1) * NT < total; t += U * NT) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int tu = t + u * NT;
      cross_one<C, INV, LOADM, true>(x, tu / x.W, tu % x.W, bad);
    }
  }
  for (; t < total; t += NT) cross_one<C, INV, LOADM, true>(x, t / x.W, t % x.W, bad);
  if (bad) atomicOr(x.status, ST_RANGE);
}

__device__ void cross_rt(const KArgs& x, bool inv, int lm) {
  if (x.C == 16) {
    if (!inv && lm == CL_SRC16) cta_cross<16, false, CL_SRC16>(x);
    else if (inv && lm == CL_RECV) cta_cross<16, true, CL_RECV>(x);
    else if (inv) cta_cross<16, true, CL_U32>(x);
    else cta_cross<16, false, CL_U32>(x);
  } else {  // C = 8
    if (!inv && lm == CL_SRC16) cta_cross<8, false, CL_SRC16>(x);
    else if (inv && lm == CL_RECV) cta_cross<8, true, CL_RECV>(x);
    else if (inv) cta_cross<8, true, CL_U32>(x);
    else cta_cross<8, false, CL_U32>(x);
  }
  __syncthreads();
}

// MODE < 0: the output mode is read at run time (x.mode; the rarer modes share
// one body per direction); the frequent ones have bodies of their own.
template <bool INV, int MODE>
__device__ __noinline__ void cta_local(const KArgs& x) {
  for (int j1 = 0; j1 < x.C; ++j1) {
    if constexpr (MODE < 0)
      tile_body<SLoc, WL, NT, INV, LoadRows32<WL>, StoreLocalRT<WL, true>>(x, 0, j1);
    else
      tile_body<SLoc, WL, NT, INV, LoadRows32<WL>, StoreLocal<WL, MODE>>(x, 0, j1);
    __syncthreads();
  }
}

__device__ void local_rt(const KArgs& x, bool inv) {
  if (!inv && x.mode == LM_ENC) cta_local<false, LM_ENC>(x);
  else if (inv && x.mode == LM_OUT16) cta_local<true, LM_OUT16>(x);
  else if (inv) cta_local<true, -1>(x);
  else cta_local<false, -1>(x);
}

// The C local passes of one transform, each fused with the next transform's
// cross DFTs (local_cross_last): reads x.in (rows j1 * 4096 + i), writes the
// next transform's cross output to x.out2.  which = 0: D1 local (inverse),
// truncation at x.row_limit, D2 cross (forward); which = 1: D2 local (forward)
// * ahat, D3 cross (inverse).
template <int C, int WHICH>
__device__ __noinline__ void cta_local_cross(const KArgs& x) {
  constexpr bool INV_LOCAL = WHICH == 0, INV_CROSS = WHICH == 1, AHAT = WHICH == 1;
  extern __shared__ uint4 smem_raw[];
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw);
  const uint32_t* tw = INV_LOCAL ? x.twi : x.twf;
  for (int j1 = 0; j1 < C; ++j1) {
    LoadRows32<WL> load = LoadRows32<WL>::make(x, 0, j1);
    NopStore nop;
    dif_first<SLoc, WL, NT, INV_LOCAL>(sm, tw, load, nop);
    __syncthreads();
    dif_mid<SLoc, WL, NT, INV_LOCAL>(sm, tw + SLoc::TW2_OFF);
    mid_last_sync<SLoc, WL, NT>();
    local_cross_last<SLoc, WL, NT, INV_LOCAL, C, INV_CROSS, AHAT, true>(sm, x, j1, 0);
    __syncthreads();
  }
}

__device__ void local_cross_rt(const KArgs& x, int which) {
  if (x.C == 16) {
    if (which == 0) cta_local_cross<16, 0>(x);
    else cta_local_cross<16, 1>(x);
  } else {
    if (which == 0) cta_local_cross<8, 0>(x);
    else cta_local_cross<8, 1>(x);
  }
}

// Encode of columns [tile*WL, +WL) of a long code (Sec. II.B: e = FNT of the
// zero-padded source), split as n = C * 4096.
__device__ void split_encode(const RaggedGroupDev& g, int tile, uint32_t* scr) {
  KArgs c = g.xenc;
  const int c0 = tile * WL;
  c.W = min(WL, g.enc.W - c0);
  c.in = static_cast<const uint16_t*>(g.enc.in) + c0;
  c.ld_in = g.enc.ld_in;
  c.out = static_cast<uint32_t*>(g.enc.out) + c0;
  c.ld_out = g.enc.ld_out;
  c.out2 = scr;
  c.ld_work = (size_t)c.W;
  c.row_limit = g.enc.k;
  cross_rt(c, false, CL_SRC16);
  KArgs x = c;
  x.in = scr;
  x.ld_in = (size_t)c.W;
  x.mode = LM_ENC;
  local_rt(x, false);
}

// Decode (steps 4-6 of Sec. II.B) of columns [tile*WL, +WL) of a long code,
// the same pass sequence as the standalone split decode: k <= n/2 in 6
// passes, k > n/2 (product split at h = n/2) in 10.
__device__ void split_decode(const RaggedGroupDev& g, int tile, uint32_t* scr) {
  const int n = g.L, k = g.dec.k, h = n / 2;
  const int c0 = tile * WL;
  const int w = min(WL, g.dec.W - c0);
  KArgs c = g.xdec;
  c.W = w;
  c.ld_work = (size_t)w;
  c.out = static_cast<uint16_t*>(g.dec.out) + c0;
  c.ld_out = g.dec.ld_out;
  const uint32_t* recv = static_cast<const uint32_t*>(g.dec.in) + c0;
  const size_t nw = (size_t)n * w;
  uint32_t* A = scr;
  uint32_t* B0 = A + nw;
  uint32_t* B1 = B0 + nw;
  uint32_t* B2 = B1 + nw;
  auto cross = [&](bool inv, int lm, const void* in, size_t ld_in, int row_limit) {
    KArgs x = c;
    x.in = in;
    x.ld_in = ld_in;
    x.row_limit = row_limit;
    x.out2 = A;
    cross_rt(x, inv, lm);
  };
  auto local = [&](bool inv, int mode, void* o2, void* o3, int out_limit, const void* in2) {
    KArgs x = c;
    x.in = A;
    x.ld_in = (size_t)w;
    x.out2 = o2;
    x.out3 = o3;
    x.in2 = in2;
    x.out_limit = out_limit;
    x.mode = mode;
    local_rt(x, inv);
  };
  // a local pass fused with the next transform's cross pass (4 passes, not 6)
  auto local_cross = [&](int which, const uint32_t* in, uint32_t* o2, int row_limit) {
    KArgs x = c;
    x.in = in;
    x.ld_in = (size_t)w;
    x.out2 = o2;
    x.row_limit = row_limit;
    local_cross_rt(x, which);
  };
  if (!g.blocked) {
    cross(true, CL_RECV, recv, g.dec.ld_in, n);
    local_cross(0, A, B0, k);
    local_cross(1, B0, A, n);
    local(true, LM_OUT16, nullptr, nullptr, k, nullptr);
  } else {
    cross(true, CL_RECV, recv, g.dec.ld_in, n);
    local(true, LM_SPLIT, B0, B1, k, nullptr);
    cross(false, CL_U32, B0, (size_t)w, h);
    local(false, LM_X_PARTIAL, B0, B2, n, nullptr);
    cross(false, CL_U32, B1, (size_t)w, k - h);
    local(false, LM_ACCUM, nullptr, B2, n, nullptr);
    cross(true, CL_U32, B2, (size_t)w, n);
    local(true, LM_WORK, B1, nullptr, n, nullptr);
    cross(true, CL_U32, B0, (size_t)w, n);
    local(true, LM_OUT16_ADD, nullptr, nullptr, k, B1);
  }
}

// ---------------------------------------------------------------------------
// Pattern build of a long code (n >= 32768), the log-domain route of the
// one-launch build with its transforms over global scratch: one transform of
// a column (or two) of length L, as a one-CTA tile (L <= 32768) or split
// (L = 65536).  base = the group's colf / coli (tables, n, L, C).
// ---------------------------------------------------------------------------
template <int L, bool INV>
__device__ __noinline__ void col_fnt(const KArgs& base, const uint32_t* in, size_t ld_in,
                                     uint32_t* out, size_t ld_out, int W, uint32_t scale,
                                     uint32_t* scr) {
  KArgs x = base;
  x.in = in;
  x.ld_in = ld_in;
  x.out = out;
  x.ld_out = ld_out;
  x.W = W;
  x.scale = scale;
  if constexpr (L <= kTileMaxL) {
    constexpr int WT = wt_one(L);
    for (int tx = 0; tx * WT < W; ++tx) {
      tile_body<RS<L>, WT, NT, INV, LoadRows32<WT>, StoreRows32<WT>>(x, tx, 0);
      __syncthreads();
    }
  } else {
    x.row_limit = L;
    x.out2 = scr;
    x.ld_work = (size_t)W;
    cross_rt(x, INV, CL_U32);
    KArgs y = x;
    y.in = scr;
    y.ld_in = (size_t)W;
    y.mode = LM_FNT;
    local_rt(y, INV);
  }
}

// The spectrum item: position table rows, then spec = FNT(1_R).
template <int L>
__device__ __noinline__ void rg_spec(const RaggedGroupDev& g, unsigned* done, uint32_t* scr) {
  const LongPlanDev& lp = g.lp;
  const int k = g.dec.k;
  for (int z = threadIdx.x; z < L; z += NT) lp.ind[z] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += NT) lp.ind[__ldg(g.plan.pos + i)] = (uint32_t)i + 1u;
  __syncthreads();
  for (int z = threadIdx.x; z < L; z += NT) {
    const uint32_t r = lp.ind[z];
    g.plan.pat[z] = make_uint2(r ? r - 1u : 0xFFFFFFFFu, 0u);
    lp.ind[z] = r ? 1u : 0u;
  }
  __syncthreads();
  col_fnt<L, false>(g.colf, lp.ind, 1, lp.spec, 1, 1, 1u, scr);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(done, 1u);
}

// Digit t: conv[.][t] = n^-1 IFNT(spec * ghat[.][t]).  The last digit item of
// the group recombines the digits into the tables (and, for k > n/2, the
// transforms of the two halves of A mod x^k); returns true in that CTA.
template <int L>
__device__ __noinline__ bool rg_digit(const RaggedGroupDev& g, int t, uint32_t* scr) {
  __shared__ int s_last;
  const LongPlanDev& lp = g.lp;
  const PlanArgs& pa = g.plan;
  uint32_t* pr = lp.prod + (size_t)t * L;
  for (int j = threadIdx.x; j < L; j += NT)
    pr[j] = m_mul(__ldg(pa.ghat + (size_t)j * pa.D + t), __ldcg(lp.spec + j));
  __syncthreads();
  col_fnt<L, true>(g.coli, pr, 1, pa.conv + t, (size_t)pa.D, 1, pa.ninv, scr);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(pa.done, 1u) == (uint32_t)pa.D - 1u;
  __syncthreads();
  const bool last = s_last;
  __syncthreads();  // s_last is rewritten by the next digit this CTA runs
  if (!last) return false;
  __threadfence();
  const int k = g.dec.k;
  const LogFinal f{pa.conv, pa.D,     pa.b,    L,       k,        pa.exp3,
                   pa.ninv, pa.pat, pa.pat32, pa.aval, pa.ahat, pa.rowtab};
  lg_final_block<L, NT>(f);
  if (g.blocked) {
    __syncthreads();
    constexpr int H = L / 2;
    col_fnt<L, true>(g.coli, lp.aval, 1, lp.coef, 1, 1, pa.ninv, scr);
    for (int j = threadIdx.x; j < L; j += NT) {
      uint32_t a0 = 0u, a1 = 0u;
      if (k == L) {
        a0 = j == 0 ? kP - 1u : 0u;  // A = x^n - 1, A mod x^n = -1
      } else {
        if (j < H) a0 = lp.coef[j];
        if (j < k - H) a1 = lp.coef[H + j];
      }
      lp.M2[2 * j] = a0;
      lp.M2[2 * j + 1] = a1;
    }
    __syncthreads();
    col_fnt<L, false>(g.colf, lp.M2, 2, lp.E2, 2, 2, 1u, scr);
    uint32_t* ahat = const_cast<uint32_t*>(g.dec.ahat);
    uint32_t* ahat2 = const_cast<uint32_t*>(g.dec.ahat2);
    for (int j = threadIdx.x; j < L; j += NT) {
      ahat[j] = p_mul(lp.E2[2 * j], pa.ninv);
      ahat2[j] = p_mul(lp.E2[2 * j + 1], pa.ninv);
    }
  }
  if (threadIdx.x == 0) *pa.done = 0u;
  return true;
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

// tile bodies: every length up to 32768 (pattern builds in one launch up to 16384)
#define FNTRS_RAGGED_SWITCH(L, CALL) \
  switch (L) {                       \
    case 256: CALL(256); break;      \
    case 512: CALL(512); break;      \
    case 1024: CALL(1024); break;    \
    case 2048: CALL(2048); break;    \
    case 4096: CALL(4096); break;    \
    case 8192: CALL(8192); break;    \
    case 16384: CALL(16384); break;  \
    case 32768: CALL(32768); break;  \
    default: break;                  \
  }
#define FNTRS_RAGGED_SWITCH_FUSED(L, CALL) \
  switch (L) {                             \
    case 256: CALL(256); break;            \
    case 512: CALL(512); break;            \
    case 1024: CALL(1024); break;          \
    case 2048: CALL(2048); break;          \
    case 4096: CALL(4096); break;          \
    case 8192: CALL(8192); break;          \
    case 16384: CALL(16384); break;        \
    default: break;                        \
  }
#define FNTRS_RAGGED_SWITCH_LONG(L, CALL) \
  switch (L) {                            \
    case 32768: CALL(32768); break;       \
    case 65536: CALL(65536); break;       \
    default: break;                       \
  }

__global__ void __launch_bounds__(NT, 1) k_ragged(RaggedArgs ra) {
  __shared__ int s_item, s_ok;
  uint32_t* scr = ra.cta_scratch ? ra.cta_scratch + (size_t)blockIdx.x * ra.cta_words : nullptr;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(ra.next, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= ra.nitems) return;
    const RaggedItem item = ra.items[it];
    const RaggedGroupDev& g = ra.groups[item.group];
    const int L = g.L;
    dbg_enter(g.enc.status ? g.enc.status : g.dec.status);
    if (item.kind == RI_ENC) {
      if (g.split_enc) {
        split_encode(g, item.tile, scr);
      } else {
#define FNTRS_CALL(X) rg_encode<X>(g.enc, item.tile)
        FNTRS_RAGGED_SWITCH_FUSED(L, FNTRS_CALL)  // tile encodes: n <= 16384
#undef FNTRS_CALL
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(ra.enc_done + item.group, 1u);
    } else if (item.kind == RI_SPEC) {
#define FNTRS_CALL(X) rg_spec<X>(g, ra.spec_done + item.group, scr)
      FNTRS_RAGGED_SWITCH_LONG(L, FNTRS_CALL)
#undef FNTRS_CALL
    } else if (item.kind == RI_PLAN) {
      bool last = false;
      if (g.long_plan) {
        if (threadIdx.x == 0) {
          const bool ok = wait_at_least(ra.spec_done + item.group, 1u);
          if (!ok) atomicOr(g.dec.status, ST_TIMEOUT);
          __threadfence();
          s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
#define FNTRS_CALL(X) last = rg_digit<X>(g, item.tile, scr)
          FNTRS_RAGGED_SWITCH_LONG(L, FNTRS_CALL)
#undef FNTRS_CALL
        }
      } else {
#define FNTRS_CALL(X) last = rg_plan<X>(g.plan, item.tile)
        FNTRS_RAGGED_SWITCH_FUSED(L, FNTRS_CALL)
#undef FNTRS_CALL
        if (last && g.blocked) {
          __syncthreads();
#define FNTRS_CALL(X) rg_plan_tail<X>(g)
          FNTRS_RAGGED_SWITCH_FUSED(L, FNTRS_CALL)
#undef FNTRS_CALL
        }
      }
      if (last) {
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
        if (g.split_dec) {
          split_decode(g, item.tile, scr);
        } else if (g.blocked) {
#define FNTRS_CALL(X) rg_decode_split<X>(g.dec, item.tile)
          FNTRS_RAGGED_SWITCH_FUSED(L, FNTRS_CALL)
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
  const int two = L <= 16384 ? 2 * smem_words<S, wt_two(L)>() : 0;
  const int plan = L <= 16384 ? Lay<S, 1>::WORDS + L : 0;
  return std::max(one, std::max(two, plan));
}

}  // namespace

int ragged_smem_bytes() {
  const int w = std::max({body_smem_words<256>(), body_smem_words<512>(), body_smem_words<1024>(),
                          body_smem_words<2048>(), body_smem_words<4096>(),
                          body_smem_words<8192>(), body_smem_words<16384>(),
                          body_smem_words<32768>(), smem_words<SLoc, WL>()});
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
    case 16384: return wt_one(16384);
    case 32768: return kRaggedSplitWT;
    case 65536: return kRaggedSplitWT;
    default: return 0;
  }
}

int ragged_wt_dec(int L, bool blocked) {
  if (ragged_split_dec(L, blocked)) return kRaggedSplitWT;
  if (!blocked) {  // the one-CTA tile bodies (the encode of 32768 is split, this decode not)
    switch (L) {
      case 256: return wt_one(256);
      case 512: return wt_one(512);
      case 1024: return wt_one(1024);
      case 2048: return wt_one(2048);
      case 4096: return wt_one(4096);
      case 8192: return wt_one(8192);
      case 16384: return wt_one(16384);
      case 32768: return wt_one(32768);
      default: return 0;
    }
  }
  switch (L) {
    case 256: return wt_two(256);
    case 512: return wt_two(512);
    case 1024: return wt_two(1024);
    case 2048: return wt_two(2048);
    case 4096: return wt_two(4096);
    case 8192: return wt_two(8192);
    case 16384: return wt_two(16384);
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
