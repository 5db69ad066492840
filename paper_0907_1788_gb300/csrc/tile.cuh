// In-shared-memory batched FNT engine.
//
// A CTA transforms WT codewords of length L at once.  The length-L transform
// (the FNT of Sec. II.A/II.B: A_j = sum_i a_i r^(ij)) is factored as
// L = R1 * R2 * R3 (each radix <= 32, so every in-pass root is a power of two
// and its products are rotations, see field.cuh).  One pass = every thread
// loads the R values of a group into registers, runs a radix-R DFT there,
// applies the inter-pass twiddles and writes back in place.  Decimation in
// frequency (DIF) reads natural order and leaves the spectrum in
// digit-reversed "slot" order; the transposed decimation-in-time (DIT) pass
// sequence reads slot order and produces natural order.
//
// Slot layout after DIF pass p:  slot = j1*S1 + j2*S2 + j3   (S3 = 1)
// holds spectrum index          j    = j1 + R1*j2 + R1*R2*j3.
//
// Shared memory holds [slot][codeword] u32 with WT words of padding after
// every block of RL slots (RL = radix of the last pass).  A warp touches
// 32/WT consecutive slots of one block in every pass but the last, and 32/WT
// consecutive blocks in the last; the padding staggers those blocks across
// banks, and every per-register offset within a pass is a compile-time
// constant.
#pragma once
#include "dbg.cuh"
#include "field.cuh"

namespace fntrs {

template <int L_, int R1_, int R2_ = 1, int R3_ = 1>
struct Sched {
  static constexpr int L = L_, R1 = R1_, R2 = R2_, R3 = R3_;
  static_assert(R1 * R2 * R3 == L, "radices must multiply to L");
  static constexpr int NP = (R3 > 1) ? 3 : ((R2 > 1) ? 2 : 1);
  static constexpr int S1 = L / R1;
  static constexpr int S2 = (NP == 3) ? S1 / R2 : 1;
  static constexpr int RL = (NP == 3) ? R3 : ((NP == 2) ? R2 : R1);  // radix of last pass
  // twiddle tables (entries): pass 1 -> L entries, pass 2 (3-pass only) -> S1 entries
  static constexpr int TW2_OFF = L;
  static constexpr int TW_ENTRIES = (NP == 1) ? 0 : (L + ((NP == 3) ? S1 : 0));

  // spectrum index held by a slot in digit-reversed layout
  static __device__ __forceinline__ int natural(int slot) {
    if constexpr (NP == 1) {
      return slot;
    } else if constexpr (NP == 2) {
      return slot / S1 + R1 * (slot % S1);
    } else {
      const int j1 = slot / S1, rem = slot % S1;
      return j1 + R1 * (rem / S2) + R1 * R2 * (rem % S2);
    }
  }
  // the slot holding spectrum index j (the inverse of natural)
  static __device__ __forceinline__ int slot_of(int j) {
    if constexpr (NP == 1) {
      return j;
    } else if constexpr (NP == 2) {
      return (j % R1) * S1 + j / R1;
    } else {
      return (j % R1) * S1 + ((j / R1) % R2) * S2 + j / (R1 * R2);
    }
  }
};

// Padded shared-memory layout of one [L][WT] buffer.
template <class S, int WT>
struct Lay {
  static constexpr int PADW = WT < 32 ? WT : 0;
  static constexpr int LB = ilog2(S::RL);
  static constexpr int WORDS = S::L * WT + (S::L / S::RL) * PADW;
  static __device__ __forceinline__ int addr(int slot, int c) {
    return slot * WT + (slot >> LB) * PADW + c;
  }
  // pass 1: slot = q*S1 + i2
  static constexpr int P1_STRIDE = S::S1 * WT + (S::S1 >> LB) * PADW;
  // middle pass of 3: slot = b*S1 + q*S2 + i2 (S2 = RL)
  static constexpr int MID_B = P1_STRIDE;
  static constexpr int MID_STRIDE = S::S2 * WT + (S::S2 >> LB) * PADW;
  // last pass: slot = b*RL + q
  static constexpr int LAST_B = S::RL * WT + PADW;
};

template <class S, int WT>
constexpr int smem_words() {
  return S::NP >= 2 ? Lay<S, WT>::WORDS : 0;
}

// multiply register q by table entry q (table entry 0 is always 1: skipped)
template <int R>
__device__ __forceinline__ void twiddle_regs(uint32_t* x, const uint32_t* __restrict__ tw) {
  if constexpr (R >= 4) {
#pragma unroll
    for (int q = 0; q < R; q += 4) {
      const uint4 w = __ldg(reinterpret_cast<const uint4*>(tw + q));
      if (q != 0) x[q] = m_mul(x[q], w.x);
      x[q + 1] = m_mul(x[q + 1], w.y);
      x[q + 2] = m_mul(x[q + 2], w.z);
      x[q + 3] = m_mul(x[q + 3], w.w);
    }
  } else {
#pragma unroll
    for (int q = 1; q < R; ++q) x[q] = m_mul(x[q], __ldg(tw + q));
  }
}

// The same from a row of a table copied to shared memory with its 16-byte
// chunks permuted (chunk u of row i2 at chunk u ^ (i2 mod R/4)).
template <int R>
__device__ __forceinline__ void twiddle_regs_sw(uint32_t* x, const uint32_t* row, int i2) {
  static_assert(R >= 4, "");
  const int m = i2 & (R / 4 - 1);
#pragma unroll
  for (int u = 0; u < R / 4; ++u) {
    const uint4 w = reinterpret_cast<const uint4*>(row)[u ^ m];
    if (u != 0) x[4 * u] = m_mul(x[4 * u], w.x);
    x[4 * u + 1] = m_mul(x[4 * u + 1], w.y);
    x[4 * u + 2] = m_mul(x[4 * u + 2], w.z);
    x[4 * u + 3] = m_mul(x[4 * u + 3], w.w);
  }
}

// x_nat[j] = x[bitrev(j)]  (DIF output order -> natural, or the reverse)
template <int R>
__device__ __forceinline__ void bitrev_regs(uint32_t* x) {
  constexpr int B = ilog2(R);
  uint32_t y[R];
#pragma unroll
  for (int j = 0; j < R; ++j) y[j] = x[bitrev(j, B)];
#pragma unroll
  for (int j = 0; j < R; ++j) x[j] = y[j];
}

// CTA-wide barriers of the pass sequences: every thread of the CTA, or only
// the first N (named barrier 15), when the CTA has other warps (a TMA
// producer) that never take part.
struct CtaSync {
  static __device__ __forceinline__ void sync() { __syncthreads(); }
};
template <int N>
struct FirstSync {
  static_assert(N % 32 == 0, "");
  static __device__ __forceinline__ void sync() {
    asm volatile("bar.sync 15, %0;" ::"n"(N) : "memory");
  }
};

// ---------------------------------------------------------------------------
// Barrier between the middle pass and the last pass of a 3-pass schedule (in
// either direction).  With R2 = RL both passes give the S1 slots of one middle
// block b to the same G = (S1 / R2) * WT consecutive tasks, and task t runs on
// thread t mod NT; when G is a multiple of the warp size that divides NT, the
// threads that write a block are the threads that read it, so only their
// group of G threads (thread index / G) has to meet: one warp (syncwarp) or a
// named barrier of G threads (ids 1..NT/G; id 0 is __syncthreads, 15 FirstSync).  Otherwise
// the whole CTA (Sync) meets.
// ---------------------------------------------------------------------------
template <class S, int WT, int NT, class Sync = CtaSync>
__device__ __forceinline__ void mid_last_sync() {
  constexpr int G = (S::NP == 3) ? (S::S1 / S::R2) * WT : 0;
  if constexpr (S::NP == 3 && S::R2 == S::RL && G % 32 == 0 && G > 0 && NT % G == 0 &&
                NT / G <= 14) {  // ids 1..14 (15: FirstSync)
    if constexpr (G == 32) {
      __syncwarp();
    } else {
      const int id = 1 + (int)threadIdx.x / G;
      asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(G) : "memory");
    }
  } else {
    Sync::sync();
  }
}

// ---------------------------------------------------------------------------
// Pass building blocks.  Task loops run over (group g, codeword c), c fastest.
// ---------------------------------------------------------------------------

// DIF pass 1: natural-order input from a loader -> slots (or, for 1-pass
// schedules, straight to the storer).
//   load(i, c) -> value of input element i (0 <= i < L) of codeword c
//   store(j, c, v) for 1-pass schedules: spectrum index j
template <class S, int WT, int NT, bool INV, class Load, class Store>
__device__ __forceinline__ void dif_first(uint32_t* sm, const uint32_t* __restrict__ tw, Load& load,
                                          Store& store) {
  using Y = Lay<S, WT>;
  constexpr int R = S::R1, SP = S::S1, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, i2 = t / WT;
    if constexpr (kDebugBounds && S::NP >= 2) {
      if (!dbg_in(Y::addr(i2, c) + (R - 1) * Y::P1_STRIDE, Y::WORDS) ||
          !dbg_in(i2 * R + R - 1, S::L))
        continue;
    }
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = load(q * SP + i2, c);
    dft_reg<R, INV>(x);
    if constexpr (S::NP == 1) {
#pragma unroll
      for (int q = 0; q < R; ++q) store(bitrev(q, B), c, x[q]);
    } else {
      twiddle_regs<R>(x, tw + i2 * R);
      uint32_t* base = sm + Y::addr(i2, c);
#pragma unroll
      for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::P1_STRIDE] = x[q];
    }
  }
}

// DIF pass 1 in place: input element i of codeword c at the natural-order
// address Lay::addr(i, c).  Task (i2, c) reads i = q*S1 + i2 (q < R1) and
// writes the slots bitrev(q)*S1 + i2, the same addresses (S1 is a multiple of
// the last radix, so addr(q*S1 + i2) = addr(i2) + q*P1_STRIDE).
template <class S, int WT, int NT, bool INV>
__device__ __forceinline__ void dif_first_inplace(uint32_t* sm, const uint32_t* __restrict__ tw) {
  static_assert(S::NP >= 2 && S::S1 % S::RL == 0, "");
  using Y = Lay<S, WT>;
  constexpr int R = S::R1, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, i2 = t / WT;
    if (!dbg_in(Y::addr(i2, c) + (R - 1) * Y::P1_STRIDE, Y::WORDS)) continue;
    uint32_t* base = sm + Y::addr(i2, c);
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[q * Y::P1_STRIDE];
    dft_reg<R, INV>(x);
    twiddle_regs<R>(x, tw + i2 * R);
#pragma unroll
    for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::P1_STRIDE] = x[q];
  }
}

// DIF pass 2 of a 3-pass schedule, slots -> slots.
template <class S, int WT, int NT, bool INV>
__device__ __forceinline__ void dif_mid(uint32_t* sm, const uint32_t* __restrict__ tw2) {
  using Y = Lay<S, WT>;
  constexpr int R = S::R2, SP = S::S2, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, g = t / WT;
    const int b = g / SP, i2 = g % SP;
    if (!dbg_in(b * Y::MID_B + Y::addr(i2, c) + (R - 1) * Y::MID_STRIDE, Y::WORDS) ||
        !dbg_in(i2 * R + R - 1, S::S1))
      continue;
    uint32_t* base = sm + b * Y::MID_B + Y::addr(i2, c);
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[q * Y::MID_STRIDE];
    dft_reg<R, INV>(x);
    twiddle_regs<R>(x, tw2 + i2 * R);
#pragma unroll
    for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::MID_STRIDE] = x[q];
  }
}

// Last DIF pass: slots -> storer, store(j, c, v) with j the spectrum index.
template <class S, int WT, int NT, bool INV, bool LOWER, class Store>
__device__ __forceinline__ void dif_last_sel(uint32_t* sm, Store& store) {
  static_assert(S::NP >= 2, "");
  using Y = Lay<S, WT>;
  constexpr int R = S::RL, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, b = t / WT;
    if (!dbg_in(b * Y::LAST_B + c + (R - 1) * WT, Y::WORDS)) continue;
    const uint32_t* base = sm + b * Y::LAST_B + c;
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[q * WT];
    dft_reg<R, INV>(x);
    const int j0 = S::natural(b * R);
#pragma unroll
    for (int q = 0; q < R; ++q)
      if (!LOWER || (q & 1) == 0) store(j0 + (S::L / R) * bitrev(q, B), c, x[q]);
  }
}

template <class S, int WT, int NT, bool INV, class Store>
// LOWER: only spectrum indices j < L/2 are wanted (register q holds
// j = j0 + (L/R) bitrev(q) with j0 < L/R, so those are the even q); the
// others are neither computed nor stored.
__device__ __forceinline__ void dif_last(uint32_t* sm, Store& store) {
  dif_last_sel<S, WT, NT, INV, false>(sm, store);
}

// Last DIF pass writing back into the slots: spectrum index j (slot b*R +
// bitrev(q)) reduced to [0, p) when j < k, and zero otherwise (LOWER: k = L/2,
// the even registers; the odd ones are not computed).
template <class S, int WT, int NT, bool INV, bool LOWER>
__device__ __forceinline__ void dif_last_reduce(uint32_t* sm, int k) {
  static_assert(S::NP >= 2, "");
  using Y = Lay<S, WT>;
  constexpr int R = S::RL, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, b = t / WT;
    if (!dbg_in(b * Y::LAST_B + c + (R - 1) * WT, Y::WORDS)) continue;
    uint32_t* base = sm + b * Y::LAST_B + c;
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[q * WT];
    dft_reg<R, INV>(x);
    const int j0 = S::natural(b * R);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const bool keep = LOWER ? (q & 1) == 0 : j0 + (S::L / R) * bitrev(q, B) < k;
      base[bitrev(q, B) * WT] = keep ? m_to_p(x[q]) : 0u;
    }
  }
}

// Last DIF pass writing back into the slots (for a following DIT sequence).
template <class S, int WT, int NT, bool INV>
__device__ __forceinline__ void dif_last_inplace(uint32_t* sm) {
  static_assert(S::NP >= 2, "");
  using Y = Lay<S, WT>;
  constexpr int R = S::RL, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, b = t / WT;
    if (!dbg_in(b * Y::LAST_B + c + (R - 1) * WT, Y::WORDS)) continue;
    uint32_t* base = sm + b * Y::LAST_B + c;
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[q * WT];
    dft_reg<R, INV>(x);
    // register q holds spectrum digit bitrev(q): slot b*R + bitrev(q)
#pragma unroll
    for (int q = 0; q < R; ++q) base[bitrev(q, B) * WT] = x[q];
  }
}

// DIT pass 2 of a 3-pass schedule (transposed DIF pass 2), slots -> slots.
template <class S, int WT, int NT, bool INV>
__device__ __forceinline__ void dit_mid(uint32_t* sm, const uint32_t* __restrict__ tw2) {
  using Y = Lay<S, WT>;
  constexpr int R = S::R2, SP = S::S2, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, g = t / WT;
    const int b = g / SP, i2 = g % SP;
    if (!dbg_in(b * Y::MID_B + Y::addr(i2, c) + (R - 1) * Y::MID_STRIDE, Y::WORDS) ||
        !dbg_in(i2 * R + R - 1, S::S1))
      continue;
    uint32_t* base = sm + b * Y::MID_B + Y::addr(i2, c);
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[bitrev(q, B) * Y::MID_STRIDE];
    twiddle_regs<R>(x, tw2 + i2 * R);
    bitrev_regs<R>(x);
    dft_reg<R, INV>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::MID_STRIDE] = x[q];
  }
}

// DIT pass 1 (transposed DIF pass 1): slots -> natural order, handed to
// store(i, c, v) with i the natural index.
template <class S, int WT, int NT, bool INV, class Store>
__device__ __forceinline__ void dit_first(uint32_t* sm, const uint32_t* __restrict__ tw,
                                          Store& store) {
  static_assert(S::NP >= 2, "");
  using Y = Lay<S, WT>;
  constexpr int R = S::R1, SP = S::S1, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, i2 = t / WT;
    if (!dbg_in(Y::addr(i2, c) + (R - 1) * Y::P1_STRIDE, Y::WORDS) ||
        !dbg_in(i2 * R + R - 1, S::L))
      continue;
    const uint32_t* base = sm + Y::addr(i2, c);
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[bitrev(q, B) * Y::P1_STRIDE];
    twiddle_regs<R>(x, tw + i2 * R);
    bitrev_regs<R>(x);
    dft_reg<R, INV>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) store(bitrev(q, B) * SP + i2, c, x[q]);
  }
}

// DIT last-group pass (the transpose of the last DIF pass) reading slots,
// optionally multiplied by a second buffer slot-wise first, writing slots.
template <class S, int WT, int NT, bool INV, bool MUL2>
__device__ __forceinline__ void dit_last_inplace(uint32_t* sm, const uint32_t* sm2) {
  static_assert(S::NP >= 2, "");
  using Y = Lay<S, WT>;
  constexpr int R = S::RL, B = ilog2(R);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, b = t / WT;
    const int off = b * Y::LAST_B + c;
    if (!dbg_in(off + (R - 1) * WT, Y::WORDS)) continue;
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int a = off + q * WT;
      x[q] = MUL2 ? m_mul(sm[a], m_to_p(sm2[a])) : sm[a];
    }
    dft_reg<R, INV>(x);
#pragma unroll
    for (int q = 0; q < R; ++q) sm[off + bitrev(q, B) * WT] = x[q];
  }
}

}  // namespace fntrs
