// TMA-staged encode of n = 2L with k > L (a code of rate above 1/2).
//
// The FNT of the zero-padded source of length n = 2L splits into two output
// classes of length-L transforms (Sec. II.B: e_j = s(r^j)): class 0 (even j)
// transforms x_i = s_i + s_(i+L), class 1 (odd j) transforms
// x_i = (s_i - s_(i+L)) r_n^i, i < L (r_n^L = -1).  k_encode_tma holds one
// class's input in a [L][8] tile when k <= L; for k > L the source tile is
// [k][8] and the class inputs fold two rows.  The staged tile keeps 8
// codewords (a 16-byte TMA row of u16), and the transforms run on 4 of them
// at a time so that the staged rows (up to 128 KB) and the work array (64 KB)
// fit in one SM's shared memory.  Tiles are taken over by cluster launch
// control as in k_encode_tma; all waits are bounded.
#pragma once
#include "kernels.cuh"

namespace fntrs {

template <class S, int NT>
__global__ void __launch_bounds__(NT, 1)
    k_encode_tma_fold(KArgs a, const uint32_t* __restrict__ twc, int rows_staged, int box_rows,
                      const __grid_constant__ CUtensorMap tsrc) {
  dbg_enter(a.status);
  static_assert(S::NP == 3 || S::NP == 2, "");
  static_assert(2 * S::R1 <= 32, "class-1 pass-1 factors must be rotations");
  constexpr int WS = 8, WT = 4, C = 2;  // staged / transformed codewords per tile
  using Y = Lay<S, WT>;
  constexpr int R = S::R1, SP = S::S1, B = ilog2(R), L = S::L;
  constexpr int WORK_BYTES = ((Y::WORDS * 4) + 127) / 128 * 128;
  extern __shared__ __align__(128) uint4 smem_raw[];
  uint32_t* work = reinterpret_cast<uint32_t*>(smem_raw);
  uint16_t* stage = reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(smem_raw) + WORK_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(stage) +
                                              (size_t)rows_staged * WS * 2);
  uint64_t* cbar = bar + 1;
  uint4* resp = reinterpret_cast<uint4*>(bar + 2);
  __shared__ int s_next;
  const int ntiles = (a.W + WS - 1) / WS;
  const int nbox = rows_staged / box_rows;
  const uint32_t tx_bytes = (uint32_t)rows_staged * WS * 2;
  int tile = blockIdx.x;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(cbar, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && tile < ntiles) {
    mbar_expect_tx(bar, tx_bytes);
    for (int bx = 0; bx < nbox; ++bx)
      tma_load_2d(stage + (size_t)bx * box_rows * WS, &tsrc, tile * WS, bx * box_rows, bar);
    clc_request(resp, cbar);
  }
  uint32_t parity = 0, cphase = 0;
  bool pending = tile < ntiles;  // thread 0: a cancel request is outstanding
  uint32_t* out = static_cast<uint32_t*>(a.out);
  const size_t ld = a.ld_out;
  while (tile < ntiles) {
    const bool ok = mbar_wait(bar, parity);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(a.status, ST_TIMEOUT);
        mbar_wait(bar, parity);  // let the copy in flight land before exiting
        if (pending) mbar_wait(cbar, cphase);
      }
      return;
    }
    parity ^= 1u;
#pragma unroll 1
    for (int h = 0; h < WS / WT; ++h) {
      const int col0 = tile * WS + h * WT;
#pragma unroll 1
      for (int cc = 0; cc < C; ++cc) {
        // pass 1 from the staged source, two rows folded per input
        for (int t = threadIdx.x; t < (L / R) * WT; t += NT) {
          const int c = t % WT, i2 = t / WT, cs = h * WT + c;
          uint32_t x[R];
#pragma unroll
          for (int q = 0; q < R; ++q) {
            const int row = q * SP + i2;  // < L <= rows_staged
            const uint32_t v = stage[row * WS + cs];
            const uint32_t u = row + L < rows_staged ? (uint32_t)stage[(row + L) * WS + cs] : 0u;
            x[q] = cc == 0 ? v + u : m_sub(v, u);  // rows >= k are zero (TMA fill)
          }
          if (cc == 1) {
            constexpr int e = Pow2Root<(2 * R > 32 ? 32 : 2 * R)>::e;
#pragma unroll
            for (int q = 1; q < R; ++q) x[q] = m_rot_rt(x[q], (uint32_t)(e * q));
          }
          dft_reg<R, false>(x);
          if (cc == 1) {
            const uint4* tw4 = reinterpret_cast<const uint4*>(twc + i2 * R);
#pragma unroll
            for (int q = 0; q < R; q += 4) {
              const uint4 w = __ldg(tw4 + q / 4);
              x[q] = m_mul(x[q], w.x);
              x[q + 1] = m_mul(x[q + 1], w.y);
              x[q + 2] = m_mul(x[q + 2], w.z);
              x[q + 3] = m_mul(x[q + 3], w.w);
            }
          } else {
            twiddle_regs<R>(x, a.twf + i2 * R);
          }
          uint32_t* base = work + Y::addr(i2, c);
#pragma unroll
          for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::P1_STRIDE] = x[q];
        }
        __syncthreads();
        if (h == WS / WT - 1 && cc == C - 1 && threadIdx.x == 0) {
          // the stage is free: take over a pending CTA's tile and prefetch it
          int nxt = clc_take(resp, cbar, cphase);
          pending = false;
          if (nxt == kClcTimeout) atomicOr(a.status, ST_TIMEOUT);
          if (nxt >= 0 && nxt < ntiles) {
            fence_proxy_async();
            mbar_expect_tx(bar, tx_bytes);
            for (int bx = 0; bx < nbox; ++bx)
              tma_load_2d(stage + (size_t)bx * box_rows * WS, &tsrc, nxt * WS, bx * box_rows,
                          bar);
            clc_request(resp, cbar);
            pending = true;
          } else {
            nxt = ntiles;
          }
          s_next = nxt;
        }
        if constexpr (S::NP == 3) {
          dif_mid<S, WT, NT, false>(work, a.twf + S::TW2_OFF);
          __syncthreads();
        }
        // last pass -> encoded rows cc + C*j
        {
          constexpr int RL = S::RL, BL = ilog2(RL);
          for (int t = threadIdx.x; t < (L / RL) * WT; t += NT) {
            const int c = t % WT, b = t / WT;
            const uint32_t* base = work + b * Y::LAST_B + c;
            uint32_t x[RL];
#pragma unroll
            for (int q = 0; q < RL; ++q) x[q] = base[q * WT];
            dft_reg<RL, false>(x);
            const int col = col0 + c;
            if (col < a.W) {
              uint32_t* o = out + (size_t)(cc + C * S::natural(b * RL)) * ld + col;
              const size_t step = (size_t)C * (L / RL) * ld;
#pragma unroll
              for (int q = 0; q < RL; ++q) o[bitrev(q, BL) * step] = m_to_p(x[q]);
            }
          }
        }
        __syncthreads();
      }
    }
    tile = s_next;
  }
}

}  // namespace fntrs
