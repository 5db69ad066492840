// Last step of the log-domain pattern build (steps 1-3 of Sec. II.B), one
// position j at a time.  The digit convolutions conv[j][t] (exact integers
// below p) recombine into S(j) = sum_{z in R} log_3(1 - r^(z-j)) mod p-1, and
// with log_3 r^j = j * 65536/n:
//   j received:  log A'(r^j) = j(k-1) * 65536/n + S(j), weight
//                c_j = -r^-j / A'(r^j) = -3^-(log r^j + log A'(r^j)),
//   j erased:    log A(r^j)  = jk * 65536/n + S(j),
// and ahat_j = n^-1 (A(r^j) - r^(jk)) = n^-1 FNT(A mod x^k)_j (A(r^j) = 0 for
// received j), or A(r^j) itself (aval) when the step-6 product is split.
#pragma once
#include <stdint.h>

#include "field.cuh"

namespace fntrs {

struct LogFinal {
  const uint32_t* conv;  // [n][D]
  int D, b, n, k;
  const uint32_t* exp3;  // 3^e, e < 65536
  uint32_t ninv;
  uint2* pat;       // .x = received row (0xFFFFFFFF: erased), .y = weight (written)
  uint32_t* pat32;  // (row << 17) | weight, 0 for erased positions
  uint32_t* aval;   // A(r^j) or null
  uint32_t* ahat;   // n^-1 FNT(A mod x^k) or null
  uint32_t* rowtab = nullptr;  // (j << 17) | weight at index row, or null
};

// exp3 index of position j: the weight's exponent (received) or log A(r^j) (erased)
__device__ __forceinline__ uint32_t lg_exp_index(const LogFinal& f, int j, uint32_t row,
                                                 uint32_t S) {
  const uint32_t jl = (uint32_t)j * (65536u / (uint32_t)f.n);  // log_3 r^j
  if (row != 0xFFFFFFFFu) {
    const uint32_t ld = (jl * (uint32_t)(f.k - 1) + S) & 0xFFFFu;  // log A'(r^j)
    return (0u - (jl + ld)) & 0xFFFFu;  // c = -3^-(log r^j + log A'(r^j))
  }
  return (jl * (uint32_t)f.k + S) & 0xFFFFu;
}

// exp3 index of r^(jk)
__device__ __forceinline__ uint32_t lg_rjk_index(const LogFinal& f, int j) {
  return ((uint32_t)j * (65536u / (uint32_t)f.n) * (uint32_t)f.k) & 0xFFFFu;
}

// x = exp3[lg_exp_index], rjk = exp3[lg_rjk_index]
__device__ __forceinline__ void lg_store(const LogFinal& f, int j, uint32_t row, uint32_t x,
                                         uint32_t rjk) {
  uint32_t A = 0u;
  if (row != 0xFFFFFFFFu) {
    const uint32_t c = kP - x;
    f.pat[j].y = c;
    f.pat32[j] = (row << 17) | c;
    if (f.rowtab) f.rowtab[row] = ((uint32_t)j << 17) | c;
  } else {
    f.pat32[j] = 0u;
    A = x;
  }
  if (f.aval) f.aval[j] = A;
  if (f.ahat) f.ahat[j] = p_mul(m_to_p(m_sub(A, rjk)), f.ninv);
}

// S(j) from the digit convolutions, read through L2 (they may come from other
// CTAs of the same launch)
__device__ __forceinline__ uint32_t lg_digits(const LogFinal& f, int j) {
  uint32_t S = 0u;
  for (int t = 0; t < f.D; ++t) S += __ldcg(f.conv + (size_t)j * f.D + t) << (f.b * t);
  return S;
}

// One position; `row` = pat[j].x as read by the caller.
__device__ __forceinline__ void lg_final_one(const LogFinal& f, int j, uint32_t row) {
  const uint32_t x = __ldg(f.exp3 + lg_exp_index(f, j, row, lg_digits(f, j)));
  lg_store(f, j, row, x, f.ahat ? __ldg(f.exp3 + lg_rjk_index(f, j)) : 0u);
}

// All L positions by one CTA of NT threads, loads batched per thread (at
// most 16 positions per thread per round).
template <int L, int NT>
__device__ __forceinline__ void lg_final_block(const LogFinal& f) {
  constexpr int PJ = (L + NT - 1) / NT < 16 ? (L + NT - 1) / NT : 16;
  for (int base = 0; base < L; base += PJ * NT) {
    uint32_t row[PJ], x[PJ], r[PJ];
#pragma unroll
    for (int u = 0; u < PJ; ++u) {
      const int j = base + (int)threadIdx.x + u * NT;
      row[u] = j < L ? __ldcg(&f.pat[j].x) : 0xFFFFFFFFu;
      x[u] = 0u;
    }
    // digit-major so that each round has PJ independent loads in flight
    for (int t = 0; t < f.D; ++t) {
#pragma unroll
      for (int u = 0; u < PJ; ++u) {
        const int j = base + (int)threadIdx.x + u * NT;
        if (j < L) x[u] += __ldcg(f.conv + (size_t)j * f.D + t) << (f.b * t);
      }
    }
#pragma unroll
    for (int u = 0; u < PJ; ++u) {
      const int j = base + (int)threadIdx.x + u * NT;
      if (j < L) {
        r[u] = f.ahat ? __ldg(f.exp3 + lg_rjk_index(f, j)) : 0u;
        x[u] = __ldg(f.exp3 + lg_exp_index(f, j, row[u], x[u]));
      }
    }
#pragma unroll
    for (int u = 0; u < PJ; ++u) {
      const int j = base + (int)threadIdx.x + u * NT;
      if (j < L) lg_store(f, j, row[u], x[u], r[u]);
    }
  }
}

}  // namespace fntrs
