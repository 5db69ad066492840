// Per-erasure-pattern preparation on the device (Sec. II.B, steps 1-3).
// Two routes compute the same tables: the log-domain correlation below
// (default: a handful of batched FNTs) and the paper's product tree:
//   step 1  A(x) = prod_{i<k} (x - r^(z_i)) by a product tree: leaves are
//           multiplied 32 at a time in registers, then pairs of nodes with
//           FNT products level by level ("M(n) = 3 FNTs");
//   step 2  A'(x), coefficient (i+1) A_(i+1);
//   step 3  A'(r^j) for all j at once by one FNT_n (r has order n, so the
//           evaluation on the geometric progression 1, r, .., r^(n-1) is the
//           transform itself);
// then the weights c_i = -r^(-z_i) / A'(r^(z_i)) used by step 4 (they fold
// the sign and the index shift of step 5's power series into the scatter),
// and the transform of A mod x^k used by step 6.
#include <cuda_runtime.h>

#include "field.cuh"
#include "kargs.h"
#include "logplan.cuh"

namespace fntrs {

void count_launch();

namespace {

constexpr int kLeaf = 32;

__global__ void k_pat_init(uint2* pat, int n) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n) pat[z] = make_uint2(0xFFFFFFFFu, 0u);
}

// nodes of degree <= 32: out[m][j] = coefficient m of prod_{i in node j} (x - x_i)
__global__ void k_leaves(const uint32_t* __restrict__ pos, int k,
                         const uint32_t* __restrict__ powf, uint32_t* __restrict__ out, int nodes) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nodes) return;
  uint32_t c[kLeaf + 1];
#pragma unroll
  for (int m = 0; m <= kLeaf; ++m) c[m] = m == 0 ? 1u : 0u;
#pragma unroll
  for (int t = 0; t < kLeaf; ++t) {
    const int i = j * kLeaf + t;
    if (i < k) {
      const uint32_t x = __ldg(powf + pos[i]);
#pragma unroll
      for (int m = kLeaf; m >= 1; --m) c[m] = m_sub(c[m - 1], m_mul(c[m], x));
      c[0] = m_sub(0u, m_mul(c[0], x));
    }
  }
#pragma unroll
  for (int m = 0; m <= kLeaf; ++m) out[(size_t)m * nodes + j] = m_to_p(c[m]);
}

// Big product-tree level (L = 2d > tile limit): pack both children of every
// pair as columns 2p, 2p+1 of an [L][2*npairs] matrix (missing right child = 1).
__global__ void k_big_pack(const uint32_t* __restrict__ lvl, int d, int nodes, int L,
                           uint32_t* __restrict__ M) {
  const int npairs = (nodes + 1) / 2, cols = 2 * npairs;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)L * cols) return;
  const int col = (int)(t % cols), i = (int)(t / cols);
  uint32_t v = 0u;
  if (col < nodes) {
    if (i <= d) v = lvl[(size_t)i * nodes + col];
  } else if (i == 0) {
    v = 1u;  // missing right sibling
  }
  M[t] = v;
}

// Q[i][p] = M^[i][2p] * M^[i][2p+1]
__global__ void k_big_mul(const uint32_t* __restrict__ Mh, int npairs, int L,
                          uint32_t* __restrict__ Q) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)L * npairs) return;
  const int p = (int)(t % npairs), i = (int)(t / npairs);
  const size_t r = (size_t)i * 2 * npairs;
  Q[t] = m_to_p(m_mul(Mh[r + 2 * p], Mh[r + 2 * p + 1]));
}

// products (already scaled, in [0,p)) -> next level [L+1][npairs] with the wrap fix
__global__ void k_big_fix(const uint32_t* __restrict__ Q, int d, int k, int npairs, int L,
                          uint32_t* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)(L + 1) * npairs) return;
  const int p = (int)(t % npairs), i = (int)(t / npairs);
  const bool full = (long long)k >= (long long)(2 * p + 2) * d;
  uint32_t v;
  if (i == L) {
    v = full ? 1u : 0u;
  } else {
    v = Q[(size_t)i * npairs + p];
    if (i == 0 && full) v = v == 0u ? 65536u : v - 1u;
  }
  out[t] = v;
}

// Columns of M [n][ncols]: 0 -> A' coefficients, 1 -> A mod x^k (or A0),
// 2 -> A1 (coefficients h..k-1 of A) when the product is split at h.
__global__ void k_pat_prep(const uint32_t* __restrict__ A, int k, int n, int ncols, int h,
                           uint32_t* __restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t dA = 0u;
  if (i < k) dA = p_mul((uint32_t)((i + 1) % kP), A[i + 1]);
  M[(size_t)i * ncols + 0] = dA;
  if (ncols == 2) {
    M[(size_t)i * ncols + 1] = i < k ? A[i] : 0u;
  } else {
    M[(size_t)i * ncols + 1] = i < h ? A[i] : 0u;
    M[(size_t)i * ncols + 2] = (i < k - h) ? A[h + i] : 0u;
  }
}

// pattern table and step-6 tables from E = FNT_n(M)
__global__ void k_pat_final(const uint32_t* __restrict__ E, int ncols, const uint32_t* __restrict__ pos,
                            int k, int n, const uint32_t* __restrict__ powi, uint32_t ninv,
                            uint2* __restrict__ pat, uint32_t* __restrict__ ahat,
                            uint32_t* __restrict__ ahat2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < k) {
    const uint32_t z = pos[t];
    const uint32_t dAx = E[(size_t)z * ncols + 0];  // A'(r^z)
    const uint32_t inv = p_inv(dAx);
    // c = -r^-z / A'(r^z)
    const uint32_t c = m_to_p(m_sub(0u, m_mul(inv, __ldg(powi + z))));
    pat[z] = make_uint2((uint32_t)t, c);
  }
  if (t < n) {
    ahat[t] = p_mul(E[(size_t)t * ncols + 1], ninv);
    if (ncols == 3) ahat2[t] = p_mul(E[(size_t)t * ncols + 2], ninv);
  }
}

// ---------------------------------------------------------------------------
// Log-domain pattern build.  With g[d] = log_3(1 - r^d) (d != 0), g[0] = 0 and
// S(j) = sum_{z in R} g[z - j] (a cyclic correlation of the indicator 1_R):
//   j not received:  log A(r^j)  = j*k*(65536/n)     + S(j)   (mod 65536)
//   j received:      log A'(r^j) = j*(k-1)*(65536/n) + S(j)
// because r^j - r^z = r^j (1 - r^(z-j)).  S is computed exactly as a sum of
// D digit-wise cyclic convolutions over F_p (each digit < 2^b with
// k (2^b - 1) < p, so no convolution value wraps).
// ---------------------------------------------------------------------------

__global__ void k_lg_init(uint2* pat, uint32_t* ind, int n) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n) {
    pat[z] = make_uint2(0xFFFFFFFFu, 0u);
    ind[z] = 0u;
  }
}

__global__ void k_lg_scatter(const uint32_t* __restrict__ pos, int k, uint2* pat, uint32_t* ind) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) {
    const uint32_t z = pos[i];
    ind[z] = 1u;
    pat[z].x = (uint32_t)i;
  }
}

// P[j][t] = spec[j] * Ghat[j][t]
__global__ void k_lg_mul(const uint32_t* __restrict__ spec, const uint32_t* __restrict__ ghat,
                         int D, int n, uint32_t* __restrict__ P) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * D) return;
  const int j = (int)(t / D);
  P[t] = m_to_p(m_mul(ghat[t], m_to_p(spec[j])));
}

// weights of received positions; A(r^j) of the others (aval) and, unless the
// step-6 product is split, ahat_j = n^-1 (A(r^j) - r^(jk)) = n^-1 FNT(A mod x^k)_j.
__global__ void k_lg_final(LogFinal f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < f.n) lg_final_one(f, j, f.pat[j].x);
}

// coefficient halves of A (k > n/2): M[j][0] = A_j (j < h), M[j][1] = A_(h+j) (j < k-h);
// k = n means A = x^n - 1, A mod x^n = -1.
__global__ void k_lg_halves(const uint32_t* __restrict__ coef, int n, int k, uint32_t* M) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int h = n / 2;
  uint32_t a0 = 0u, a1 = 0u;
  if (k == n) {
    a0 = j == 0 ? kP - 1u : 0u;
  } else {
    if (j < h) a0 = coef[j];
    if (j < k - h) a1 = coef[h + j];
  }
  M[(size_t)j * 2] = a0;
  M[(size_t)j * 2 + 1] = a1;
}

__global__ void k_lg_scale2(const uint32_t* __restrict__ E, int n, uint32_t ninv,
                            uint32_t* __restrict__ ahat, uint32_t* __restrict__ ahat2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  ahat[j] = p_mul(E[(size_t)j * 2], ninv);
  ahat2[j] = p_mul(E[(size_t)j * 2 + 1], ninv);
}

// compact per-position entry (row << 17) | weight for the staged decode, and
// the per-row entry (position << 17) | weight of each received row
__global__ void k_pat32(const uint2* __restrict__ pat, uint32_t* __restrict__ pat32,
                        uint32_t* __restrict__ rowtab, int n) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < n) {
    const uint2 e = pat[z];
    pat32[z] = e.y ? ((e.x << 17) | e.y) : 0u;
    if (e.y && rowtab && e.x < (uint32_t)n) rowtab[e.x] = ((uint32_t)z << 17) | e.y;
  }
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_pat32(const uint2* pat, uint32_t* pat32, uint32_t* rowtab, int n, cudaStream_t st) {
  k_pat32<<<blocks_for(n, 256), 256, 0, st>>>(pat, pat32, rowtab, n);
  count_launch();
}

void launch_lg_init(uint2* pat, uint32_t* ind, int n, cudaStream_t st) {
  k_lg_init<<<blocks_for(n, 256), 256, 0, st>>>(pat, ind, n);
  count_launch();
}
void launch_lg_scatter(const uint32_t* pos, int k, uint2* pat, uint32_t* ind, cudaStream_t st) {
  k_lg_scatter<<<blocks_for(k, 256), 256, 0, st>>>(pos, k, pat, ind);
  count_launch();
}
void launch_lg_mul(const uint32_t* spec, const uint32_t* ghat, int D, int n, uint32_t* P,
                   cudaStream_t st) {
  k_lg_mul<<<blocks_for((long long)n * D, 256), 256, 0, st>>>(spec, ghat, D, n, P);
  count_launch();
}
void launch_lg_final(const uint32_t* conv, int D, int b, int n, int k, const uint32_t* exp3,
                     uint32_t ninv, uint2* pat, uint32_t* pat32, uint32_t* aval, uint32_t* ahat,
                     uint32_t* rowtab, cudaStream_t st) {
  const LogFinal f{conv, D, b, n, k, exp3, ninv, pat, pat32, aval, ahat, rowtab};
  k_lg_final<<<blocks_for(n, 256), 256, 0, st>>>(f);
  count_launch();
}
void launch_lg_halves(const uint32_t* coef, int n, int k, uint32_t* M, cudaStream_t st) {
  k_lg_halves<<<blocks_for(n, 256), 256, 0, st>>>(coef, n, k, M);
  count_launch();
}
void launch_lg_scale2(const uint32_t* E, int n, uint32_t ninv, uint32_t* ahat, uint32_t* ahat2,
                      cudaStream_t st) {
  k_lg_scale2<<<blocks_for(n, 256), 256, 0, st>>>(E, n, ninv, ahat, ahat2);
  count_launch();
}

void launch_pat_init(uint2* pat, int n, cudaStream_t st) {  // product-tree route
  k_pat_init<<<blocks_for(n, 256), 256, 0, st>>>(pat, n);
  count_launch();
}

void launch_leaves(const uint32_t* pos, int k, const uint32_t* powf, uint32_t* out, int nodes,
                   cudaStream_t st) {
  k_leaves<<<blocks_for(nodes, 64), 64, 0, st>>>(pos, k, powf, out, nodes);
  count_launch();
}

void launch_big_pack(const uint32_t* lvl, int d, int nodes, int L, uint32_t* M, cudaStream_t st) {
  const int cols = 2 * ((nodes + 1) / 2);
  k_big_pack<<<blocks_for((long long)L * cols, 256), 256, 0, st>>>(lvl, d, nodes, L, M);
  count_launch();
}

void launch_big_mul(const uint32_t* Mh, int npairs, int L, uint32_t* Q, cudaStream_t st) {
  k_big_mul<<<blocks_for((long long)L * npairs, 256), 256, 0, st>>>(Mh, npairs, L, Q);
  count_launch();
}

void launch_big_fix(const uint32_t* Q, int d, int k, int npairs, int L, uint32_t* out,
                    cudaStream_t st) {
  k_big_fix<<<blocks_for((long long)(L + 1) * npairs, 256), 256, 0, st>>>(Q, d, k, npairs, L,
                                                                           out);
  count_launch();
}

void launch_pat_prep(const uint32_t* A, int k, int n, int ncols, int h, uint32_t* M,
                     cudaStream_t st) {
  k_pat_prep<<<blocks_for(n, 256), 256, 0, st>>>(A, k, n, ncols, h, M);
  count_launch();
}

void launch_pat_final(const uint32_t* E, int ncols, const uint32_t* pos, int k, int n,
                      const uint32_t* powi, uint32_t ninv, uint2* pat, uint32_t* ahat,
                      uint32_t* ahat2, cudaStream_t st) {
  const int m = n > k ? n : k;
  k_pat_final<<<blocks_for(m, 256), 256, 0, st>>>(E, ncols, pos, k, n, powi, ninv, pat, ahat,
                                                  ahat2);
  count_launch();
}

}  // namespace fntrs
