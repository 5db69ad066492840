// Direct (quadratic) systematic encoder and decoder, the paper's alternative
// for short codes (Sec. III, Tables I and II: "direct encoding" of the n - k
// non-systematic symbols, O((n-k) k), and "direct decoding" of the missing
// source symbols).
//
// Both are products of a matrix over F_p by the batch of codewords:
//   encode  e_j = sum_i G[j][i] s_i, j in [k, n_out): G[j][i] = L_i(r^j), the
//           Lagrange basis of the nodes r^0 .. r^(k-1) at r^j (the intermediate
//           polynomial of the systematic code takes the value s_i at r^i);
//   decode  the first k received positions z_l are the nodes; a source row m < k
//           that was received is copied, a missing one is
//           s_m = sum_l D[m][l] v_l with D[m][l] = L_l(r^m) for those nodes.
// L_i(x) = w_i A(x) / (x - x_i), A = prod (x - x_l), w_i = 1 / A'(x_i): the
// matrices are built on the host in O(rows * k) (one batched inversion per
// row) -- G once per plan, D once per erasure pattern -- and the products run in
// a tiled integer kernel: 64-bit accumulation of the exact 17 x 32-bit products
// (IMAD.WIDE), one reduction per output (2^32 = 1 mod p).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/fnt_rs.h"
#include "field.cuh"
#include "internal.h"
#include "kargs.h"

namespace fntrs {

void count_launch();

namespace {

constexpr uint32_t kPh = 65537u;

uint32_t hm(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) % kPh); }
uint32_t hp(uint32_t a, uint64_t e) {
  uint64_t r = 1, x = a % kPh;
  while (e) {
    if (e & 1) r = r * x % kPh;
    x = x * x % kPh;
    e >>= 1;
  }
  return (uint32_t)r;
}
uint32_t hsub(uint32_t a, uint32_t b) { return (a + kPh - b) % kPh; }

// out[i] = 1 / in[i] for all i (one inversion: prefix products); no zero inputs
void batch_inverse(const std::vector<uint32_t>& in, std::vector<uint32_t>& out) {
  const size_t m = in.size();
  out.resize(m);
  if (m == 0) return;
  std::vector<uint32_t> pre(m);
  uint32_t acc = 1;
  for (size_t i = 0; i < m; ++i) {
    pre[i] = acc;
    acc = hm(acc, in[i]);
  }
  uint32_t inv = hp(acc, kPh - 2);
  for (size_t i = m; i-- > 0;) {
    out[i] = hm(inv, pre[i]);
    inv = hm(inv, in[i]);
  }
}

// rows[t][l] = L_l(x_t) for the nodes xs (distinct) and points pts (no node among them)
void lagrange_rows(const std::vector<uint32_t>& xs, const std::vector<uint32_t>& pts,
                   std::vector<uint32_t>& rows) {
  const size_t k = xs.size(), m = pts.size();
  // w_l = 1 / prod_{j != l} (x_l - x_j)
  std::vector<uint32_t> dA(k, 1), w;
  for (size_t l = 0; l < k; ++l)
    for (size_t j = 0; j < k; ++j)
      if (j != l) dA[l] = hm(dA[l], hsub(xs[l], xs[j]));
  batch_inverse(dA, w);
  rows.assign(m * k, 0);
  std::vector<uint32_t> diff(k), inv;
  for (size_t t = 0; t < m; ++t) {
    uint32_t A = 1;
    for (size_t l = 0; l < k; ++l) {
      diff[l] = hsub(pts[t], xs[l]);
      A = hm(A, diff[l]);
    }
    batch_inverse(diff, inv);
    uint32_t* row = rows.data() + t * k;
    for (size_t l = 0; l < k; ++l) row[l] = hm(hm(w[l], A), inv[l]);
  }
}

// C[r][c] = sum_t A[r][t] B[t][c] mod p for r < M, c < W (A: [M][K] u32 in
// [0, p), row-major; B: [K][ld_b] values taken mod p, above 65536 flagged).
// 64 x 64 outputs per CTA, 256 threads with 4 x 4 each, K in chunks of 32.
// Output: u32 rows row0 + r of out32, or u16 rows mrow[r] of out16 (65536 ->
// 0 with the range flag).
template <class TB>
__global__ void __launch_bounds__(256) k_fp_gemm(const uint32_t* __restrict__ A, int M, int K,
                                                 const TB* __restrict__ B, size_t ld_b, int W,
                                                 uint32_t* __restrict__ out32, size_t row0,
                                                 uint16_t* __restrict__ out16,
                                                 const uint32_t* __restrict__ mrow, size_t ld_out,
                                                 int* status) {
  constexpr int TM = 64, TN = 64, TK = 32;
  __shared__ uint32_t As[TK][TM + 1];
  __shared__ uint32_t Bs[TK][TN];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = blockIdx.y * TM, c0 = blockIdx.x * TN;
  uint64_t acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  bool bad = false;
  for (int k0 = 0; k0 < K; k0 += TK) {
    // A tile [64][32] -> As[t][r] (transposed), B tile [32][64]
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      const int r = e / TK, t = e % TK;
      As[t][r] = (r0 + r < M && k0 + t < K) ? A[(size_t)(r0 + r) * K + k0 + t] : 0u;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      const int t = e / TN, c = e % TN;
      uint32_t v = 0;
      if (k0 + t < K && c0 + c < W) {
        v = (uint32_t)B[(size_t)(k0 + t) * ld_b + c0 + c];
        bad |= v > 65536u;
      }
      Bs[t][c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < TK; ++t) {
      uint32_t a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[t][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[t][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += (uint64_t)a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c >= W) continue;
      const uint32_t v = m_to_p(m_add((uint32_t)acc[i][j], (uint32_t)(acc[i][j] >> 32)));
      if (out32) {
        out32[(row0 + r) * ld_out + c] = v;
      } else {
        bad |= v > 65535u;
        out16[(size_t)mrow[r] * ld_out + c] = (uint16_t)(v > 65535u ? 0u : v);
      }
    }
  }
  if (bad) atomicOr(status, ST_RANGE);
}

// encode: enc[i][c] = src[i][c], i < k
__global__ void k_copy_src(const uint16_t* __restrict__ src, size_t ld_src, uint32_t* enc,
                           size_t ld_enc, int k, int W) {
  const size_t total = (size_t)k * W;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / W, c = t % W;
    enc[r * ld_enc + c] = src[r * ld_src + c];
  }
}

// decode: out[map[l].y][c] = recv[map[l].x][c] mod p for the received source
// rows (65536 -> 0 and received values above 65536 raise the range flag)
__global__ void k_copy_recv(const uint32_t* __restrict__ recv, size_t ld_recv,
                            const uint2* __restrict__ map, int nmap, uint16_t* out, size_t ld_out,
                            int W, int* status) {
  const size_t total = (size_t)nmap * W;
  bool bad = false;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t l = t / W, c = t % W;
    const uint2 e = map[l];
    const uint32_t v = recv[(size_t)e.x * ld_recv + c];
    const uint32_t r = m_to_p(v);
    bad |= v > 65536u || r > 65535u;
    out[(size_t)e.y * ld_out + c] = (uint16_t)(r > 65535u ? 0u : r);
  }
  if (bad) atomicOr(status, ST_RANGE);
}

unsigned grid_for(const fnt_rs_plan_s* p, size_t work) {
  const size_t want = (work + 255) / 256;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)p->sms * 8));
}

template <class TB>
int launch_gemm(const uint32_t* A, int M, int K, const TB* B, size_t ld_b, int W, uint32_t* out32,
                size_t row0, uint16_t* out16, const uint32_t* mrow, size_t ld_out, int* status,
                cudaStream_t st) {
  if (M <= 0 || W <= 0) return FNT_RS_OK;
  const dim3 grid((unsigned)((W + 63) / 64), (unsigned)((M + 63) / 64));
  if (grid.y > 65535u) return FNT_RS_E_ARG;
  k_fp_gemm<TB><<<grid, 256, 0, st>>>(A, M, K, B, ld_b, W, out32, row0, out16, mrow, ld_out,
                                      status);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

}  // namespace

constexpr uint32_t kDirectMaxK = 1024;
constexpr uint32_t kDirectMaxN = 16384;

struct DirectState {
  uint32_t* G = nullptr;     // [(n - k)][k]: L_i(r^j), j = k .. n-1
  uint32_t* D = nullptr;     // [k][k] max: rows of the missing source symbols
  uint32_t* mrow = nullptr;  // [k]: output row of each D row
  uint2* cmap = nullptr;     // [k]: {received row, output row} of received source rows
  std::vector<uint32_t> key;
  int nmiss = 0, ncopy = 0;
  bool pattern_ready = false;
};

bool direct_available(const fnt_rs_plan_s* p) {
  return p->k <= kDirectMaxK && p->n <= kDirectMaxN && p->u == 1;
}

void direct_free(fnt_rs_plan_s* p) {
  DirectState* s = p->direct;
  if (!s) return;
  cudaFree(s->G);
  cudaFree(s->D);
  delete s;
  p->direct = nullptr;
}

int direct_enable(fnt_rs_plan_s* p) {
  if (p->direct) return FNT_RS_OK;
  if (!direct_available(p)) return FNT_RS_E_ARG;
  const uint32_t n = p->n, k = p->k;
  DirectState* s = new DirectState();
  p->direct = s;
  auto fail = [&](int rc) {
    direct_free(p);
    return rc;
  };
  const uint32_t r = hp(3, 65536u / n);
  std::vector<uint32_t> xs(k), pts(n - k), G;
  for (uint32_t i = 0; i < k; ++i) xs[i] = hp(r, i);
  for (uint32_t j = k; j < n; ++j) pts[j - k] = hp(r, j);
  lagrange_rows(xs, pts, G);
  int rc;
  const size_t gbytes = std::max<size_t>(4, G.size() * 4);
  // G | D (k x k) | mrow (k) | cmap (k uint2)
  const size_t dwords = (size_t)k * k + k + 2 * (size_t)k;
  if ((rc = cuda_ok(cudaMalloc(&s->G, gbytes)))) return fail(rc);
  if ((rc = cuda_ok(cudaMalloc(&s->D, dwords * 4)))) return fail(rc);
  s->mrow = s->D + (size_t)k * k;
  s->cmap = reinterpret_cast<uint2*>(s->mrow + k);
  if (!G.empty() &&
      (rc = cuda_ok(cudaMemcpy(s->G, G.data(), G.size() * 4, cudaMemcpyHostToDevice))))
    return fail(rc);
  return FNT_RS_OK;
}

int direct_encode_sys(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                      size_t ld_enc, size_t W, cudaStream_t st) {
  DirectState* s = p->direct;
  if (!s) return FNT_RS_E_ARG;
  const int k = (int)p->k;
  k_copy_src<<<grid_for(p, (size_t)k * W), 256, 0, st>>>(src, ld_src, enc, ld_enc, k, (int)W);
  count_launch();
  int rc = cuda_ok(cudaGetLastError());
  if (rc) return rc;
  return launch_gemm<uint16_t>(s->G, (int)(p->n_out - p->k), k, src, ld_src, (int)W, enc,
                               (size_t)k, nullptr, nullptr, ld_enc, p->status, st);
}

int direct_decode_sys(fnt_rs_plan_s* p, const uint32_t* recv, size_t ld_recv,
                      const uint32_t* positions, uint16_t* out, size_t ld_out, size_t W,
                      cudaStream_t st) {
  DirectState* s = p->direct;
  if (!s) return FNT_RS_E_ARG;
  const uint32_t n = p->n, k = p->k;
  std::vector<uint32_t> key(positions, positions + k);
  if (!s->pattern_ready || s->key != key) {
    s->pattern_ready = false;
    const uint32_t r = hp(3, 65536u / n);
    std::vector<uint32_t> xs(k), pts, mrow, D;
    std::vector<uint2> cmap;
    std::vector<char> got(k, 0);
    for (uint32_t l = 0; l < k; ++l) {
      xs[l] = hp(r, key[l]);
      if (key[l] < k) {
        got[key[l]] = 1;
        cmap.push_back(make_uint2(l, key[l]));
      }
    }
    for (uint32_t m = 0; m < k; ++m)
      if (!got[m]) {
        pts.push_back(hp(r, m));
        mrow.push_back(m);
      }
    lagrange_rows(xs, pts, D);
    int rc;
    if (!D.empty() && (rc = cuda_ok(cudaMemcpyAsync(s->D, D.data(), D.size() * 4,
                                                    cudaMemcpyHostToDevice, st))))
      return rc;
    if (!mrow.empty() && (rc = cuda_ok(cudaMemcpyAsync(s->mrow, mrow.data(), mrow.size() * 4,
                                                       cudaMemcpyHostToDevice, st))))
      return rc;
    if (!cmap.empty() && (rc = cuda_ok(cudaMemcpyAsync(s->cmap, cmap.data(), cmap.size() * 8,
                                                       cudaMemcpyHostToDevice, st))))
      return rc;
    // the host vectors are staged by the copies (pageable memory) before they return
    s->nmiss = (int)mrow.size();
    s->ncopy = (int)cmap.size();
    s->key.swap(key);
    s->pattern_ready = true;
  }
  if (s->ncopy) {
    k_copy_recv<<<grid_for(p, (size_t)s->ncopy * W), 256, 0, st>>>(recv, ld_recv, s->cmap,
                                                                     s->ncopy, out, ld_out,
                                                                     (int)W, p->status);
    count_launch();
    const int rc = cuda_ok(cudaGetLastError());
    if (rc) return rc;
  }
  return launch_gemm<uint32_t>(s->D, s->nmiss, (int)k, recv, ld_recv, (int)W, nullptr, 0, out,
                               s->mrow, ld_out, p->status, st);
}

}  // namespace fntrs
