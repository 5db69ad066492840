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
// the 5th-generation tensor cores (tcgen05, below), with a tiled integer kernel
// (64-bit accumulation of exact products on IMAD.WIDE) kept for comparison
// (environment FNTRS_DIRECT_SIMT=1).
//
// Tensor-core product, exact over F_p: every operand is split into two signed
// 8-bit limbs, x = lo + 256 hi with lo in [-128, 127] and hi in [-128, 128]
// (matrix entries balanced to (-p/2, p/2], data centred by -32768), which BF16
// holds exactly.  The four limb products accumulate in FP32 in tensor memory;
// each term is at most 128 * 128 = 2^14 and K <= 1024 of them sum to at most
// 2^24 in magnitude, so every partial sum is an exact FP32 integer.  The
// epilogue forms c00 + 256 (c01 + c10) + 65536 c11 (65536 = -1 mod p), adds
// 32768 times the row sum of the matrix for the centring and reduces mod p.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdlib>

#include <algorithm>
#include <vector>

#include "../../include/fnt_rs.h"
#include "field.cuh"
#include "internal.h"
#include "kargs.h"
#include "umma.cuh"

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
                                                 int* status, const uint32_t* __restrict__ rmap) {
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
        const size_t row = rmap ? (size_t)rmap[k0 + t] : (size_t)(k0 + t);
        v = (uint32_t)B[row * ld_b + c0 + c];
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
        out16[(mrow ? (size_t)mrow[r] : (size_t)r) * ld_out + c] = (uint16_t)(v > 65535u ? 0u : v);
      }
    }
  }
  if (bad) atomicOr(status, ST_RANGE);
}

// ---- tensor-core product ---------------------------------------------------
// Operand tiles of R rows x 64 K-values in the K-major core-matrix layout
// (8 rows x 8 values = 128 bytes per core matrix, 128 bytes apart along K,
// 1024 bytes apart along the rows), the two limbs of a tile one tile apart:
// the global image of one (row tile, K chunk) pair is exactly what its
// shared-memory stage holds, so one bulk copy moves it.  A (the matrix) has
// 128-row tiles, B (the data, as the N x K operand) 64-row tiles.
constexpr int kTcRows = 128, kTcN = 64, kTcK = 64;
constexpr int kTcTile = kTcRows * kTcK, kTcBTile = kTcN * kTcK;  // elements per limb tile
constexpr int kTcABytes = 2 * kTcTile * 2, kTcBBytes = 2 * kTcBTile * 2;  // both limbs, bf16
constexpr int kTcStages = 4;
constexpr int kTcStageBytes = kTcABytes + kTcBBytes;
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024;  // one CTA (one TMEM user) per SM
constexpr uint32_t kTcCols = 4 * kTcN;                      // four FP32 accumulators
constexpr uint32_t kTcIdesc = idesc_bf16_f32<128, kTcN>();

__device__ __forceinline__ int tc_off(int r, int k) {
  return (r >> 3) * 512 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint16_t bf16_bits(int v) {  // |v| <= 256: exact
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
}

// v in [-32768, 32768] -> v = lo + 256 hi, lo in [-128, 127], hi in [-128, 128]
__device__ __forceinline__ void split_limbs(int v, int& lo, int& hi) {
  lo = ((v + 128) & 255) - 128;
  hi = (v - lo) / 256;
}

// limb tiles of A [M][K] (entries in [0, p), balanced); tile (mt, kc) at
// ((mt * Kc + kc) * 2 + limb) * kTcTile
__global__ void k_tc_limbs_a(const uint32_t* __restrict__ A, int M, int K, int Kc,
                             uint16_t* __restrict__ out, size_t total) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = t / kTcTile;
    const int e = (int)(t % kTcTile), r = e / kTcK, kk = e % kTcK;
    const int mt = (int)(tile / Kc), kc = (int)(tile % Kc);
    const int row = mt * kTcRows + r, col = kc * kTcK + kk;
    int v = 0;
    if (row < M && col < K) {
      const uint32_t a = A[(size_t)row * K + col];
      v = a > 32768u ? (int)a - 65537 : (int)a;
    }
    int lo, hi;
    split_limbs(v, lo, hi);
    uint16_t* o = out + tile * 2 * kTcTile + tc_off(r, kk);
    o[0] = bf16_bits(lo);
    o[kTcTile] = bf16_bits(hi);
  }
}

// limb tiles of the data B [K][ld_b] seen as the N x K operand (row n = column
// n of B), centred: x - 32768 with x = value mod p (received values above
// 65536 raise the range flag); tile (nt, kc) at ((nt * Kc + kc) * 2 + limb) * kTcBTile
// With `copy` set, B is also copied there as u32 rows (the systematic rows of
// an encode, read once for both).
// With `rmap` set, row k of the operand is row rmap[k] of B.
template <class TB>
__global__ void k_tc_limbs_b(const TB* __restrict__ B, size_t ld_b, int K, int W, int Kc,
                             uint16_t* __restrict__ out, size_t total, int* status,
                             uint32_t* __restrict__ copy, size_t ld_copy,
                             const uint32_t* __restrict__ rmap) {
  bool bad = false;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t tile = t / kTcBTile;
    const int e = (int)(t % kTcBTile), kk = e / kTcN, r = e % kTcN;  // r fastest: coalesced
    const int nt = (int)(tile / Kc), kc = (int)(tile % Kc);
    const int n = nt * kTcN + r, k = kc * kTcK + kk;
    int v = 0;
    if (n < W && k < K) {
      const size_t row = rmap ? (size_t)rmap[k] : (size_t)k;
      const uint32_t x = (uint32_t)B[row * ld_b + n];
      bad |= x > 65536u;
      v = (int)m_to_p(x) - 32768;
      if (copy) copy[(size_t)k * ld_copy + n] = x;
    }
    int lo, hi;
    split_limbs(v, lo, hi);
    uint16_t* o = out + tile * 2 * kTcBTile + tc_off(r, kk);
    o[0] = bf16_bits(lo);
    o[kTcBTile] = bf16_bits(hi);
  }
  if (bad) atomicOr(status, ST_RANGE);
}

// C = A B over F_p for one 128 x 64 output tile.  Thread 0 keeps up to
// kTcStages K chunks in flight (one bulk copy of the A chunk and one of the B
// chunk per stage, completing on the stage's `full` barrier) and, per chunk,
// issues 4 K-steps x 4 limb pairs of 128x64x16 BF16 MMAs into four FP32
// accumulators, whose completion (tcgen05.commit) frees the stage.  All waits
// are bounded.  Output as in k_fp_gemm.
__global__ void __launch_bounds__(128, 1)
    k_fp_gemm_tc(const uint16_t* __restrict__ Al, const uint16_t* __restrict__ Bl, int M, int Kc,
                 int W, const uint32_t* __restrict__ corr, uint32_t* __restrict__ out32,
                 size_t row0, uint16_t* __restrict__ out16, const uint32_t* __restrict__ mrow,
                 size_t ld_out, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t full[kTcStages], empty[kTcStages];
  __shared__ uint32_t tslot;
  __shared__ int s_ok;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int mt = blockIdx.y, nt = blockIdx.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    s_ok = 1;
  }
  if (warp == 0) tmem_alloc(&tslot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tslot;
  if (threadIdx.x == 0) {
    const uint8_t* gA = reinterpret_cast<const uint8_t*>(Al) + (size_t)mt * Kc * kTcABytes;
    const uint8_t* gB = reinterpret_cast<const uint8_t*>(Bl) + (size_t)nt * Kc * kTcBBytes;
    auto load = [&](int c) {
      uint8_t* st = base + (c % kTcStages) * kTcStageBytes;
      uint64_t* bar = &full[c % kTcStages];
      mbar_expect_tx(bar, kTcStageBytes);
      bulk_g2s(st, gA + (size_t)c * kTcABytes, kTcABytes, bar);
      bulk_g2s(st + kTcABytes, gB + (size_t)c * kTcBBytes, kTcBBytes, bar);
    };
    const int pre = Kc < kTcStages ? Kc : kTcStages;
    for (int c = 0; c < pre; ++c) load(c);
    int loaded = pre, issued = 0;
    bool ok = true;
    for (int c = 0; c < Kc; ++c) {
      const int s = c % kTcStages;
      const uint32_t ph = (uint32_t)(c / kTcStages) & 1u;
      if (!(ok = mbar_wait(&full[s], ph))) break;
      tc_fence_after();
      const uint16_t* sA = reinterpret_cast<const uint16_t*>(base + s * kTcStageBytes);
      const uint16_t* sB = reinterpret_cast<const uint16_t*>(base + s * kTcStageBytes + kTcABytes);
#pragma unroll
      for (int k = 0; k < kTcK / 16; ++k)
#pragma unroll
        for (int la = 0; la < 2; ++la)
#pragma unroll
          for (int lb = 0; lb < 2; ++lb)
            mma_bf16(taddr + (uint32_t)(2 * la + lb) * kTcN,
                     smem_desc(sA + la * kTcTile + k * 128, 128, 1024),
                     smem_desc(sB + lb * kTcBTile + k * 128, 128, 1024), kTcIdesc,
                     (c > 0 || k > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
      issued = c + 1;
      if (c + kTcStages < Kc) {
        // the stage is refilled once its MMAs are done; the other stages stay in flight
        if (!(ok = mbar_wait(&empty[s], ph))) break;
        load(c + kTcStages);
        loaded = c + kTcStages + 1;
      }
    }
    if (ok && issued > 0) {  // the last commit covers every MMA issued before it
      const int c = issued - 1;
      ok = mbar_wait(&empty[c % kTcStages], (uint32_t)(c / kTcStages) & 1u);
    }
    if (!ok) {
      atomicOr(status, ST_TIMEOUT);
      // bounded waits for the copies and MMAs still in flight before TMEM is freed
      for (int c = issued; c < loaded; ++c)
        mbar_wait(&full[c % kTcStages], (uint32_t)(c / kTcStages) & 1u);
      if (issued > 0)
        mbar_wait(&empty[(issued - 1) % kTcStages], (uint32_t)((issued - 1) / kTcStages) & 1u);
      s_ok = 0;
    }
  }
  __syncthreads();
  if (s_ok) {
    // each thread combines its accumulator row into a [128][65] tile in the
    // (now free) stage memory; the tile then leaves in whole rows
    uint32_t* tile = reinterpret_cast<uint32_t*>(base);
    tc_fence_after();
    const int rl = warp * 32 + lane;
    const int r = mt * kTcRows + rl;
    const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
    // |value| < 2^34 + 2^17 < 65537 * 2^18: adding that multiple of p makes it positive
    const int64_t bias = (r < M ? (int64_t)corr[r] : 0) + 65537ll * (1ll << 18);
    for (int j0 = 0; j0 < kTcN; j0 += 16) {
      float c00[16], c01[16], c10[16], c11[16];
      tmem_ld16(lane_addr + 0u * kTcN + (uint32_t)j0, c00);
      tmem_ld16(lane_addr + 1u * kTcN + (uint32_t)j0, c01);
      tmem_ld16(lane_addr + 2u * kTcN + (uint32_t)j0, c10);
      tmem_ld16(lane_addr + 3u * kTcN + (uint32_t)j0, c11);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const uint64_t u = (uint64_t)((int64_t)__float2int_rn(c00[i]) +
                                      256 * ((int64_t)__float2int_rn(c01[i]) +
                                             (int64_t)__float2int_rn(c10[i])) -
                                      (int64_t)__float2int_rn(c11[i]) + bias);
        // 2^32 = 1 mod p: fold the high word, then reduce
        tile[rl * (kTcN + 1) + j0 + i] = m_to_p(m_add((uint32_t)u, (uint32_t)(u >> 32)));
      }
    }
    __syncthreads();
    bool bad = false;
    for (int e = threadIdx.x; e < kTcRows * kTcN; e += 128) {
      const int rr = e / kTcN, j = e % kTcN;
      const int row = mt * kTcRows + rr, col = nt * kTcN + j;
      if (row >= M || col >= W) continue;
      const uint32_t v = tile[rr * (kTcN + 1) + j];
      if (out32) {
        out32[(row0 + row) * ld_out + col] = v;
      } else {
        bad |= v > 65535u;
        out16[(mrow ? (size_t)mrow[row] : (size_t)row) * ld_out + col] =
            (uint16_t)(v > 65535u ? 0u : v);
      }
    }
    if (bad) atomicOr(status, ST_RANGE);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(taddr, kTcCols);
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
                cudaStream_t st, const uint32_t* rmap = nullptr) {
  if (M <= 0 || W <= 0) return FNT_RS_OK;
  const dim3 grid((unsigned)((W + 63) / 64), (unsigned)((M + 63) / 64));
  if (grid.y > 65535u) return FNT_RS_E_ARG;
  k_fp_gemm<TB><<<grid, 256, 0, st>>>(A, M, K, B, ld_b, W, out32, row0, out16, mrow, ld_out,
                                      status, rmap);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

}  // namespace

constexpr uint32_t kDirectMaxK = 1024;  // also the exactness bound of the tensor-core product
constexpr uint32_t kDirectMaxN = 16384;

// One matrix of a direct product: u32 entries in [0, p) (the integer kernel's
// operand and the source of the limb tiles), the tensor-core limb tiles and
// the per-row centring correction 32768 * row sum.
struct DirectMat {
  uint32_t* a = nullptr;
  uint32_t* corr = nullptr;
  uint16_t* limbs = nullptr;
  int rows = 0;
};

struct DirectState {
  bool simt = false;  // FNTRS_DIRECT_SIMT=1: the integer kernel instead of the tensor cores
  // systematic encode: G [(n - k)][k] = L_i(r^j), j = k .. n-1 (built when selected)
  DirectMat G;
  // non-systematic encode: V [n][k] = r^(ij) (built when selected)
  DirectMat V;
  // systematic decode, per pattern: D [missing][k], its output rows and the copies
  DirectMat D;
  uint32_t* mrow = nullptr;  // [k]
  uint2* cmap = nullptr;     // [k]: {received row, output row}
  std::vector<uint32_t> dkey;
  int nmiss = 0, ncopy = 0;
  bool d_ready = false;
  // non-systematic decode, per pattern: M [k][k] = coefficients of the Lagrange basis
  DirectMat Mi;
  uint32_t* rmap = nullptr;  // [k]: slot-buffer row of basis index l (= its position)
  std::vector<uint32_t> mkey;
  bool m_ready = false;
};

namespace {

int tiles(int rows) { return (rows + kTcRows - 1) / kTcRows; }
int ntiles(int cols) { return (cols + kTcN - 1) / kTcN; }
int kchunks(int K) { return (K + kTcK - 1) / kTcK; }
size_t limb_bytes(int rows, int K) { return (size_t)tiles(rows) * kchunks(K) * kTcABytes; }
size_t data_limb_bytes(int cols, int K) { return (size_t)ntiles(cols) * kchunks(K) * kTcBBytes; }

std::vector<uint32_t> centring(const std::vector<uint32_t>& rows, size_t k) {
  const size_t m = k ? rows.size() / k : 0;
  std::vector<uint32_t> c(m);
  for (size_t t = 0; t < m; ++t) {
    uint64_t acc = 0;
    for (size_t l = 0; l < k; ++l) acc += rows[t * k + l];
    c[t] = hm((uint32_t)(acc % kPh), 32768u);
  }
  return c;
}

int limbs_a(const fnt_rs_plan_s* p, const uint32_t* A, int M, int K, uint16_t* out,
            cudaStream_t st) {
  const size_t total = (size_t)tiles(M) * kchunks(K) * kTcTile;
  if (total == 0) return FNT_RS_OK;
  k_tc_limbs_a<<<grid_for(p, total), 256, 0, st>>>(A, M, K, kchunks(K), out, total);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

void mat_free(DirectMat& m) {
  cudaFree(m.a);
  cudaFree(m.limbs);
  m = DirectMat{};
}

// device storage for up to `rows` x k entries (+ limbs unless simt)
int mat_alloc(DirectMat& m, int rows, int k, bool simt) {
  if (m.a) return FNT_RS_OK;
  int rc = cuda_ok(cudaMalloc(&m.a, ((size_t)std::max(rows, 1) * k + std::max(rows, 1)) * 4));
  if (rc) return rc;
  m.corr = m.a + (size_t)std::max(rows, 1) * k;
  if (!simt && (rc = cuda_ok(cudaMalloc(&m.limbs, std::max<size_t>(16, limb_bytes(rows, k))))))
    return rc;
  return FNT_RS_OK;
}

// host matrix -> device entries, corrections and limb tiles (on st; the host
// vectors are staged by the pageable copies before they return)
int mat_upload(const fnt_rs_plan_s* p, DirectMat& m, const std::vector<uint32_t>& a, int rows,
               int k, bool simt, cudaStream_t st) {
  m.rows = rows;
  if (rows == 0) return FNT_RS_OK;
  const std::vector<uint32_t> c = centring(a, (size_t)k);
  int rc = cuda_ok(cudaMemcpyAsync(m.a, a.data(), a.size() * 4, cudaMemcpyHostToDevice, st));
  if (!rc)
    rc = cuda_ok(cudaMemcpyAsync(m.corr, c.data(), c.size() * 4, cudaMemcpyHostToDevice, st));
  if (!rc && !simt) rc = limbs_a(p, m.a, rows, k, m.limbs, st);
  return rc;
}

template <class TB>
int gemm_tc(fnt_rs_plan_s* p, const uint16_t* Al, const uint32_t* corr, int M, const TB* B,
            size_t ld_b, int W, void* work, uint32_t* out32, size_t row0, uint16_t* out16,
            const uint32_t* mrow, size_t ld_out, cudaStream_t st, uint32_t* copy = nullptr,
            size_t ld_copy = 0, const uint32_t* rmap = nullptr) {
  if (W <= 0 || (M <= 0 && !copy)) return FNT_RS_OK;
  if (reinterpret_cast<uintptr_t>(work) % 16 != 0) return FNT_RS_E_ARG;  // bulk-copy source
  static bool attr[64] = {};  // the opt-in is per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr[dev & 63]) {
    if (cudaFuncSetAttribute(k_fp_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTcSmem) != cudaSuccess)
      return FNT_RS_E_CUDA;
    attr[dev & 63] = true;
  }
  const int K = (int)p->k, Kc = kchunks(K);
  uint16_t* Bl = static_cast<uint16_t*>(work);
  const size_t total = (size_t)ntiles(W) * Kc * kTcBTile;
  k_tc_limbs_b<TB><<<grid_for(p, total), 256, 0, st>>>(B, ld_b, K, W, Kc, Bl, total, p->status,
                                                        copy, ld_copy, rmap);
  count_launch();
  if (M <= 0) return cuda_ok(cudaGetLastError());
  const dim3 grid((unsigned)ntiles(W), (unsigned)tiles(M));
  if (grid.y > 65535u) return FNT_RS_E_ARG;
  k_fp_gemm_tc<<<grid, 128, kTcSmem, st>>>(Al, Bl, M, Kc, W, corr, out32, row0, out16, mrow,
                                           ld_out, p->status);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

// C = A B with A one of the direct matrices (rows m.rows), on the tensor cores
// or (systematic ops with FNTRS_DIRECT_SIMT=1) the integer kernel, which must
// not write the rows it reads
template <class TB>
int product(fnt_rs_plan_s* p, const DirectMat& m, const TB* B, size_t ld_b, int W, void* work,
            uint32_t* out32, size_t row0, uint16_t* out16, const uint32_t* mrow, size_t ld_out,
            cudaStream_t st, bool simt, const uint32_t* rmap = nullptr) {
  if (simt)
    return launch_gemm<TB>(m.a, m.rows, (int)p->k, B, ld_b, W, out32, row0, out16, mrow, ld_out,
                           p->status, st, rmap);
  return gemm_tc<TB>(p, m.limbs, m.corr, m.rows, B, ld_b, W, work, out32, row0, out16, mrow,
                     ld_out, st, nullptr, 0, rmap);
}

uint32_t root_of(uint32_t n) { return hp(3, 65536u / n); }

}  // namespace

bool direct_available(const fnt_rs_plan_s* p) {
  return p->k <= kDirectMaxK && p->n <= kDirectMaxN && p->u == 1;
}

size_t direct_ws_bytes(const fnt_rs_plan_s* p, size_t W) {
  if (!p->direct || W == 0) return 0;
  return data_limb_bytes((int)W, (int)p->k);
}

void direct_free(fnt_rs_plan_s* p) {
  DirectState* s = p->direct;
  if (!s) return;
  mat_free(s->G);
  mat_free(s->V);
  mat_free(s->D);
  mat_free(s->Mi);
  cudaFree(s->mrow);
  cudaFree(s->rmap);
  delete s;
  p->direct = nullptr;
}

// Builds what the direct method of `op` needs (FNT_RS_OP_ENCODE / _DECODE /
// _ENCODE_SYS / _DECODE_SYS): plan-level matrices now, per-pattern buffers
// reserved for later.  Synchronises the device.
int direct_enable(fnt_rs_plan_s* p, int op) {
  if (!direct_available(p)) return FNT_RS_E_ARG;
  if (!p->direct) {
    p->direct = new DirectState();
    const char* e = std::getenv("FNTRS_DIRECT_SIMT");
    p->direct->simt = e && e[0] == '1';
  }
  DirectState* s = p->direct;
  const uint32_t n = p->n, k = p->k;
  const uint32_t r = root_of(n);
  int rc = FNT_RS_OK;
  if (op == FNT_RS_OP_ENCODE_SYS && !s->G.a) {
    std::vector<uint32_t> xs(k), pts(n - k), G;
    for (uint32_t i = 0; i < k; ++i) xs[i] = hp(r, i);
    for (uint32_t j = k; j < n; ++j) pts[j - k] = hp(r, j);
    lagrange_rows(xs, pts, G);
    if ((rc = mat_alloc(s->G, (int)(n - k), (int)k, s->simt)) ||
        (rc = mat_upload(p, s->G, G, (int)(n - k), (int)k, s->simt, nullptr)))
      return rc;
  } else if (op == FNT_RS_OP_ENCODE && !s->V.a) {
    std::vector<uint32_t> V((size_t)n * k);
    for (uint32_t j = 0; j < n; ++j) {
      const uint32_t rj = hp(r, j);
      uint32_t x = 1;
      for (uint32_t i = 0; i < k; ++i, x = hm(x, rj)) V[(size_t)j * k + i] = x;
    }
    if ((rc = mat_alloc(s->V, (int)n, (int)k, false)) ||
        (rc = mat_upload(p, s->V, V, (int)n, (int)k, false, nullptr)))
      return rc;
  } else if (op == FNT_RS_OP_DECODE_SYS && !s->D.a) {
    if ((rc = mat_alloc(s->D, (int)k, (int)k, s->simt))) return rc;
    const size_t k2 = (k + 1) & ~1u;  // cmap (8-byte entries) starts 8-byte aligned
    if (!s->mrow && (rc = cuda_ok(cudaMalloc(&s->mrow, k2 * 4 + (size_t)k * 8)))) return rc;
    s->cmap = reinterpret_cast<uint2*>(s->mrow + k2);
  } else if (op == FNT_RS_OP_DECODE && !s->Mi.a) {
    if ((rc = mat_alloc(s->Mi, (int)k, (int)k, false))) return rc;
    if ((rc = cuda_ok(cudaMalloc(&s->rmap, (size_t)k * 4)))) return rc;
  }
  return cuda_ok(cudaDeviceSynchronize());
}

bool direct_ready(const fnt_rs_plan_s* p, int op) {
  const DirectState* s = p->direct;
  if (!s) return false;
  switch (op) {
    case FNT_RS_OP_ENCODE_SYS: return s->G.a != nullptr;
    case FNT_RS_OP_ENCODE: return s->V.a != nullptr;
    case FNT_RS_OP_DECODE_SYS: return s->D.a != nullptr;
    case FNT_RS_OP_DECODE: return s->Mi.a != nullptr;
    default: return false;
  }
}

int direct_encode_sys(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                      size_t ld_enc, size_t W, void* workspace, cudaStream_t st) {
  DirectState* s = p->direct;
  if (!direct_ready(p, FNT_RS_OP_ENCODE_SYS)) return FNT_RS_E_ARG;
  if (!s->simt && !workspace) return FNT_RS_E_WORKSPACE;
  const int k = (int)p->k;
  const int M = (int)(p->n_out - p->k);
  if (!s->simt)  // the systematic rows are copied by the kernel that splits the source
    return gemm_tc<uint16_t>(p, s->G.limbs, s->G.corr, M, src, ld_src, (int)W, workspace, enc,
                             (size_t)k, nullptr, nullptr, ld_enc, st, enc, ld_enc);
  k_copy_src<<<grid_for(p, (size_t)k * W), 256, 0, st>>>(src, ld_src, enc, ld_enc, k, (int)W);
  count_launch();
  const int rc = cuda_ok(cudaGetLastError());
  if (rc) return rc;
  return launch_gemm<uint16_t>(s->G.a, M, k, src, ld_src, (int)W, enc, (size_t)k, nullptr,
                               nullptr, ld_enc, p->status, st);
}

int direct_decode_sys(fnt_rs_plan_s* p, const uint32_t* recv, size_t ld_recv,
                      const uint32_t* positions, uint16_t* out, size_t ld_out, size_t W,
                      void* workspace, cudaStream_t st) {
  DirectState* s = p->direct;
  if (!direct_ready(p, FNT_RS_OP_DECODE_SYS)) return FNT_RS_E_ARG;
  if (!s->simt && !workspace) return FNT_RS_E_WORKSPACE;
  const uint32_t n = p->n, k = p->k;
  std::vector<uint32_t> key(positions, positions + k);
  if (!s->d_ready || s->dkey != key) {
    s->d_ready = false;
    const uint32_t r = root_of(n);
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
    int rc = mat_upload(p, s->D, D, (int)mrow.size(), (int)k, s->simt, st);
    if (!rc && !mrow.empty())
      rc = cuda_ok(cudaMemcpyAsync(s->mrow, mrow.data(), mrow.size() * 4, cudaMemcpyHostToDevice,
                                   st));
    if (!rc && !cmap.empty())
      rc = cuda_ok(cudaMemcpyAsync(s->cmap, cmap.data(), cmap.size() * 8, cudaMemcpyHostToDevice,
                                   st));
    if (rc) return rc;
    s->nmiss = (int)mrow.size();
    s->ncopy = (int)cmap.size();
    s->dkey.swap(key);
    s->d_ready = true;
  }
  if (s->ncopy) {
    k_copy_recv<<<grid_for(p, (size_t)s->ncopy * W), 256, 0, st>>>(recv, ld_recv, s->cmap,
                                                                     s->ncopy, out, ld_out,
                                                                     (int)W, p->status);
    count_launch();
    const int rc = cuda_ok(cudaGetLastError());
    if (rc) return rc;
  }
  return product<uint32_t>(p, s->D, recv, ld_recv, (int)W, workspace, nullptr, 0, out, s->mrow,
                           ld_out, st, s->simt);
}

int direct_encode(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                  size_t ld_enc, size_t W, void* workspace, cudaStream_t st) {
  DirectState* s = p->direct;
  if (!direct_ready(p, FNT_RS_OP_ENCODE)) return FNT_RS_E_ARG;
  if (!workspace) return FNT_RS_E_WORKSPACE;
  DirectMat v = s->V;
  v.rows = (int)p->n_out;  // a punctured code keeps the first n_out rows
  return product<uint16_t>(p, v, src, ld_src, (int)W, workspace, enc, 0, nullptr, nullptr,
                           ld_enc, st, false);
}

int direct_decode(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv, size_t ld_recv,
                  uint16_t* out, size_t ld_out, size_t W, void* workspace, cudaStream_t st,
                  int slots, uint32_t* out32) {
  DirectState* s = p->direct;
  if (!direct_ready(p, FNT_RS_OP_DECODE)) return FNT_RS_E_ARG;
  if (!workspace) return FNT_RS_E_WORKSPACE;
  const uint32_t n = p->n, k = p->k;
  std::vector<uint32_t> key = sl.key;
  if (&sl == &p->sys) {
    key.resize(k);
    for (uint32_t i = 0; i < k; ++i) key[i] = i;
  }
  if (!s->m_ready || s->mkey != key) {
    s->m_ready = false;
    // M[i][l] = coefficient i of L_l(x) = w_l A(x) / (x - x_l), A = prod (x - x_m)
    const uint32_t r = root_of(n);
    std::vector<uint32_t> xs(k), A(k + 1, 0), M((size_t)k * k), q(k), wl(k), dA(k);
    for (uint32_t l = 0; l < k; ++l) xs[l] = hp(r, key[l]);
    A[0] = 1;
    for (uint32_t m = 0; m < k; ++m) {  // multiply by (x - x_m)
      for (uint32_t i = m + 1; i > 0; --i) A[i] = (A[i - 1] + hm(kPh - xs[m], A[i])) % kPh;
      A[0] = hm(kPh - xs[m], A[0]);
    }
    std::vector<std::vector<uint32_t>> Q(k);
    for (uint32_t l = 0; l < k; ++l) {
      // synthetic division: Q = A / (x - x_l), degree k-1; A'(x_l) = Q(x_l)
      q[k - 1] = A[k];
      for (uint32_t i = k - 1; i > 0; --i) q[i - 1] = (A[i] + hm(xs[l], q[i])) % kPh;
      uint32_t v = 0;
      for (uint32_t i = k; i-- > 0;) v = (hm(v, xs[l]) + q[i]) % kPh;
      dA[l] = v;
      Q[l] = q;
    }
    batch_inverse(dA, wl);
    for (uint32_t l = 0; l < k; ++l)
      for (uint32_t i = 0; i < k; ++i) M[(size_t)i * k + l] = hm(wl[l], Q[l][i]);
    int rc = mat_upload(p, s->Mi, M, (int)k, (int)k, false, st);
    if (!rc) rc = cuda_ok(cudaMemcpyAsync(s->rmap, key.data(), (size_t)k * 4,
                                          cudaMemcpyHostToDevice, st));
    if (rc) return rc;
    s->mkey.swap(key);
    s->m_ready = true;
  }
  // tensor cores only: the source limbs are split off before the product, so the
  // output may overwrite the received rows (the systematic code's in-place use)
  return product<uint32_t>(p, s->Mi, recv, ld_recv, (int)W, workspace, out32, 0,
                           out32 ? nullptr : out, nullptr, ld_out, st, false,
                           slots ? s->rmap : nullptr);
}

}  // namespace fntrs
