// The paper's own decode route (decode schedule FNT_RS_SCHED_PAPER).
//
// Sec. II.B evaluates polynomials on geometric progressions by the chirp
// identity r^(ij) = b_(i+j) / (b_i b_j), b_i = r^(t_i), t_i = i(i-1)/2, which
// turns an evaluation into the middle coefficients of one polynomial product;
// Sec. III counts that route as 4 FNT_2n per codeword (the middle product of
// step 5 and the product by A of step 6, each three FNT_2n with one transform
// precomputed).  This file runs that route on the GPU, for comparison with the
// library's default decode (3 FNT_n per codeword, see kernels.cuh):
//   per pattern  step 3 by the chirp: A'(r^i) = b_i^-1 sum_j (a'_j / b_j) b_(i+j),
//                read off coefficients n-1+i of (sum_j c_j x^(n-1-j)) * (sum b_i x^i),
//                c_j = a'_j / b_j; the weights 1/A'(x_i) of step 4 follow;
//   per codeword step 5: N'(q^m) = b'_m^-1 sum_z (n_z / b'_z) b'_(m+z) with
//                q = r^-1, b'_i = q^(t_i), n_z = v_i / A'(x_i) at z = z_i (the same
//                middle product, length 2n), S_j = -N'(q^(j+1)), j < k;
//                step 6: P = (A S) mod x^k by FNT_2n.
// The cyclic products have length 2n: the wrapped terms of a product of
// degree <= 3n - 2 land on coefficients 0 .. n-2, below the ones read.
// Needs a root of order 2n (n <= 32768) and k <= n/2 (A mod x^k then has a
// length-n transform the pattern tables already hold).
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

constexpr uint32_t kP32 = 65537u;

uint32_t h_pow(uint32_t a, uint64_t e) {
  uint64_t r = 1, x = a % kP32;
  while (e) {
    if (e & 1) r = r * x % kP32;
    x = x * x % kP32;
    e >>= 1;
  }
  return (uint32_t)r;
}
uint32_t h_inv(uint32_t a) { return h_pow(a, kP32 - 2); }

unsigned grid_for(const fnt_rs_plan_s* p, size_t work) {
  const size_t want = (work + 255) / 256;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)p->sms * 8));
}

// a_i = nc * X_i (X = n^-1 times the coefficients of A mod x^k).  G (2n):
// G[n-1-j] = c_j = a'_j / b_j for j < n (a'_j = (j+1) a_(j+1), a'_(k-1) = k from
// the monic x^k term), G[n..2n) = 0.  Z (2n): the coefficients of A mod x^k.
__global__ void k_pap_deriv(const uint32_t* __restrict__ X, uint32_t n, uint32_t k, uint32_t nc,
                            const uint32_t* __restrict__ binv, uint32_t* __restrict__ G,
                            uint32_t* __restrict__ Z) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * n; t += gridDim.x * blockDim.x) {
    uint32_t g = 0;
    if (t < n) {
      const uint32_t j = n - 1 - t;
      if (j + 1 < k)
        g = p_mul(p_mul(p_mul(nc, X[j + 1]), j + 1), binv[j]);
      else if (j + 1 == k)
        g = p_mul(k % kP, binv[j]);
    }
    G[t] = g;
    Z[t] = t < k ? p_mul(nc, X[t]) : 0u;
  }
}

// y[r][c] = y[r][c] * tab[r] (canonical)
__global__ void k_pap_mul_rows(uint32_t* __restrict__ y, size_t ld, const uint32_t* __restrict__ tab,
                               uint32_t rows, uint32_t W) {
  const size_t total = (size_t)rows * W;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / W, c = t % W;
    uint32_t* v = y + r * ld + c;
    *v = p_mul(*v, __ldg(tab + r));
  }
}

// Step 4 weights from the chirp product Y (2n): A'(r^z) = Y[n-1+z] / b_z;
// wg[i] = 1 / (A'(x_i) b'_z) for z = pos[i]; pmap[n-1-z] = i.
__global__ void k_pap_weights(const uint32_t* __restrict__ Y, uint32_t n, uint32_t k,
                              const uint32_t* __restrict__ pos, const uint32_t* __restrict__ binv,
                              const uint32_t* __restrict__ bqinv, uint32_t* __restrict__ wg,
                              uint32_t* __restrict__ pmap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const uint32_t z = pos[i];
    const uint32_t d = p_mul(Y[n - 1 + z], binv[z]);
    wg[i] = p_mul(p_inv(d), bqinv[z]);
    pmap[n - 1 - z] = i;
  }
}

// G[r][c] (r < 2n): n_z / b'_z at r = n-1-z for a received z (one of the first
// k positions), else 0.  Received values above 65536 raise the range flag.
__global__ void k_pap_gather(const uint32_t* __restrict__ recv, size_t ld_recv, int slots,
                             const uint32_t* __restrict__ pmap, const uint32_t* __restrict__ wg,
                             uint32_t n, uint32_t W, uint32_t* __restrict__ G, size_t ld,
                             int* status) {
  const size_t total = (size_t)2 * n * W;
  bool bad = false;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(t / W), c = (uint32_t)(t % W);
    uint32_t v = 0;
    if (r < n) {
      const uint32_t i = __ldg(pmap + r);
      if (i != 0xFFFFFFFFu) {
        const size_t row = slots ? (size_t)(n - 1 - r) : (size_t)i;
        const uint32_t x = recv[row * ld_recv + c];
        bad |= x > 65536u;
        v = p_mul(x, __ldg(wg + i));
      }
    }
    G[(size_t)r * ld + c] = v;
  }
  if (bad) atomicOr(status, ST_RANGE);
}

// F[j][c] = S_j = -N'(q^(j+1)) = Y[n+j][c] * sc[j] for j < k, 0 for k <= j < 2n
__global__ void k_pap_extract(const uint32_t* __restrict__ Y, uint32_t* __restrict__ F, size_t ld,
                              uint32_t n, uint32_t k, const uint32_t* __restrict__ sc, uint32_t W) {
  const size_t total = (size_t)2 * n * W;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t j = t / W, c = t % W;
    F[j * ld + c] = j < k ? p_mul(Y[(n + j) * ld + c], __ldg(sc + j)) : 0u;
  }
}

// out[j][c] = P_j for j < k: 16-bit symbols (65536 -> 0 with the range flag)
// or, with out32, the coefficients as u32
__global__ void k_pap_out(const uint32_t* __restrict__ F, size_t ld, uint32_t k, uint32_t W,
                          uint16_t* __restrict__ out, size_t ld_out, uint32_t* __restrict__ out32,
                          int* status) {
  const size_t total = (size_t)k * W;
  bool bad = false;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t j = t / W, c = t % W;
    const uint32_t v = F[j * ld + c];
    if (out32) {
      out32[j * ld_out + c] = v;
    } else {
      bad |= v > 65535u;
      out[j * ld_out + c] = (uint16_t)(v > 65535u ? 0u : v);
    }
  }
  if (bad) atomicOr(status, ST_RANGE);
}

}  // namespace

// Per-plan state of the route: the length-2n helper plan (its transforms),
// the chirp tables and, per pattern slot, the step 4-6 tables.
struct PaperSlotTabs {
  std::vector<uint32_t> key;
  bool ready = false;
  uint32_t* pmap = nullptr;  // [n]: received index i at row n-1-z_i, else ~0
  uint32_t* wg = nullptr;    // [k]: 1 / (A'(x_i) b'_(z_i))
  uint32_t* ahat2 = nullptr; // [2n]: FNT_2n(A mod x^k)
};

struct PaperState {
  fnt_rs_plan_s* p2 = nullptr;
  uint32_t* binv = nullptr;   // [n] 1 / b_i
  uint32_t* bqinv = nullptr;  // [n] 1 / b'_z
  uint32_t* sc = nullptr;     // [n] -1 / b'_(j+1)
  uint32_t* hr = nullptr;     // [2n] FNT_2n(b_0 .. b_(2n-1))
  uint32_t* hq = nullptr;     // [2n] FNT_2n(b'_0 .. b'_(2n-1))
  uint32_t* X = nullptr;      // per-pattern scratch: [n] | G [2n] | F [2n] | Z [2n] | pos [n]
  uint32_t* G = nullptr;
  uint32_t* F = nullptr;
  uint32_t* Z = nullptr;
  uint32_t* pos = nullptr;
  void* work = nullptr;       // helper-plan transform scratch for one column
  PaperSlotTabs tabs[kPatternSlots + 1];
};

bool paper_available(const fnt_rs_plan_s* p) {
  return p->n >= 2 && p->n <= 32768 && !p->blocked && p->u == 1;
}

void paper_free(fnt_rs_plan_s* p) {
  PaperState* s = p->paper;
  if (!s) return;
  cudaFree(s->binv);
  cudaFree(s->X);
  cudaFree(s->work);
  for (auto& t : s->tabs) cudaFree(t.pmap);
  if (s->p2) fnt_rs_plan_destroy(s->p2);
  delete s;
  p->paper = nullptr;
}

size_t paper_ws_bytes(const fnt_rs_plan_s* p, size_t W) {
  if (!p->paper || W == 0) return 0;
  const size_t n2 = 2 * (size_t)p->n;
  return 2 * align256(n2 * W * 4) + align256(fnt_columns_work_bytes(p->paper->p2, W));
}

int paper_enable(fnt_rs_plan_s* p, cudaStream_t st) {
  if (p->paper) return FNT_RS_OK;
  if (!paper_available(p)) return FNT_RS_E_ARG;
  const uint32_t n = p->n, k = p->k, n2 = 2 * n;
  PaperState* s = new PaperState();
  p->paper = s;
  auto fail = [&](int rc) {
    paper_free(p);
    return rc;
  };
  int rc = fnt_rs_plan_create(&s->p2, n2, 1, FNT_RS_P, 0, st);
  if (rc) return fail(rc);
  // chirp tables: b_i = r^(t_i), b'_i = r^(-t_i), t_i = i(i-1)/2 (exponents mod n)
  const uint32_t r = h_pow(3, 65536u / n);
  std::vector<uint32_t> br(n2), bq(n2), host(5 * (size_t)n);
  for (uint32_t i = 0; i < n2; ++i) {
    const uint64_t t = (i ? (uint64_t)i * (i - 1) / 2 : 0) % n;
    br[i] = h_pow(r, t);
    bq[i] = h_pow(r, (n - t) % n);
  }
  uint32_t* binv = host.data();
  uint32_t* bqinv = binv + n;
  uint32_t* sc = bqinv + n;
  for (uint32_t i = 0; i < n; ++i) {
    binv[i] = h_inv(br[i]);
    bqinv[i] = h_inv(bq[i]);
    sc[i] = (kP32 - h_inv(bq[i + 1])) % kP32;
  }
  // device: binv | bqinv | sc | hr | hq (3n + 4n words)
  if ((rc = cuda_ok(cudaMalloc(&s->binv, (size_t)7 * n * 4)))) return fail(rc);
  s->bqinv = s->binv + n;
  s->sc = s->bqinv + n;
  s->hr = s->sc + n;
  s->hq = s->hr + n2;
  if ((rc = cuda_ok(cudaMalloc(&s->X, ((size_t)n + 3 * (size_t)n2 + n) * 4)))) return fail(rc);
  s->G = s->X + n;
  s->F = s->G + n2;
  s->Z = s->F + n2;
  s->pos = s->Z + n2;
  const size_t wb = fnt_columns_work_bytes(s->p2, 1);
  if (wb && (rc = cuda_ok(cudaMalloc(&s->work, wb)))) return fail(rc);
  for (auto& t : s->tabs) {
    if ((rc = cuda_ok(cudaMalloc(&t.pmap, ((size_t)n + k + n2) * 4)))) return fail(rc);
    t.wg = t.pmap + n;
    t.ahat2 = t.wg + k;
  }
  if ((rc = cuda_ok(cudaMemcpyAsync(s->binv, host.data(), (size_t)3 * n * 4,
                                    cudaMemcpyHostToDevice, st))))
    return fail(rc);
  if ((rc = cuda_ok(cudaMemcpyAsync(s->G, br.data(), (size_t)n2 * 4, cudaMemcpyHostToDevice, st))))
    return fail(rc);
  if ((rc = cuda_ok(cudaMemcpyAsync(s->F, bq.data(), (size_t)n2 * 4, cudaMemcpyHostToDevice, st))))
    return fail(rc);
  if ((rc = fnt_columns(s->p2, s->G, 1, s->hr, 1, 1, false, s->work, st))) return fail(rc);
  if ((rc = fnt_columns(s->p2, s->F, 1, s->hq, 1, 1, false, s->work, st))) return fail(rc);
  if ((rc = cuda_ok(cudaStreamSynchronize(st)))) return fail(rc);  // host vectors go away
  return FNT_RS_OK;
}

namespace {

// Step 3 by the chirp and the step 4-6 tables of the pattern in `sl`.
int paper_tables(fnt_rs_plan_s* p, const PatternSlot& sl, PaperSlotTabs& t, cudaStream_t st) {
  PaperState* s = p->paper;
  const uint32_t n = p->n, k = p->k, n2 = 2 * n;
  std::vector<uint32_t> key = sl.key;
  if (&sl == &p->sys) {
    key.resize(k);
    for (uint32_t i = 0; i < k; ++i) key[i] = i;
  }
  if (t.ready && t.key == key) return FNT_RS_OK;
  t.ready = false;
  int rc = cuda_ok(cudaMemcpyAsync(s->pos, key.data(), (size_t)k * 4, cudaMemcpyHostToDevice, st));
  if (rc) return rc;
  // coefficients of A mod x^k from the pattern's n^-1 FNT_n(A mod x^k)
  if ((rc = fnt_columns(p, sl.ahat, 1, s->X, 1, 1, true, nullptr, st))) return rc;
  k_pap_deriv<<<grid_for(p, n2), 256, 0, st>>>(s->X, n, k, n % kP32, s->binv, s->G, s->Z);
  count_launch();
  // chirp product: Y = IFNT_2n(FNT_2n(G) * FNT_2n(b))
  if ((rc = fnt_columns(s->p2, s->G, 1, s->F, 1, 1, false, s->work, st))) return rc;
  k_pap_mul_rows<<<grid_for(p, n2), 256, 0, st>>>(s->F, 1, s->hr, n2, 1);
  count_launch();
  if ((rc = fnt_columns(s->p2, s->F, 1, s->G, 1, 1, true, s->work, st))) return rc;
  if ((rc = cuda_ok(cudaMemsetAsync(t.pmap, 0xFF, (size_t)n * 4, st)))) return rc;
  k_pap_weights<<<grid_for(p, k), 256, 0, st>>>(s->G, n, k, s->pos, s->binv, s->bqinv, t.wg,
                                                 t.pmap);
  count_launch();
  // step 6 multiplier: FNT_2n(A mod x^k)
  if ((rc = fnt_columns(s->p2, s->Z, 1, t.ahat2, 1, 1, false, s->work, st))) return rc;
  if ((rc = cuda_ok(cudaGetLastError()))) return rc;
  t.key.swap(key);
  t.ready = true;
  return FNT_RS_OK;
}

}  // namespace

int paper_decode(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv, size_t ld_recv,
                 uint16_t* out, size_t ld_out, size_t W, void* workspace, cudaStream_t st,
                 int slots, uint32_t* out32) {
  PaperState* s = p->paper;
  if (!s) return FNT_RS_E_ARG;
  if (!workspace) return FNT_RS_E_WORKSPACE;
  const ptrdiff_t idx = &sl == &p->sys ? kPatternSlots : &sl - p->slots;
  if (idx < 0 || idx > kPatternSlots) return FNT_RS_E_ARG;
  PaperSlotTabs& t = s->tabs[idx];
  int rc = paper_tables(p, sl, t, st);
  if (rc) return rc;
  const uint32_t n = p->n, k = p->k, n2 = 2 * n;
  const size_t buf = align256((size_t)n2 * W * 4);
  uint32_t* G = static_cast<uint32_t*>(workspace);
  uint32_t* F = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(workspace) + buf);
  void* work = static_cast<uint8_t*>(workspace) + 2 * buf;
  const unsigned g2 = grid_for(p, (size_t)n2 * W);
  // step 4 + step 5 as a middle product at length 2n
  k_pap_gather<<<g2, 256, 0, st>>>(recv, ld_recv, slots, t.pmap, t.wg, n, (uint32_t)W, G, W,
                                   p->status);
  count_launch();
  if ((rc = fnt_columns(s->p2, G, W, F, W, W, false, work, st))) return rc;
  k_pap_mul_rows<<<g2, 256, 0, st>>>(F, W, s->hq, n2, (uint32_t)W);
  count_launch();
  if ((rc = fnt_columns(s->p2, F, W, G, W, W, true, work, st))) return rc;
  k_pap_extract<<<g2, 256, 0, st>>>(G, F, W, n, k, s->sc, (uint32_t)W);
  count_launch();
  // step 6: P = (A S) mod x^k
  if ((rc = fnt_columns(s->p2, F, W, G, W, W, false, work, st))) return rc;
  k_pap_mul_rows<<<g2, 256, 0, st>>>(G, W, t.ahat2, n2, (uint32_t)W);
  count_launch();
  if ((rc = fnt_columns(s->p2, G, W, F, W, W, true, work, st))) return rc;
  k_pap_out<<<grid_for(p, (size_t)k * W), 256, 0, st>>>(F, W, k, (uint32_t)W, out, ld_out, out32,
                                                        p->status);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

}  // namespace fntrs
