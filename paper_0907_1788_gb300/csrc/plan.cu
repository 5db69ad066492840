// Host side of libfntrs: plans, twiddle tables, pattern cache, dispatch and
// the C ABI declared in include/fnt_rs.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/fnt_rs.h"
#include "dbg.cuh"
#include "internal.h"
#include "kargs.h"
#include "sched.h"

namespace fntrs {

// ---------------------------------------------------------------------------
// launch counter and tile-op registry
// ---------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static TileOps g_ops[17];
static std::once_flag g_ops_once;

void register_ops(const TileOps& ops) {
  int b = 0;
  while ((1 << b) < ops.L) ++b;
  g_ops[b] = ops;
}

static void init_ops() {
  std::call_once(g_ops_once, [] {
    register_tile_ops_small();
    register_tile_ops_mid();
    register_tile_ops_big();
    register_tile_ops_huge();
  });
}

const TileOps& tile_ops(int L) {
  init_ops();
  int b = 0;
  while ((1 << b) < L) ++b;
  return g_ops[b];
}

int launch_encode_tma_small(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st);
int launch_encode_tma_mid(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st);
int launch_encode_tma_big(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st);
// n = 8192 with k > 4096: the two classes fold two source rows (inst_fold.cu)
int launch_encode_tma_fold(const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st);

int launch_decode_tma_small(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st);
int launch_decode_tma_mid(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st);
int launch_decode_tma_big(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st);

int launch_decode_tma(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  if (L <= 256) return launch_decode_tma_small(L, a, t, st);
  if (L <= 2048) return launch_decode_tma_mid(L, a, t, st);
  return launch_decode_tma_big(L, a, t, st);
}

int launch_encode_tma(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  if (L <= 256) return launch_encode_tma_small(L, C, a, t, st);
  if (L <= 2048) return launch_encode_tma_mid(L, C, a, t, st);
  return launch_encode_tma_big(L, C, a, t, st);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  });
  return fn;
}

void launch_lg_init(uint2* pat, uint32_t* ind, int n, cudaStream_t st);
void launch_lg_scatter(const uint32_t* pos, int k, uint2* pat, uint32_t* ind, cudaStream_t st);
void launch_lg_mul(const uint32_t* spec, const uint32_t* ghat, int D, int n, uint32_t* P,
                   cudaStream_t st);
void launch_lg_final(const uint32_t* conv, int D, int b, int n, int k, const uint32_t* exp3,
                     uint32_t ninv, uint2* pat, uint32_t* pat32, uint32_t* aval, uint32_t* ahat,
                     uint32_t* rowtab, cudaStream_t st);
void launch_pat32(const uint2* pat, uint32_t* pat32, uint32_t* rowtab, int n, cudaStream_t st);
void launch_lg_halves(const uint32_t* coef, int n, int k, uint32_t* M, cudaStream_t st);
void launch_lg_scale2(const uint32_t* E, int n, uint32_t ninv, uint32_t* ahat, uint32_t* ahat2,
                      cudaStream_t st);
void launch_pat_init(uint2* pat, int n, cudaStream_t st);
void launch_leaves(const uint32_t* pos, int k, const uint32_t* powf, uint32_t* out, int nodes,
                   cudaStream_t st);
void launch_big_pack(const uint32_t* lvl, int d, int nodes, int L, uint32_t* M, cudaStream_t st);
void launch_big_mul(const uint32_t* Mh, int npairs, int L, uint32_t* Q, cudaStream_t st);
void launch_big_fix(const uint32_t* Q, int d, int k, int npairs, int L, uint32_t* out,
                    cudaStream_t st);
void launch_pat_prep(const uint32_t* A, int k, int n, int ncols, int h, uint32_t* M,
                     cudaStream_t st);
void launch_pat_final(const uint32_t* E, int ncols, const uint32_t* pos, int k, int n,
                      const uint32_t* powi, uint32_t ninv, uint2* pat, uint32_t* ahat,
                      uint32_t* ahat2, cudaStream_t st);

// ---------------------------------------------------------------------------
// F_p helpers on the host (plan tables)
// ---------------------------------------------------------------------------
static uint32_t hmul(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) % FNT_RS_P); }
static uint32_t hpow(uint32_t a, uint64_t e) {
  uint64_t r = 1, b = a % FNT_RS_P;
  while (e) {
    if (e & 1) r = r * b % FNT_RS_P;
    b = b * b % FNT_RS_P;
    e >>= 1;
  }
  return (uint32_t)r;
}
uint32_t hinv(uint32_t a) { return hpow(a, FNT_RS_P - 2); }
static int ilog2i(uint32_t v) {
  int b = 0;
  while ((1u << b) < v) ++b;
  return b;
}
static int bitrev_h(int v, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
  return r;
}
// default root of order n: 3^(65536/n) (Sec. II.B)
static uint32_t default_root(uint32_t n) { return hpow(3, 65536u / n); }

// ---------------------------------------------------------------------------
// Device tables per transform length L (default root), shared by all plans
// on a device: per-pass schedule tables and the powers r_L^e, r_L^-e.
// ---------------------------------------------------------------------------

static std::mutex g_tab_mu;
static std::map<std::pair<int, int>, Tables> g_tables;

static std::vector<uint32_t> sched_table(int L, bool inverse) {
  int r[3];
  sched_radices(L, r);
  std::vector<uint32_t> out;
  if (r[1] == 1) return out;  // single pass: no twiddles
  uint32_t w = default_root(L);
  if (inverse) w = hinv(w);
  const int S1 = L / r[0];
  out.resize(L + (r[2] > 1 ? S1 : 0));
  const int b0 = ilog2i(r[0]);
  for (int i2 = 0; i2 < S1; ++i2)
    for (int q = 0; q < r[0]; ++q)
      out[(size_t)i2 * r[0] + q] = hpow(w, (uint64_t)i2 * bitrev_h(q, b0) % L);
  if (r[2] > 1) {
    const uint32_t w2 = hpow(w, r[0]);  // root of order S1
    const int S2 = S1 / r[1], b1 = ilog2i(r[1]);
    for (int i2 = 0; i2 < S2; ++i2)
      for (int q = 0; q < r[1]; ++q)
        out[L + (size_t)i2 * r[1] + q] = hpow(w2, (uint64_t)i2 * bitrev_h(q, b1) % S1);
  }
  return out;
}

// The pass-1 part of the forward table (L entries, row i2 = the R1 entries of
// task i2) with the 16-byte chunks of each row permuted: chunk u of row i2 at
// chunk u ^ (i2 mod R1/4).  Copied into shared memory by the staged decode,
// whose warps read chunk u of 32/WT consecutive rows at once: the permutation
// puts those reads in different banks.
static std::vector<uint32_t> sched_table_swizzled(int L) {
  int r[3];
  sched_radices(L, r);
  const std::vector<uint32_t> t = sched_table(L, false);
  std::vector<uint32_t> out;
  const int R = r[0], S1 = L / R, nch = R / 4;
  if (t.empty() || R < 4) return out;
  out.resize(L);
  for (int i2 = 0; i2 < S1; ++i2)
    for (int u = 0; u < nch; ++u)
      for (int e = 0; e < 4; ++e)
        out[(size_t)i2 * R + 4 * (u ^ (i2 % nch)) + e] = t[(size_t)i2 * R + 4 * u + e];
  return out;
}

static int upload(uint32_t** dst, const std::vector<uint32_t>& v) {
  const size_t bytes = std::max<size_t>(16, v.size() * sizeof(uint32_t));
  if (cudaMalloc(dst, bytes) != cudaSuccess) return FNT_RS_E_CUDA;
  if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return FNT_RS_E_CUDA;
  return FNT_RS_OK;
}

int get_tables(int L, Tables* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FNT_RS_E_CUDA;
  std::lock_guard<std::mutex> lk(g_tab_mu);
  auto it = g_tables.find({dev, L});
  if (it != g_tables.end()) {
    *out = it->second;
    return FNT_RS_OK;
  }
  Tables t;
  std::vector<uint32_t> pf(L), pi(L);
  const uint32_t r = default_root(L), ri = hinv(r);
  uint32_t a = 1, b = 1;
  for (int e = 0; e < L; ++e) {
    pf[e] = a;
    pi[e] = b;
    a = hmul(a, r);
    b = hmul(b, ri);
  }
  int rc;
  if ((rc = upload(&t.powf, pf)) || (rc = upload(&t.powi, pi))) return rc;
  if (L <= kTileMaxL) {
    if ((rc = upload(&t.twf, sched_table(L, false))) || (rc = upload(&t.twi, sched_table(L, true))))
      return rc;
    if (L >= 4096 && (rc = upload(&t.twf_sw, sched_table_swizzled(L)))) return rc;
  }
  g_tables[{dev, L}] = t;
  *out = t;
  return FNT_RS_OK;
}

// 3^e mod p for e < 65536 (3 is a primitive root, Sec. II.A), one table per device.
static std::mutex g_exp_mu;
static std::map<int, uint32_t*> g_exp3;

static int get_exp3(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FNT_RS_E_CUDA;
  std::lock_guard<std::mutex> lk(g_exp_mu);
  auto it = g_exp3.find(dev);
  if (it != g_exp3.end()) {
    *out = it->second;
    return FNT_RS_OK;
  }
  std::vector<uint32_t> t(65536);
  uint32_t x = 1;
  for (int e = 0; e < 65536; ++e) {
    t[e] = x;
    x = hmul(x, 3);
  }
  uint32_t* d = nullptr;
  int rc = upload(&d, t);
  if (rc) return rc;
  g_exp3[dev] = d;
  *out = d;
  return FNT_RS_OK;
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------


}  // namespace fntrs

using namespace fntrs;


namespace fntrs {

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? FNT_RS_OK : FNT_RS_E_CUDA; }

// columns per chunk of a split transform with `nbuf` [n][Wc] workspace buffers
size_t split_chunk(uint32_t n, int nbuf) {
  size_t wc = kChunkBudget / ((size_t)nbuf * n * 4);
  wc = std::max<size_t>(8, wc / 8 * 8);
  return wc;
}

// Schedules.  Encode: TMA-staged tile (n <= 8192 when the TMA shape exists),
// one-CTA tile (n <= 32768), two-pass split (n > 8192).  Decode: TMA-staged
// tile (64 <= n <= 8192, k <= n/2), one-CTA tile (n <= 16384, or n = 32768
// with k <= n/2), split passes (n >= 16384).  All give the same words.
bool sched_available(const fnt_rs_plan_s* p, int op, int s) {
  const uint32_t n = p->n;
  if (op == FNT_RS_OP_ENCODE) {
    switch (s) {
      case FNT_RS_SCHED_TMA: return p->enc_L != 0 && p->u == 1 && !p->no_tma;
      case FNT_RS_SCHED_TILE: return n <= (uint32_t)kTileMaxL;
      case FNT_RS_SCHED_SPLIT: return n > 8192;
      case FNT_RS_SCHED_DIRECT: return direct_available(p);
      default: return false;
    }
  }
  if (op == FNT_RS_OP_DECODE) {
    switch (s) {
      case FNT_RS_SCHED_TMA: return n >= 64 && n <= 8192 && !p->blocked && !p->no_tma;
      case FNT_RS_SCHED_CPA: return tile_ops((int)n).decode_cpa != nullptr && !p->blocked &&
                                    !p->split;
      case FNT_RS_SCHED_TILE: return !p->split;
      case FNT_RS_SCHED_SPLIT: return n >= 16384;
      case FNT_RS_SCHED_PAPER: return paper_available(p);
      case FNT_RS_SCHED_DIRECT: return direct_available(p);
      default: return false;
    }
  }
  return false;
}

int sched_effective(const fnt_rs_plan_s* p, int op) {
  const int chosen = op == FNT_RS_OP_ENCODE ? p->sched_enc : p->sched_dec;
  if (chosen) return chosen;
  if (op == FNT_RS_OP_ENCODE) {
    if (sched_available(p, op, FNT_RS_SCHED_TMA)) return FNT_RS_SCHED_TMA;
    return p->n <= 8192 ? FNT_RS_SCHED_TILE : FNT_RS_SCHED_SPLIT;
  }
  if (sched_available(p, op, FNT_RS_SCHED_TMA)) return FNT_RS_SCHED_TMA;
  // n = 16384: the staged two-codeword tile beats the direct loads (11-12% measured)
  if (p->n == 16384 && sched_available(p, op, FNT_RS_SCHED_CPA)) return FNT_RS_SCHED_CPA;
  return p->split ? FNT_RS_SCHED_SPLIT : FNT_RS_SCHED_TILE;
}

int enc_nbuf(const fnt_rs_plan_s* p) {
  return sched_effective(p, FNT_RS_OP_ENCODE) == FNT_RS_SCHED_SPLIT ? 1 : 0;
}
int dec_nbuf(const fnt_rs_plan_s* p) {
  return sched_effective(p, FNT_RS_OP_DECODE) == FNT_RS_SCHED_SPLIT ? (p->blocked ? 4 : 2) : 0;
}
int enc_nbuf_max(const fnt_rs_plan_s* p) { return p->n > 8192 ? 1 : 0; }
int dec_nbuf_max(const fnt_rs_plan_s* p) { return p->n >= 16384 ? (p->blocked ? 4 : 2) : 0; }
int fnt_nbuf(const fnt_rs_plan_s* p) { return p->split ? 1 : 0; }

size_t dec_ws_now(const fnt_rs_plan_s* p, size_t W) {
  const int s = sched_effective(p, FNT_RS_OP_DECODE);
  if (s == FNT_RS_SCHED_PAPER) return paper_ws_bytes(p, W);
  if (s == FNT_RS_SCHED_DIRECT) return direct_ws_bytes(p, W);
  return ws_bytes(p, W, dec_nbuf(p));
}
size_t dec_ws_max(const fnt_rs_plan_s* p, size_t W) {
  return std::max({ws_bytes(p, W, dec_nbuf_max(p)), paper_ws_bytes(p, W), direct_ws_bytes(p, W)});
}

static bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

size_t ws_bytes(const fnt_rs_plan_s* p, size_t W, int nbuf) {
  if (nbuf == 0 || W == 0) return 0;
  const size_t wc = std::min(W, split_chunk(p->n, nbuf));
  return (size_t)nbuf * p->n * wc * 4;
}

// Batched transform of an [L][W] u32 matrix with the default root of order L,
// out = (inverse ? L^-1 : 1) * scale_extra * FNT(in), values reduced.
// For L above the tile limit the caller provides `work` of L*W words.
static int run_fnt_default(int L, const uint32_t* in, size_t ld_in, uint32_t* out, size_t ld_out,
                           int W, bool inverse, uint32_t row_mul, uint32_t* work,
                           cudaStream_t st) {
  Tables t;
  int rc = get_tables(L, &t);
  if (rc) return rc;
  const uint32_t scale = inverse ? hinv((uint32_t)L % FNT_RS_P) : 1u;
  if (L <= kTileMaxL) {
    const TileOps& ops = tile_ops(L);
    KArgs a;
    a.in = in;
    a.ld_in = ld_in;
    a.out = out;
    a.ld_out = ld_out;
    a.W = W;
    a.n = L;
    a.L = L;
    a.C = 1;
    a.scale = scale;
    a.twf = t.twf;
    a.twi = t.twi;
    (inverse ? a.in_row_mul : a.row_mul) = row_mul;
    (inverse ? ops.fnt_inv : ops.fnt_fwd)(a, 1, st);
    return cuda_ok(cudaGetLastError());
  }
  Tables tl;
  if ((rc = get_tables(kLocalL, &tl))) return rc;
  const int C = L / kLocalL;
  KArgs a;
  a.in = in;
  a.ld_in = ld_in;
  a.out = out;
  a.ld_out = ld_out;
  a.out2 = work;
  a.ld_work = (size_t)W;
  a.W = W;
  a.n = L;
  a.L = kLocalL;
  a.C = C;
  a.row_limit = L;
  a.scale = scale;
  a.powf = t.powf;
  a.powi = t.powi;
  (inverse ? a.in_row_mul : a.row_mul) = row_mul;
  cross_launcher(C, inverse, CL_U32)(a, 1, st);
  KArgs b = a;
  b.in = work;
  b.ld_in = (size_t)W;
  b.twf = tl.twf;
  b.twi = tl.twi;
  local_launcher(inverse, LM_FNT)(b, C, st);
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// pattern build (steps 1-3) into slot `si`
// ---------------------------------------------------------------------------
size_t pattern_scratch_words(uint32_t n, uint32_t k) {
  // product tree: level ping-pong, [n][3] matrix + transform, big-level matrices + work
  size_t K2 = 1;
  while (K2 < k) K2 <<= 1;
  const size_t lvl = 4 * (size_t)k + 4 * 64 + 2 * K2 + 64;
  const size_t big = (K2 > (size_t)kTreeTileL / 2) ? 8 * (size_t)(2 * K2) + 8 * K2 : 0;
  const size_t tree = 2 * lvl + 9 * (size_t)n + big + 1024;
  // log route: ind, spec, aval, coef (n each), M2, E2 (2n each), P, conv, work (n*16 each)
  const size_t lg = 8 * (size_t)n + 3 * 16 * (size_t)n + 1024;
  return std::max(tree, lg);
}

int alloc_pattern_tables(PatternSlot& sl, size_t n, bool staging) {
  if (cudaMalloc(&sl.pat, n * sizeof(uint2)) != cudaSuccess ||
      cudaMalloc(&sl.ahat, n * 4) != cudaSuccess || cudaMalloc(&sl.ahat2, n * 4) != cudaSuccess ||
      cudaMalloc(&sl.pos_d, n * 4) != cudaSuccess || cudaMalloc(&sl.pat32, n * 4) != cudaSuccess ||
      cudaMalloc(&sl.rowtab, n * 4) != cudaSuccess ||
      cudaMalloc(&sl.done, 4) != cudaSuccess || cudaMemset(sl.done, 0, 4) != cudaSuccess)
    return FNT_RS_E_CUDA;
  if (staging && (cudaMallocHost(&sl.pos_h, n * 4) != cudaSuccess ||
                  cudaEventCreateWithFlags(&sl.staged, cudaEventDisableTiming) != cudaSuccess))
    return FNT_RS_E_CUDA;
  if (staging) {
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, sl.pos_h, 0) == cudaSuccess)
      sl.pos_map = static_cast<const uint32_t*>(dp);
    else
      cudaGetLastError();  // not mapped: positions go through pos_d
  }
  return FNT_RS_OK;
}

void free_pattern_tables(PatternSlot& sl) {
  cudaFree(sl.pat);
  cudaFree(sl.ahat);
  cudaFree(sl.ahat2);
  cudaFree(sl.pos_d);
  cudaFree(sl.pat32);
  cudaFree(sl.rowtab);
  cudaFree(sl.done);
  if (sl.pos_h) cudaFreeHost(sl.pos_h);
  if (sl.staged) cudaEventDestroy(sl.staged);
  sl = PatternSlot{};
}

// Log-domain build of the pattern tables (see pattern.cu); `scratch` holds
// pattern_scratch_words(n, k) words (the plan's own scratch when null).
bool fused_plan_applies(const fnt_rs_plan_s* p) {
  return !p->plan_tree && !p->split && tile_ops((int)p->n).plan_fused != nullptr;
}

int build_pattern_log(fnt_rs_plan_s* p, PatternSlot& sl, cudaStream_t st, uint32_t* scratch,
                      const uint32_t* pos) {
  const int n = (int)p->n, k = (int)p->k, D = p->lg_D;
  uint32_t* ind = scratch ? scratch : p->pscratch;
  uint32_t* spec = ind + n;
  uint32_t* aval = spec + n;
  uint32_t* coef = aval + n;
  uint32_t* M2 = coef + n;
  uint32_t* E2 = M2 + 2 * (size_t)n;
  uint32_t* P = E2 + 2 * (size_t)n;
  uint32_t* conv = P + 16 * (size_t)n;
  uint32_t* work = conv + 16 * (size_t)n;
  int rc;
  const TileOps& ops = tile_ops(n);
  if (!p->split && ops.plan_fused) {
    PlanArgs pa;
    pa.k = k;
    pa.D = D;
    pa.b = p->lg_b;
    pa.ninv = p->ninv;
    pa.twf = p->tn.twf;
    pa.twi = p->tn.twi;
    pa.pos = pos ? pos : sl.pos_d;
    pa.ghat = p->ghat;
    pa.exp3 = p->exp3;
    pa.conv = conv;
    pa.pat = sl.pat;
    pa.pat32 = sl.pat32;
    pa.rowtab = sl.rowtab;
    pa.aval = p->blocked ? aval : nullptr;
    pa.ahat = p->blocked ? nullptr : sl.ahat;
    pa.done = sl.done;
    pa.status = p->status;
    ops.plan_fused(pa, st);
    if (!p->blocked) return cuda_ok(cudaGetLastError());
  } else {
    launch_lg_init(sl.pat, ind, n, st);
    launch_lg_scatter(sl.pos_d, k, sl.pat, ind, st);
    if ((rc = run_fnt_default(n, ind, 1, spec, 1, 1, false, 1, work, st))) return rc;
    launch_lg_mul(spec, p->ghat, D, n, P, st);
    if ((rc = run_fnt_default(n, P, D, conv, D, D, true, 1, work, st))) return rc;
    if (!p->blocked) {
      launch_lg_final(conv, D, p->lg_b, n, k, p->exp3, p->ninv, sl.pat, sl.pat32, nullptr,
                      sl.ahat, sl.rowtab, st);
      return cuda_ok(cudaGetLastError());
    }
    launch_lg_final(conv, D, p->lg_b, n, k, p->exp3, p->ninv, sl.pat, sl.pat32, aval, nullptr,
                    sl.rowtab, st);
  }
  if ((rc = run_fnt_default(n, aval, 1, coef, 1, 1, true, 1, work, st))) return rc;
  launch_lg_halves(coef, n, k, M2, st);
  if ((rc = run_fnt_default(n, M2, 2, E2, 2, 2, false, 1, work, st))) return rc;
  launch_lg_scale2(E2, n, p->ninv, sl.ahat, sl.ahat2, st);
  return cuda_ok(cudaGetLastError());
}

int build_pattern(fnt_rs_plan_s* p, PatternSlot& sl, cudaStream_t st) {
  const int n = (int)p->n, k = (int)p->k;
  uint32_t* base = p->pscratch;
  size_t K2 = 1;
  while (K2 < (size_t)k) K2 <<= 1;
  const size_t lvl_words = 4 * (size_t)k + 4 * 64 + 2 * K2 + 64;
  uint32_t* lv[2] = {base, base + lvl_words};
  uint32_t* M = base + 2 * lvl_words;
  uint32_t* E = M + 3 * (size_t)n;
  uint32_t* work = E + 3 * (size_t)n;        // 3n words: split-transform work of the pattern FNT
  uint32_t* big = work + 3 * (size_t)n;       // big-level matrices
  int rc;
  launch_pat_init(sl.pat, n, st);
  // step 1: leaves (up to 32 factors per node) then pairwise FNT products
  int nodes = (k + 31) / 32, d = 32;
  launch_leaves(sl.pos_d, k, p->tn.powf, lv[0], nodes, st);
  int cur = 0;
  while (nodes > 1) {
    const int L = 2 * d, npairs = (nodes + 1) / 2;
    uint32_t* dst = lv[cur ^ 1];
    if (L <= kTreeTileL) {
      Tables t;
      if ((rc = get_tables(L, &t))) return rc;
      KArgs a;
      a.in = lv[cur];
      a.ld_in = (size_t)nodes;
      a.out = dst;
      a.k = k;
      a.L = L;
      a.deg_child = d;
      a.nodes = nodes;
      a.twf = t.twf;
      a.twi = t.twi;
      a.scale = hinv((uint32_t)L % FNT_RS_P);
      tile_ops(L).poly_level(a, 1, st);
    } else {
      const int cols = 2 * npairs;
      uint32_t* Mb = big;
      uint32_t* Mh = Mb + (size_t)L * cols;
      uint32_t* Q = Mh + (size_t)L * cols;
      uint32_t* Qi = Q + (size_t)L * npairs;
      uint32_t* wk = Qi + (size_t)L * npairs;
      launch_big_pack(lv[cur], d, nodes, L, Mb, st);
      if ((rc = run_fnt_default(L, Mb, cols, Mh, cols, cols, false, 1, wk, st))) return rc;
      launch_big_mul(Mh, npairs, L, Q, st);
      if ((rc = run_fnt_default(L, Q, npairs, Qi, npairs, npairs, true, 1, wk, st))) return rc;
      launch_big_fix(Qi, d, k, npairs, L, dst, st);
    }
    cur ^= 1;
    nodes = npairs;
    d = L;
  }
  // steps 2-3 and the step-6 transform(s)
  const int ncols = p->blocked ? 3 : 2;
  launch_pat_prep(lv[cur], k, n, ncols, n / 2, M, st);
  if ((rc = run_fnt_default(n, M, ncols, E, ncols, ncols, false, 1, work, st))) return rc;
  launch_pat_final(E, ncols, sl.pos_d, k, n, p->tn.powi, p->ninv, sl.pat, sl.ahat, sl.ahat2, st);
  launch_pat32(sl.pat, sl.pat32, sl.rowtab, n, st);
  return cuda_ok(cudaGetLastError());
}

int validate_positions(const fnt_rs_plan_s* p, const uint32_t* pos, uint32_t npos) {
  if (!pos) return FNT_RS_E_ARG;
  if (npos < p->k) return FNT_RS_E_POSITIONS;
  std::vector<uint8_t> seen(p->n, 0);
  for (uint32_t i = 0; i < npos; ++i) {
    if (pos[i] >= p->n_out || seen[pos[i]]) return FNT_RS_E_POSITIONS;
    seen[pos[i]] = 1;
  }
  return FNT_RS_OK;
}

// Find or build the pattern of the first k positions; sets p->current.
static int prepare(fnt_rs_plan_s* p, const uint32_t* positions, uint32_t npos, cudaStream_t st) {
  int rc = validate_positions(p, positions, npos);
  if (rc) return rc;
  // map positions for a non-default root: r'^z = r^(u z)
  std::vector<uint32_t> key(positions, positions + p->k);
  if (p->u != 1)
    for (auto& z : key) z = (uint32_t)(((uint64_t)z * p->u) & (p->n - 1));
  ++p->clock;
  for (int s = 0; s < kPatternSlots; ++s) {
    if (p->slots[s].valid && p->slots[s].key == key) {
      p->slots[s].last_use = p->clock;
      p->current = s;
      return FNT_RS_OK;
    }
  }
  int victim = 0;
  for (int s = 0; s < kPatternSlots; ++s) {
    if (!p->slots[s].valid) { victim = s; break; }
    if (p->slots[s].last_use < p->slots[victim].last_use) victim = s;
  }
  PatternSlot& sl = p->slots[victim];
  sl.valid = false;
  // the slot's staging buffer may still be read by its previous build
  if ((rc = cuda_ok(cudaEventSynchronize(sl.staged)))) return rc;
  std::memcpy(sl.pos_h, key.data(), key.size() * 4);
  if (sl.pos_map && fused_plan_applies(p)) {
    // the one-launch build reads the positions from the pinned buffer itself,
    // so it does not queue behind a copy
    if ((rc = build_pattern_log(p, sl, st, nullptr, sl.pos_map))) return rc;
    if ((rc = cuda_ok(cudaEventRecord(sl.staged, st)))) return rc;
  } else {
    if ((rc = cuda_ok(cudaMemcpyAsync(sl.pos_d, sl.pos_h, key.size() * 4,
                                      cudaMemcpyHostToDevice, st))))
      return rc;
    if ((rc = cuda_ok(cudaEventRecord(sl.staged, st)))) return rc;
    if ((rc = p->plan_tree ? build_pattern(p, sl, st) : build_pattern_log(p, sl, st))) return rc;
  }
  sl.key.swap(key);
  sl.valid = true;
  sl.last_use = p->clock;
  p->current = victim;
  return FNT_RS_OK;
}

int prepare_pattern(fnt_rs_plan_s* p, const uint32_t* positions, uint32_t npos, cudaStream_t st) {
  return prepare(p, positions, npos, st);
}

// ---------------------------------------------------------------------------
// encode / decode / fnt dispatch
// ---------------------------------------------------------------------------
// TMA-staged encode (cluster-launch-control tile scheduling); returns 1 if it was not applicable.
// Points an encode's output at the 16-bit wire matrix (columns from c0 on).
static void set_wire(KArgs& a, const WireSpec* w, size_t c0) {
  if (!w) return;
  a.out = w->enc + c0;
  a.ld_out = w->ld;
  a.wire = 1;
  a.wire_rows = (int)w->rows;
  a.col_base = (int)(w->col0 + c0);
  a.esc = w->esc;
  a.esc_count = w->count;
  a.esc_cap = w->cap;
}

static int encode_tma(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                      size_t ld_enc, size_t W, cudaStream_t st, const WireSpec* wire) {
  if (p->no_tma || p->enc_L == 0 || p->u != 1) return 1;
  if ((reinterpret_cast<uintptr_t>(src) % 16) != 0 || (ld_src * 2) % 16 != 0) return 1;
  auto fn = tmap_encode_fn();
  if (!fn) return 1;
  if (p->enc_fold && wire) return 1;  // the folding kernel writes u32 symbols only
  const int L = p->enc_L, C = p->enc_C;
  const int WT = tile_ops(L).wt1;  // 8 codewords of 16-bit source: one 16-byte TMA row
  const int box_rows = std::min(256, L);
  const int rows_staged = (int)((p->k + box_rows - 1) / box_rows) * box_rows;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)p->k};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_src * 2};
  const cuuint32_t box[2] = {(cuuint32_t)WT, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<uint16_t*>(src), dims, strides, box,
         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 1;
  const int ntiles = (int)((W + WT - 1) / WT);
  KArgs a;
  a.out = enc;
  a.ld_out = ld_enc;
  a.W = (int)W;
  a.n = (int)p->n;
  a.k = (int)p->k;
  a.L = L;
  a.C = C;
  a.twf = p->tenc.twf;
  a.status = p->status;
  set_wire(a, wire, 0);
  TmaEncodeArgs t;
  t.twc = p->twc;
  t.rows_staged = rows_staged;
  t.box_rows = box_rows;
  t.grid = ntiles;  // one CTA per tile; running CTAs take over pending ones
  t.map = &map;
  if ((p->enc_fold ? launch_encode_tma_fold(a, t, st) : launch_encode_tma(L, C, a, t, st)) != 0)
    return 1;
  return cuda_ok(cudaGetLastError());
}

int do_encode(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                     size_t ld_enc, size_t W, void* workspace, cudaStream_t st,
                     const WireSpec* wire) {
  int sched = sched_effective(p, FNT_RS_OP_ENCODE);
  if (sched == FNT_RS_SCHED_DIRECT) {
    if (!wire) return direct_encode(p, src, ld_src, enc, ld_enc, W, workspace, st);
    // the 16-bit wire output is written by the transform kernels only
    sched = sched_available(p, FNT_RS_OP_ENCODE, FNT_RS_SCHED_TMA)
                ? FNT_RS_SCHED_TMA
                : (p->n <= 8192 ? FNT_RS_SCHED_TILE : FNT_RS_SCHED_SPLIT);
  }
  if (sched == FNT_RS_SCHED_TMA) {
    const int t = encode_tma(p, src, ld_src, enc, ld_enc, W, st, wire);
    if (t != 1) return t;  // else (unaligned pointers) the one-CTA tile below
  }
  if (sched == FNT_RS_SCHED_SPLIT)
    return do_encode_two_pass(p, src, ld_src, enc, ld_enc, W, static_cast<uint32_t*>(workspace),
                              st, wire);
  KArgs a;
  a.in = src;
  a.ld_in = ld_src;
  a.out = enc;
  a.ld_out = ld_enc;
  a.W = (int)W;
  a.n = (int)p->n;
  a.k = (int)p->k;
  a.powf = p->tn.powf;
  a.row_mul = p->uinv;
  a.L = (int)p->n;
  a.C = 1;
  a.twf = p->tn.twf;
  a.twi = p->tn.twi;
  set_wire(a, wire, 0);
  tile_ops((int)p->n).encode(a, 1, st);
  return cuda_ok(cudaGetLastError());
}

int do_encode_two_pass(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                       size_t ld_enc, size_t W, uint32_t* workspace, cudaStream_t st,
                       const WireSpec* wire) {
  if (p->n <= 8192) return do_encode(p, src, ld_src, enc, ld_enc, W, nullptr, st, wire);
  const size_t wc = split_chunk(p->n, 1);
  uint32_t* work = static_cast<uint32_t*>(workspace);
  for (size_t c0 = 0; c0 < W; c0 += wc) {
    const int w = (int)std::min(wc, W - c0);
    KArgs a;
    a.in = src + c0;
    a.ld_in = ld_src;
    a.out = enc ? enc + c0 : nullptr;  // (the wire output replaces it)
    a.ld_out = ld_enc;
    a.out2 = work;
    a.ld_work = (size_t)w;
    a.W = w;
    a.n = (int)p->n;
    a.k = (int)p->k;
    a.L = kLocalL;
    a.C = p->C_local;
    a.row_limit = (int)p->k;
    a.powf = p->tn.powf;
    a.powi = p->tn.powi;
    a.row_mul = p->uinv;
    cross_launcher(p->C_local, false, CL_SRC16)(a, 1, st);
    KArgs b = a;
    b.in = work;
    b.ld_in = (size_t)w;
    b.twf = p->tl.twf;
    b.twi = p->tl.twi;
    set_wire(b, wire, c0);
    local_launcher(false, LM_ENC)(b, p->C_local, st);
  }
  return cuda_ok(cudaGetLastError());
}

// Decode with tiles staged by cp.async (packed rows, k <= n/2): half-width
// tiles, two CTAs per SM, for n in {4096, 8192}; two-codeword tiles, one CTA
// per SM, for n = 16384.  Returns 1 if not applicable.
static int decode_cpa(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv,
                      size_t ld_recv, uint16_t* out, size_t ld_out, size_t W, cudaStream_t st,
                      uint32_t* out32) {
  if (p->split || p->blocked || p->n > 32768) return 1;
  const TileOps& ops = tile_ops((int)p->n);
  if (!ops.decode_cpa) return 1;
  const size_t row_bytes = (size_t)ops.wt_cpa * 4;  // 8 or 16: the copy size
  if (reinterpret_cast<uintptr_t>(recv) % row_bytes != 0 || (ld_recv * 4) % row_bytes != 0)
    return 1;
  KArgs a;
  a.in = recv;
  a.ld_in = ld_recv;
  a.out = out;
  a.ld_out = ld_out;
  a.W = (int)W;
  a.n = (int)p->n;
  a.k = (int)p->k;
  a.L = (int)p->n;
  a.C = 1;
  a.twf = p->tn.twf;
  a.twi = p->tn.twi;
  a.ahat = sl.ahat;
  a.status = p->status;
  a.out32 = out32;
  if (ops.decode_cpa(a, sl.pat32, st) != 0) return 1;
  return cuda_ok(cudaGetLastError());
}

// TMA-staged decode (one CTA per tile, cluster launch control; packed rows,
// n <= tile limit, k <= n/2);
// returns 1 if not applicable.
static int decode_tma(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv,
                      size_t ld_recv, uint16_t* out, size_t ld_out, size_t W, cudaStream_t st,
                      uint32_t* out32) {
  if (p->no_tma || p->split || p->blocked || p->n < 64 || p->n > 8192) return 1;
  if ((reinterpret_cast<uintptr_t>(recv) % 16) != 0 || (ld_recv * 4) % 16 != 0) return 1;
  auto fn = tmap_encode_fn();
  if (!fn) return 1;
  const int L = (int)p->n;
  const TileOps& ops = tile_ops(L);
  const int WT = ops.wt1;
  const int box_rows = std::min(256, L);
  const int rows_staged = (int)((p->k + box_rows - 1) / box_rows) * box_rows;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)p->k};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_recv * 4};
  const cuuint32_t box[2] = {(cuuint32_t)WT, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t*>(recv), dims, strides, box,
         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return 1;
  KArgs a;
  a.out = out;
  a.ld_out = ld_out;
  a.W = (int)W;
  a.n = L;
  a.k = (int)p->k;
  a.L = L;
  a.C = 1;
  a.twf = p->tn.twf;
  a.twi = p->tn.twi;
  a.twf_sw = p->tn.twf_sw;
  a.ahat = sl.ahat;
  a.status = p->status;
  a.out32 = out32;
  TmaDecodeArgs t;
  t.pat32 = sl.pat32;
  t.rowtab = sl.rowtab;
  t.rows_staged = rows_staged;
  t.box_rows = box_rows;
  t.sms = p->sms;
  t.map = &map;
  if (launch_decode_tma(L, a, t, st) != 0) return 1;
  return cuda_ok(cudaGetLastError());
}

int do_decode_tables(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv,
                     size_t ld_recv, uint16_t* out, size_t ld_out, size_t W, void* workspace,
                     cudaStream_t st, int slots, uint32_t* out32) {
  const int sched = sched_effective(p, FNT_RS_OP_DECODE);
  if (sched == FNT_RS_SCHED_PAPER)
    return paper_decode(p, sl, recv, ld_recv, out, ld_out, W, workspace, st, slots, out32);
  if (sched == FNT_RS_SCHED_DIRECT)
    return direct_decode(p, sl, recv, ld_recv, out, ld_out, W, workspace, st, slots, out32);
  if (!slots && sched == FNT_RS_SCHED_TMA) {
    const int t = decode_tma(p, sl, recv, ld_recv, out, ld_out, W, st, out32);
    if (t != 1) return t;  // else (unaligned rows) the one-CTA tile below
  }
  if (!slots && sched == FNT_RS_SCHED_CPA) {
    const int t = decode_cpa(p, sl, recv, ld_recv, out, ld_out, W, st, out32);
    if (t != 1) return t;
  }
  KArgs a;
  a.slots = slots;
  a.in = recv;
  a.ld_in = ld_recv;
  a.out = out;
  a.ld_out = ld_out;
  a.n = (int)p->n;
  a.k = (int)p->k;
  a.h = (int)p->n / 2;
  a.pat = sl.pat;
  a.ahat = sl.ahat;
  a.ahat2 = sl.ahat2;
  a.status = p->status;
  a.out32 = out32;
  if (sched != FNT_RS_SCHED_SPLIT) {
    const TileOps& ops = tile_ops((int)p->n);
    a.W = (int)W;
    a.L = (int)p->n;
    a.C = 1;
    a.twf = p->tn.twf;
    a.twi = p->tn.twi;
    Launch fn = p->blocked ? ops.decode_split : ops.decode;
    if (!fn) return FNT_RS_E_ARG;
    fn(a, 1, st);
    return cuda_ok(cudaGetLastError());
  }
  const int nbuf = dec_nbuf(p);
  const size_t wc = split_chunk(p->n, nbuf);
  const size_t nw = (size_t)p->n;
  for (size_t c0 = 0; c0 < W; c0 += wc) {
    const int w = (int)std::min(wc, W - c0);
    uint32_t* A = static_cast<uint32_t*>(workspace);
    uint32_t* B0 = A + nw * w;
    uint32_t* B1 = B0 + nw * w;
    uint32_t* B2 = B1 + nw * w;
    KArgs c = a;
    c.in = recv + c0;
    c.out = out + c0;
    c.W = w;
    c.L = kLocalL;
    c.C = p->C_local;
    c.ld_work = (size_t)w;
    c.powf = p->tn.powf;
    c.powi = p->tn.powi;
    c.twf = p->tl.twf;
    c.twi = p->tl.twi;
    auto cross = [&](bool inv, int lm, const void* in, size_t ld_in, int row_limit) {
      KArgs x = c;
      x.in = in;
      x.ld_in = ld_in;
      x.row_limit = row_limit;
      x.out2 = A;
      cross_launcher(p->C_local, inv, lm)(x, 1, st);
    };
    auto local = [&](bool inv, int mode, void* o2, void* o3, int out_limit, const void* in2) {
      KArgs x = c;
      x.in = A;
      x.ld_in = (size_t)w;
      x.out2 = o2;
      x.out3 = o3;
      x.in2 = in2;
      x.out_limit = out_limit;
      local_launcher(inv, mode)(x, p->C_local, st);
    };
    if (!p->blocked) {
      cross(true, CL_RECV, recv + c0, ld_recv, (int)p->n);
      local(true, LM_WORK, B0, nullptr, (int)p->k, nullptr);
      cross(false, CL_U32, B0, (size_t)w, (int)p->k);
      local(false, LM_WORK_AHAT, B0, nullptr, (int)p->n, nullptr);
      cross(true, CL_U32, B0, (size_t)w, (int)p->n);
      local(true, LM_OUT16, nullptr, nullptr, (int)p->k, nullptr);
    } else {
      const int h = (int)p->n / 2;
      cross(true, CL_RECV, recv + c0, ld_recv, (int)p->n);
      local(true, LM_SPLIT, B0, B1, (int)p->k, nullptr);
      cross(false, CL_U32, B0, (size_t)w, h);
      local(false, LM_X_PARTIAL, B0, B2, (int)p->n, nullptr);
      cross(false, CL_U32, B1, (size_t)w, (int)p->k - h);
      local(false, LM_ACCUM, nullptr, B2, (int)p->n, nullptr);
      cross(true, CL_U32, B2, (size_t)w, (int)p->n);
      local(true, LM_WORK, B1, nullptr, (int)p->n, nullptr);
      cross(true, CL_U32, B0, (size_t)w, (int)p->n);
      local(true, LM_OUT16_ADD, nullptr, nullptr, (int)p->k, B1);
    }
  }
  return cuda_ok(cudaGetLastError());
}

}  // namespace fntrs

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* fnt_rs_strerror(int code) {
  switch (code) {
    case FNT_RS_OK: return "ok";
    case FNT_RS_E_ARG: return "invalid argument";
    case FNT_RS_E_UNSUPPORTED_P: return "unsupported field: p must be 65537";
    case FNT_RS_E_ROOT: return "root does not have order exactly n";
    case FNT_RS_E_POSITIONS: return "positions: fewer than k, duplicate, or >= n";
    case FNT_RS_E_BUDGET: return "request exceeds the admission budget";
    case FNT_RS_E_CUDA: return "CUDA runtime error";
    case FNT_RS_E_RANGE: return "value out of range (decoded 65536 or received > 65536)";
    case FNT_RS_E_TIMEOUT: return "a bounded device wait gave up";
    case FNT_RS_E_BOUNDS:
      return "a device index check of the debug build failed (the access was skipped)";
    case FNT_RS_E_WORKSPACE:
      return "workspace missing or too small (or, for fnt_rs_encode_noalloc, the encode "
             "workspace exceeds FNT_RS_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown status";
  }
}

uint64_t fnt_rs_launch_count(void) { return g_launches.load(); }

int fnt_rs_plan_create(fnt_rs_plan* out, uint32_t n, uint32_t k, uint32_t p_, uint32_t root,
                       void* stream) {
  if (!out) return FNT_RS_E_ARG;
  *out = nullptr;
  if (n < 2 || n > 65536 || (n & (n - 1)) != 0 || k < 1 || k > n) return FNT_RS_E_ARG;
  if (p_ != FNT_RS_P) return FNT_RS_E_UNSUPPORTED_P;
  uint32_t u = 1;
  if (root != 0) {
    if (root >= FNT_RS_P || hpow(root, n) != 1 || hpow(root, n / 2) != FNT_RS_P - 1)
      return FNT_RS_E_ROOT;
    // root = default^u with u odd
    const uint32_t r0 = default_root(n);
    uint32_t acc = r0;
    u = 0;
    for (uint32_t e = 1; e < n; e += 2) {
      if (acc == root) { u = e; break; }
      acc = hmul(acc, hmul(r0, r0));
    }
    if (u == 0) return FNT_RS_E_ROOT;
  }
  init_ops();
  fnt_rs_plan_s* p = new (std::nothrow) fnt_rs_plan_s();
  if (!p) return FNT_RS_E_ARG;
  cudaGetDevice(&p->dev);
  p->n = n;
  p->k = k;
  p->root = root ? root : default_root(n);
  p->u = u;
  // inverse of the odd u modulo n (n is a power of two)
  uint32_t ui = 1;
  for (int it = 0; it < 5; ++it) ui = ui * (2u - u * ui);
  p->uinv = ui & (n - 1);
  p->ninv = hinv(n % FNT_RS_P);
  // one CTA holds the transform unless the decode would need two buffers of a
  // 32768-point codeword (k > n/2) or n exceeds the tile limit
  p->split = n > (uint32_t)kTileMaxL || (n == (uint32_t)kTileMaxL && 2 * k > n);
  p->C = p->split ? (int)(n / kLocalL) : 1;
  p->blocked = k > n / 2;
  p->n_out = n;
  p->C_local = n > 8192 ? (int)(n / kLocalL) : 1;
  int rc = get_tables((int)n, &p->tn);
  if (!rc && n > 8192) rc = get_tables(kLocalL, &p->tl);
  auto fail = [&](int code) {
    fnt_rs_plan_destroy(p);
    return code;
  };
  if (rc) return fail(rc);
  {
    const char* e = std::getenv("FNTRS_NO_TMA");
    p->no_tma = e && e[0] == '1';
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->dev);
    if (n >= 64 && n <= 4096) {
      p->enc_L = (int)n;
      p->enc_C = 1;
    } else if (n == 8192) {
      p->enc_L = 4096;
      p->enc_C = 2;
      p->enc_fold = k > 4096;
    }
    if (p->enc_L && (rc = get_tables(p->enc_L, &p->tenc))) return fail(rc);
    const char* pe = std::getenv("FNTRS_PLAN");
    p->plan_tree = pe && std::strcmp(pe, "tree") == 0;
    if ((rc = get_exp3(&p->exp3))) return fail(rc);
    // digit width b with k (2^b - 1) < p: every digit convolution stays below p
    p->lg_b = 15u * k < FNT_RS_P ? 4 : (7u * k < FNT_RS_P ? 3 : (3u * k < FNT_RS_P ? 2 : 1));
    p->lg_D = (16 + p->lg_b - 1) / p->lg_b;
    {
      const int D = p->lg_D, b = p->lg_b;
      std::vector<uint32_t> dl(65537, 0);
      uint32_t x = 1;
      for (uint32_t e = 0; e < 65536; ++e) {
        dl[x] = e;
        x = hmul(x, 3);
      }
      const uint32_t r = default_root(n);
      std::vector<uint32_t> g(n, 0), dig((size_t)n * D);
      uint32_t rd = r;
      for (uint32_t d = 1; d < n; ++d) {
        g[d] = dl[(1u + FNT_RS_P - rd) % FNT_RS_P];
        rd = hmul(rd, r);
      }
      for (uint32_t d = 0; d < n; ++d) {
        const uint32_t gr = g[(n - d) & (n - 1)];  // reversed: correlation as convolution
        for (int t = 0; t < D; ++t) dig[(size_t)d * D + t] = (gr >> (b * t)) & ((1u << b) - 1u);
      }
      uint32_t *din = nullptr, *wk = nullptr;
      if ((rc = upload(&din, dig))) return fail(rc);
      if (cudaMalloc(&p->ghat, dig.size() * 4) != cudaSuccess ||
          cudaMalloc(&wk, dig.size() * 4) != cudaSuccess) {
        cudaFree(din);
        cudaFree(wk);
        return fail(FNT_RS_E_CUDA);
      }
      rc = run_fnt_default((int)n, din, D, p->ghat, D, D, false, 1, wk, S(stream));
      if (!rc) rc = cuda_ok(cudaStreamSynchronize(S(stream)));
      cudaFree(din);
      cudaFree(wk);
      if (rc) return fail(rc);
    }
    if (p->enc_C == 2) {
      // twc[i2*R1 + q] = r_L^(i2 * bitrev(q)) * r_n^i2, i2 < L/R1
      int r[3];
      sched_radices(p->enc_L, r);
      const int L = p->enc_L, R1 = r[0], S1 = L / R1, b0 = ilog2i(R1);
      const uint32_t rL = default_root(L), rn = default_root(n);
      std::vector<uint32_t> t((size_t)L);
      for (int i2 = 0; i2 < S1; ++i2)
        for (int q = 0; q < R1; ++q)
          t[(size_t)i2 * R1 + q] =
              hmul(hpow(rL, (uint64_t)i2 * bitrev_h(q, b0) % L), hpow(rn, (uint64_t)i2));
      if ((rc = upload(&p->twc, t))) return fail(rc);
    }
  }
  if (cudaMalloc(&p->status, sizeof(int)) != cudaSuccess) return fail(FNT_RS_E_CUDA);
  if (cudaMemsetAsync(p->status, 0, sizeof(int), S(stream)) != cudaSuccess)
    return fail(FNT_RS_E_CUDA);
  p->pscratch_words = pattern_scratch_words(n, k);
  if (cudaMalloc(&p->pscratch, p->pscratch_words * 4) != cudaSuccess) return fail(FNT_RS_E_CUDA);
  for (auto& sl : p->slots)
    if ((rc = alloc_pattern_tables(sl, n, true))) return fail(rc);
  if ((rc = pipe_init(p->pipe))) return fail(rc);
  if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return fail(FNT_RS_E_CUDA);
  *out = p;
  return FNT_RS_OK;
}

void fnt_rs_plan_destroy(fnt_rs_plan p) {
  if (!p) return;
  cudaDeviceSynchronize();
  cudaFree(p->status);
  cudaFree(p->pscratch);
  cudaFree(p->twc);
  cudaFree(p->ghat);
  for (auto& sl : p->slots) free_pattern_tables(sl);
  free_pattern_tables(p->sys);
  pipe_free(p->pipe);
  paper_free(p);
  direct_free(p);
  delete p;
}

size_t fnt_rs_workspace_bytes(fnt_rs_plan p, size_t W, int op) {
  if (!p) return 0;
  switch (op) {
    case FNT_RS_OP_ENCODE:
      return std::max(ws_bytes(p, W, enc_nbuf_max(p)) +
                          (p->n_out < p->n ? align256((size_t)p->n * W * 4) : 0),
                      direct_ws_bytes(p, W));
    case FNT_RS_OP_ENCODE_SYS:
    case FNT_RS_OP_DECODE_SYS: return sys_workspace_bytes(p, W);
    case FNT_RS_OP_DECODE: return dec_ws_max(p, W);
    case FNT_RS_OP_FNT: return ws_bytes(p, W, fnt_nbuf(p));
    case FNT_RS_OP_ENCODE_HOST:
    case FNT_RS_OP_DECODE_HOST:
    case FNT_RS_OP_ENCODE_WIRE_HOST:
    case FNT_RS_OP_DECODE_WIRE_HOST: return host_workspace_bytes(p, W, op);
    case FNT_RS_OP_ENCODE_WIRE:
    case FNT_RS_OP_DECODE_WIRE: return wire_workspace_bytes(p, W, op);
    default: return 0;
  }
}



int fnt_rs_encode(fnt_rs_plan p, const uint16_t* src, size_t ld_src, uint32_t* enc, size_t ld_enc,
                  size_t W, void* workspace, void* stream) {
  if (!p || W == 0) return W == 0 && p ? FNT_RS_OK : FNT_RS_E_ARG;
  if (!src || !enc || ld_src < W || ld_enc < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned(src, 2) || !aligned(enc, 4)) return FNT_RS_E_ARG;
  if (sched_effective(p, FNT_RS_OP_ENCODE) == FNT_RS_SCHED_DIRECT) {
    // the direct product writes the n_out rows of a punctured code itself
    if (direct_ws_bytes(p, W) && !workspace) return FNT_RS_E_WORKSPACE;
    return direct_encode(p, src, ld_src, enc, ld_enc, W, workspace, S(stream));
  }
  if (p->n_out == p->n) {
    if (ws_bytes(p, W, enc_nbuf(p)) && !workspace) return FNT_RS_E_WORKSPACE;
    return do_encode(p, src, ld_src, enc, ld_enc, W, workspace, S(stream));
  }
  // punctured code: all n rows into the workspace, the first n_out kept
  if (!workspace) return FNT_RS_E_WORKSPACE;
  uint32_t* full = static_cast<uint32_t*>(workspace);
  void* rest = static_cast<uint8_t*>(workspace) + align256((size_t)p->n * W * 4);
  int rc = do_encode(p, src, ld_src, full, W, W, rest, S(stream));
  if (rc) return rc;
  return cuda_ok(cudaMemcpy2DAsync(enc, ld_enc * 4, full, W * 4, W * 4, p->n_out,
                                   cudaMemcpyDeviceToDevice, S(stream)));
}

int fnt_rs_decode_prepare(fnt_rs_plan p, const uint32_t* positions, uint32_t npos, void* stream) {
  if (!p) return FNT_RS_E_ARG;
  return prepare(p, positions, npos, S(stream));
}

int fnt_rs_decode(fnt_rs_plan p, const uint32_t* recv, size_t ld_recv, const uint32_t* positions,
                  uint32_t npos, uint16_t* out, size_t ld_out, size_t W, void* workspace,
                  void* stream) {
  if (!p) return FNT_RS_E_ARG;
  if ((W && (!recv || !out)) || ld_recv < W || ld_out < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned(recv, 4) || !aligned(out, 2)) return FNT_RS_E_ARG;
  if (dec_ws_now(p, W) && !workspace) return FNT_RS_E_WORKSPACE;
  int rc = prepare(p, positions, npos, S(stream));
  if (rc) return rc;
  if (W == 0) return FNT_RS_OK;
  return do_decode_tables(p, p->slots[p->current], recv, ld_recv, out, ld_out, W, workspace,
                          S(stream), 0);
}

int fnt_rs_decode_slots(fnt_rs_plan p, const uint32_t* slots, size_t ld_slots,
                        const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out,
                        size_t W, void* workspace, void* stream) {
  if (!p) return FNT_RS_E_ARG;
  if ((W && (!slots || !out)) || ld_slots < W || ld_out < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned(slots, 4) || !aligned(out, 2)) return FNT_RS_E_ARG;
  if (dec_ws_now(p, W) && !workspace) return FNT_RS_E_WORKSPACE;
  if (p->u != 1) return FNT_RS_E_ROOT;  // slot rows follow the default root's positions
  int rc = prepare(p, positions, npos, S(stream));
  if (rc) return rc;
  if (W == 0) return FNT_RS_OK;
  return do_decode_tables(p, p->slots[p->current], slots, ld_slots, out, ld_out, W, workspace,
                          S(stream), 1);
}

int fnt_rs_decode_full(fnt_rs_plan p, const uint32_t* enc, size_t ld_enc, uint16_t* out,
                       size_t ld_out, size_t W, void* workspace, void* stream) {
  if (!p || p->n_out < p->n) return FNT_RS_E_ARG;  // a punctured codeword is never complete
  if (W == 0) return FNT_RS_OK;
  if ((W && (!enc || !out)) || ld_enc < W || ld_out < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned(enc, 4) || !aligned(out, 2)) return FNT_RS_E_ARG;
  if (ws_bytes(p, W, fnt_nbuf(p)) && !workspace) return FNT_RS_E_WORKSPACE;
  cudaStream_t st = S(stream);
  KArgs a;
  a.in = enc;
  a.ld_in = ld_enc;
  a.out = out;
  a.ld_out = ld_out;
  a.n = (int)p->n;
  a.k = (int)p->k;
  a.scale = p->ninv;
  a.in_row_mul = p->uinv;
  a.status = p->status;
  if (!p->split) {
    a.W = (int)W;
    a.L = (int)p->n;
    a.C = 1;
    a.twf = p->tn.twf;
    a.twi = p->tn.twi;
    tile_ops((int)p->n).lossless(a, 1, st);
    return cuda_ok(cudaGetLastError());
  }
  const size_t wc = split_chunk(p->n, 1);
  uint32_t* work = static_cast<uint32_t*>(workspace);
  for (size_t c0 = 0; c0 < W; c0 += wc) {
    const int w = (int)std::min(wc, W - c0);
    KArgs c = a;
    c.in = enc + c0;
    c.out = out + c0;
    c.W = w;
    c.L = kLocalL;
    c.C = p->C;
    c.row_limit = (int)p->n;
    c.out2 = work;
    c.ld_work = (size_t)w;
    c.powf = p->tn.powf;
    c.powi = p->tn.powi;
    cross_launcher(p->C, true, CL_U32)(c, 1, st);
    KArgs b = c;
    b.in = work;
    b.ld_in = (size_t)w;
    b.in_row_mul = 1;
    b.out_limit = (int)p->k;
    b.twf = p->tl.twf;
    b.twi = p->tl.twi;
    local_launcher(true, LM_OUT16)(b, p->C, st);
  }
  return cuda_ok(cudaGetLastError());
}

}  // extern "C"

namespace fntrs {

size_t fnt_columns_work_bytes(const fnt_rs_plan_s* p, size_t W) {
  if (p->n <= (uint32_t)kTileMaxL || W == 0) return 0;
  return (size_t)p->n * std::min(W, split_chunk(p->n, 1)) * 4;
}

int fnt_columns(fnt_rs_plan_s* p, const uint32_t* in, size_t ld_in, uint32_t* out,
                size_t ld_out, size_t W, bool inverse, void* work, cudaStream_t st) {
  if (p->n <= (uint32_t)kTileMaxL)
    return run_fnt_default((int)p->n, in, ld_in, out, ld_out, (int)W, inverse, p->uinv, nullptr,
                           st);
  const size_t wc = split_chunk(p->n, 1);
  for (size_t c0 = 0; c0 < W; c0 += wc) {
    const int w = (int)std::min(wc, W - c0);
    int rc = run_fnt_default((int)p->n, in + c0, ld_in, out + c0, ld_out, w, inverse, p->uinv,
                             static_cast<uint32_t*>(work), st);
    if (rc) return rc;
  }
  return FNT_RS_OK;
}

}  // namespace fntrs

extern "C" {

int fnt_rs_fnt(fnt_rs_plan p, const uint32_t* in, size_t ld_in, uint32_t* out, size_t ld_out,
               size_t W, int inverse, void* workspace, void* stream) {
  if (!p) return FNT_RS_E_ARG;
  if (W == 0) return FNT_RS_OK;
  if (!in || !out || ld_in < W || ld_out < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned(in, 4) || !aligned(out, 4)) return FNT_RS_E_ARG;
  if (ws_bytes(p, W, fnt_nbuf(p)) && !workspace) return FNT_RS_E_WORKSPACE;
  return fnt_columns(p, in, ld_in, out, ld_out, W, inverse != 0, workspace, S(stream));
}

int fnt_rs_set_schedule(fnt_rs_plan p, int op, int sched) {
  if (p && (op == FNT_RS_OP_ENCODE_SYS || op == FNT_RS_OP_DECODE_SYS)) {
    if (sched != FNT_RS_SCHED_AUTO && sched != FNT_RS_SCHED_DIRECT) return FNT_RS_E_ARG;
    if (sched == FNT_RS_SCHED_DIRECT) {
      if (!direct_available(p)) return FNT_RS_E_ARG;
      const int rc = direct_enable(p, op);
      if (rc) return rc;
    }
    (op == FNT_RS_OP_ENCODE_SYS ? p->sched_sys_enc : p->sched_sys_dec) = sched;
    return FNT_RS_OK;
  }
  if (!p || (op != FNT_RS_OP_ENCODE && op != FNT_RS_OP_DECODE)) return FNT_RS_E_ARG;
  if (sched != FNT_RS_SCHED_AUTO && !sched_available(p, op, sched)) return FNT_RS_E_ARG;
  if (sched == FNT_RS_SCHED_PAPER) {
    const int rc = paper_enable(p, nullptr);
    if (rc) return rc;
  }
  if (sched == FNT_RS_SCHED_DIRECT) {
    const int rc = direct_enable(p, op);
    if (rc) return rc;
  }
  (op == FNT_RS_OP_ENCODE ? p->sched_enc : p->sched_dec) = sched;
  return FNT_RS_OK;
}

int fnt_rs_get_schedule(fnt_rs_plan p, int op) {
  if (p && (op == FNT_RS_OP_ENCODE_SYS || op == FNT_RS_OP_DECODE_SYS)) {
    const int s = op == FNT_RS_OP_ENCODE_SYS ? p->sched_sys_enc : p->sched_sys_dec;
    // the FNT route interpolates with the decode schedule
    return s ? s : sched_effective(p, FNT_RS_OP_DECODE);
  }
  if (!p || (op != FNT_RS_OP_ENCODE && op != FNT_RS_OP_DECODE)) return FNT_RS_E_ARG;
  return sched_effective(p, op);
}

int fnt_rs_autotune(fnt_rs_plan p, size_t W, int op, fnt_rs_tune_result* out, int cap,
                    void* stream) {
  if (!p || W == 0 || (op != FNT_RS_OP_ENCODE && op != FNT_RS_OP_DECODE)) return FNT_RS_E_ARG;
  // Only the transform schedules (integer pipes) are candidates: the plain code's
  // encode and decode never switch to the tensor-core product by themselves;
  // FNT_RS_SCHED_DIRECT stays an explicit choice through fnt_rs_set_schedule.
  std::vector<int> cand;
  for (int s : {FNT_RS_SCHED_TMA, FNT_RS_SCHED_CPA, FNT_RS_SCHED_TILE, FNT_RS_SCHED_SPLIT})
    if (sched_available(p, op, s)) cand.push_back(s);
  if (cand.empty()) return FNT_RS_E_ARG;
  cudaStream_t st = S(stream);
  const size_t n = p->n, k = p->k;
  size_t w = std::min(W, std::max<size_t>(8, ((size_t)1 << 29) / (n * 4)));
  if (w >= 8) w = w / 8 * 8;
  const bool enc_op = op == FNT_RS_OP_ENCODE;
  const size_t wsb = std::max(ws_bytes(p, w, enc_op ? enc_nbuf_max(p) : dec_nbuf_max(p)),
                              direct_ws_bytes(p, w));
  uint16_t* src = nullptr;
  uint32_t* enc = nullptr;
  uint16_t* dout = nullptr;
  void* ws = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int* saved = enc_op ? &p->sched_enc : &p->sched_dec;
  const int keep = *saved;
  std::vector<fnt_rs_tune_result> res;
  int rc = FNT_RS_OK;
  if (cudaMalloc(&src, k * w * 2) != cudaSuccess || cudaMalloc(&enc, n * w * 4) != cudaSuccess ||
      cudaMalloc(&dout, k * w * 2) != cudaSuccess ||
      (wsb && cudaMalloc(&ws, wsb) != cudaSuccess) ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemsetAsync(src, 0, k * w * 2, st) != cudaSuccess ||
      cudaMemsetAsync(enc, 0, n * w * 4, st) != cudaSuccess)
    rc = FNT_RS_E_CUDA;
  if (!rc && !enc_op) {
    // k distinct positions z_i = (a i + b) mod n (a odd: a bijection of Z/n)
    std::vector<uint32_t> pos(k);
    for (size_t i = 0; i < k; ++i) pos[i] = (uint32_t)((0x9E3779B1u * i + 12345u) & (n - 1));
    rc = prepare(p, pos.data(), (uint32_t)k, st);
  }
  for (size_t ci = 0; !rc && ci < cand.size(); ++ci) {
    *saved = cand[ci];
    auto run = [&]() {
      return enc_op ? do_encode(p, src, w, enc, w, w, ws, st)
                    : do_decode_tables(p, p->slots[p->current], enc, w, dout, w, w, ws, st, 0);
    };
    float t[5];
    for (int it = 0; it < 7 && !rc; ++it) {
      if (it >= 2 && cudaEventRecord(e0, st) != cudaSuccess) rc = FNT_RS_E_CUDA;
      if (!rc) rc = run();
      if (!rc && it >= 2) {
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t[it - 2], e0, e1) != cudaSuccess)
          rc = FNT_RS_E_CUDA;
      }
    }
    if (!rc) {
      std::sort(t, t + 5);
      res.push_back({cand[ci], t[2] * 1000.0f});
    }
  }
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = FNT_RS_E_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(src);
  cudaFree(enc);
  cudaFree(dout);
  cudaFree(ws);
  if (rc) {
    *saved = keep;
    return rc;
  }
  auto best = std::min_element(res.begin(), res.end(), [](const fnt_rs_tune_result& a,
                                                          const fnt_rs_tune_result& b) {
    return a.us < b.us;
  });
  *saved = best->sched;
  for (int i = 0; i < cap && i < (int)res.size(); ++i) out[i] = res[i];
  return (int)res.size();
}

int fnt_rs_status(fnt_rs_plan p, void* stream) {
  if (!p) return FNT_RS_E_ARG;
  int h = 0;
  cudaStream_t st = S(stream);
  if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return FNT_RS_E_CUDA;
  if (cudaMemsetAsync(p->status, 0, sizeof(int), st) != cudaSuccess) return FNT_RS_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FNT_RS_E_CUDA;
  if (h & ST_TIMEOUT) return FNT_RS_E_TIMEOUT;
  if (h & ST_BOUNDS) return FNT_RS_E_BOUNDS;
  if (h & ST_RANGE) return FNT_RS_E_RANGE;
  return FNT_RS_OK;
}

int fnt_rs_debug_bounds(void) { return FNTRS_DEBUG_BOUNDS ? 1 : 0; }

int fnt_rs_plan_info(fnt_rs_plan p, int* info, int cap) {
  if (!p || !info) return 0;
  int vals[8] = {(int)p->n, (int)p->k, p->split ? kLocalL : (int)p->n, p->C,
                 tile_ops(p->split ? kLocalL : (int)p->n).wt1,
                 tile_ops(p->split ? kLocalL : (int)p->n).wt2, p->blocked ? 1 : 0, 0};
  int cnt = 0;
  for (auto& sl : p->slots) cnt += sl.valid ? 1 : 0;
  vals[7] = cnt;
  const int m = std::min(cap, 8);
  for (int i = 0; i < m; ++i) info[i] = vals[i];
  return m;
}

}  // extern "C"
