// Kernel templates: encode, batched FNT, split-transform cross / local passes,
// fused single-CTA decode, and one level of the locator product tree.
#pragma once
#include "kargs.h"
#include "logplan.cuh"
#include "tile.cuh"
#include "tma.cuh"

namespace fntrs {

// Loads of decode tables and received words: through the read-only cache
// (CG = false) or through L2 only (CG = true, for data that other CTAs of the
// same launch may have written, as in the ragged persistent kernel).
template <bool CG, class T>
__device__ __forceinline__ T ld_tab(const T* p) {
  if constexpr (CG) {
    return __ldcg(p);
  } else {
    return __ldg(p);
  }
}

// ---------------------------------------------------------------------------
// Loaders: element i (0 <= i < L) of tile codeword c.
// ---------------------------------------------------------------------------

// Encode input (Sec. II.B: the FNT of (s_0..s_{k-1}, 0..0)).  For a transform
// split as n = C * L the CTA of output class cc (outputs j = cc + C*j') feeds
// the length-L transform with  x[i] = r_n^(i*cc) * sum_m s[i + m L] w_C^(m*cc),
// w_C = r_n^L = 2^(e_C) (a rotation); for C = 1 this is the zero-padded source.
template <int WT>
struct LoadSrcFold {
  const uint16_t* src;
  size_t ld;
  const uint32_t* powf;
  int col0, W, k, L, C, cc, eC, nmask;
  static __device__ __forceinline__ LoadSrcFold make(const KArgs& a, int tx, int ty) {
    int lc = 0;
    for (int c = a.C; c > 1; c >>= 1) lc += 1;  // log2(C)
    // e_C for C = 2,4,8,16: 16, 24, 12, 6  (2^e_C = 3^(65536/C) mod p)
    const int eC = lc == 0 ? 0 : (lc == 1 ? 16 : (lc == 2 ? 24 : (lc == 3 ? 12 : 6)));
    return LoadSrcFold{static_cast<const uint16_t*>(a.in), a.ld_in, a.powf,
                       tx * WT, a.W, a.k, a.L, a.C, ty, eC, a.n - 1};
  }
  __device__ __forceinline__ uint32_t operator()(int i, int c) const {
    const int col = col0 + c;
    if (col >= W) return 0u;
    uint32_t acc = 0u;
    int row = i;
    for (int m = 0; m < C && row < k; ++m, row += L) {
      if (!dbg_in(row, k)) break;
      const uint32_t v = src[(size_t)row * ld + col];
      acc = m == 0 ? v : m_add(acc, m_rot_rt(v, (uint32_t)(eC * m * cc)));
    }
    if (cc != 0) acc = m_mul(acc, __ldg(powf + ((i * cc) & nmask)));
    return acc;
  }
};

// Rows [row0, row0 + L) of a u32 matrix (row0 = ty * L for tile row ty).
template <int WT>
struct LoadRows32 {
  const uint32_t* in;
  size_t ld;
  size_t row0;
  int col0, W;
  uint32_t rmul, nmask;
  static __device__ __forceinline__ LoadRows32 make(const KArgs& a, int tx, int ty) {
    return LoadRows32{static_cast<const uint32_t*>(a.in), a.ld_in, (size_t)ty * a.L,
                      tx * WT, a.W, a.in_row_mul, (uint32_t)a.n - 1u};
  }
  __device__ __forceinline__ uint32_t operator()(int i, int c) const {
    const int col = col0 + c;
    if (col >= W) return 0u;
    size_t row = row0 + i;
    if (rmul != 1u) row = (rmul * (uint32_t)row) & nmask;
    if (!dbg_in((long long)row, (long long)nmask + 1)) return 0u;
    return in[row * ld + col];
  }
};

// Decode step 4 + the scatter of step 5 (Sec. II.B): the length-n vector
// u[z] = v_i * c_i at z = z_i (the first k received positions), 0 elsewhere,
// with c_i = -r^(-z_i) / A'(r^(z_i)) from the pattern table (weight 0 marks
// an unused position).  Received values above 65536 are flagged once per
// thread at the end of the kernel (see flush()).  With CG the table and the
// received words are read through L2 (see ld_tab).
template <int WT, bool CG = false>
struct LoadRecv {
  const uint32_t* recv;
  size_t ld;
  const uint2* pat;
  int* status;
  int col0, W, slots;
  uint32_t bad;
  int rows;  // rows of the received matrix: n (slots) or the first k positions (packed)
  static __device__ __forceinline__ LoadRecv make(const KArgs& a, int tx, int ty) {
    (void)ty;
    return LoadRecv{static_cast<const uint32_t*>(a.in), a.ld_in, a.pat, a.status, tx * WT, a.W,
                    a.slots, 0u, a.slots ? a.n : a.k};
  }
  __device__ __forceinline__ uint32_t operator()(int i, int c) {
    const int col = col0 + c;
    const uint2 e = ld_tab<CG>(pat + i);
    uint32_t v = 0u;
    if (e.y != 0u && col < W) {
      const size_t row = slots ? (size_t)i : (size_t)e.x;
      if (!dbg_in((long long)row, rows, status)) return 0u;
      v = CG ? __ldcg(recv + row * ld + col) : recv[row * ld + col];
    }
    bad |= v > 65536u ? 1u : 0u;
    return m_mul(v, e.y);
  }
  __device__ __forceinline__ void flush() const {
    if (bad) atomicOr(status, ST_RANGE);
  }
};

// N consecutive words at p (aligned to min(4N, 16) bytes) in the widest
// accesses that alignment allows; the stores are streaming (evict-first).
template <int N>
__device__ __forceinline__ void ld_words(const uint32_t* p, uint32_t (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int u = 0; u < N / 4; ++u) {
      const uint4 t = reinterpret_cast<const uint4*>(p)[u];
      v[4 * u] = t.x, v[4 * u + 1] = t.y, v[4 * u + 2] = t.z, v[4 * u + 3] = t.w;
    }
  } else if constexpr (N == 2) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    v[0] = t.x, v[1] = t.y;
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) v[c] = p[c];
  }
}

template <int N>
__device__ __forceinline__ void st_words(uint32_t* p, const uint32_t (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int u = 0; u < N / 4; ++u)
      reinterpret_cast<uint4*>(p)[u] = make_uint4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) p[c] = v[c];
  }
}

template <int N>
__device__ __forceinline__ void st_words_cs(uint32_t* p, const uint32_t (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int u = 0; u < N / 4; ++u)
      __stcs(reinterpret_cast<uint4*>(p) + u,
             make_uint4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]));
  } else if constexpr (N == 2) {
    __stcs(reinterpret_cast<uint2*>(p), make_uint2(v[0], v[1]));
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) __stcs(p + c, v[c]);
  }
}

// ---------------------------------------------------------------------------
// Storers: spectrum index j of tile codeword c.
// ---------------------------------------------------------------------------

// 16-bit wire output (Sec. II.B: every symbol but 65536 fits 16 bits; the
// positions of 65536 travel separately): the low 16 bits of v in [0, p) go
// to row `row`, column `col` of the u16 matrix, and a 65536 is listed in the
// escape array.  The escape is rare (one symbol in 65537 on random data), so
// the atomic is off the common path.
struct WireOut {
  uint16_t* out;
  size_t ld;
  uint2* esc;
  uint32_t* count;
  uint32_t cap;
  int rows, col_base;
  static __device__ __forceinline__ WireOut make(const KArgs& a) {
    return WireOut{static_cast<uint16_t*>(a.out), a.ld_out, a.esc, a.esc_count, a.esc_cap,
                   a.wire_rows, a.col_base};
  }
  __device__ __forceinline__ void escape(uint32_t row, int col) const {
    const uint32_t i = atomicAdd(count, 1u);
    if (i < cap) esc[i] = make_uint2(row, (uint32_t)(col_base + col));
  }
  __device__ __forceinline__ void put(uint32_t row, int col, uint32_t v) const {
    if (row >= (uint32_t)rows) return;
    out[(size_t)row * ld + col] = (uint16_t)v;
    if (v == 65536u) escape(row, col);
  }
};

// out row = cc + C*j, value reduced to [0, p) and optionally scaled.
template <int WT>
struct StoreRows32 {
  uint32_t* out;
  size_t ld;
  int col0, W, C, cc;
  uint32_t scale, rmul, nmask;
  int wire;
  WireOut wo;
  static __device__ __forceinline__ StoreRows32 make(const KArgs& a, int tx, int ty) {
    return StoreRows32{static_cast<uint32_t*>(a.out), a.ld_out, tx * WT, a.W, a.C, ty, a.scale,
                       a.row_mul, (uint32_t)a.n - 1u, a.wire, WireOut::make(a)};
  }
  __device__ __forceinline__ void operator()(int j, int c, uint32_t v) const {
    const int col = col0 + c;
    if (col >= W) return;
    if (scale != 1u) v = m_mul(v, scale);
    uint32_t row = (uint32_t)(cc + C * j);
    if (rmul != 1u) row = (rmul * row) & nmask;
    if (!dbg_in(row, (long long)nmask + 1)) return;
    if (wire)
      wo.put(row, col, m_to_p(v));
    else
      out[(size_t)row * ld + col] = m_to_p(v);
  }
};

// Reduce to [0, p); 65536 (no 16-bit symbol) becomes 0 and raises `bad`
// (a running maximum: bad ends at 65536 iff one value was out of range).
__device__ __forceinline__ uint16_t to_symbol(uint32_t v, uint32_t& bad) {
  const uint32_t r = m_to_p(v);
  bad = max(bad, r);
  return (uint16_t)r;
}

// Local pass of a split transform (n = C * L): spectrum index j of block j1
// is row j1 + C*j of the full transform, stored according to MODE (kargs.h).
// With CG the pointwise tables are read through L2 only (written by other CTAs
// of the same launch).
template <int MODE, bool CG = false>
__device__ __forceinline__ void local_store(const KArgs& a, int j1, int j, int col, uint32_t v,
                                            uint32_t& bad) {
  const size_t row = (size_t)j1 + (size_t)a.C * j;
  if (!dbg_in((long long)row, a.n, a.status)) return;
  if constexpr (MODE == LM_ENC || MODE == LM_FNT) {
    if (MODE == LM_FNT && a.scale != 1u) v = m_mul(v, a.scale);
    const size_t orow =
        a.row_mul == 1u ? row : ((a.row_mul * (uint32_t)row) & (uint32_t)(a.n - 1));
    if (MODE == LM_ENC && a.wire)
      WireOut::make(a).put((uint32_t)orow, col, m_to_p(v));
    else
      static_cast<uint32_t*>(a.out)[orow * a.ld_out + col] = m_to_p(v);
  } else if constexpr (MODE == LM_WORK) {
    if ((int)row < a.out_limit) static_cast<uint32_t*>(a.out2)[row * a.ld_work + col] = v;
  } else if constexpr (MODE == LM_WORK_AHAT) {
    static_cast<uint32_t*>(a.out2)[row * a.ld_work + col] = m_mul(v, ld_tab<CG>(a.ahat + row));
  } else if constexpr (MODE == LM_OUT16) {
    if ((int)row < a.out_limit) {
      if (a.scale != 1u) v = m_mul(v, a.scale);
      if (a.out32)
        static_cast<uint32_t*>(a.out32)[row * a.ld_out + col] = m_to_p(v);
      else
        static_cast<uint16_t*>(a.out)[row * a.ld_out + col] = to_symbol(v, bad);
    }
  } else if constexpr (MODE == LM_SPLIT) {
    if ((int)row < a.h)
      static_cast<uint32_t*>(a.out2)[row * a.ld_work + col] = v;
    else if ((int)row < a.out_limit)
      static_cast<uint32_t*>(a.out3)[(row - a.h) * a.ld_work + col] = v;
  } else if constexpr (MODE == LM_X_PARTIAL) {
    const uint32_t vp = m_to_p(v);
    static_cast<uint32_t*>(a.out2)[row * a.ld_work + col] = m_mul(vp, ld_tab<CG>(a.ahat + row));
    static_cast<uint32_t*>(a.out3)[row * a.ld_work + col] = m_mul(vp, ld_tab<CG>(a.ahat2 + row));
  } else if constexpr (MODE == LM_ACCUM) {
    uint32_t* p = static_cast<uint32_t*>(a.out3) + row * a.ld_work + col;
    *p = m_add(*p, m_mul(v, ld_tab<CG>(a.ahat + row)));
  } else if constexpr (MODE == LM_OUT16_ADD) {
    if ((int)row < a.out_limit) {
      if ((int)row >= a.h)
        v = m_add(v, static_cast<const uint32_t*>(a.in2)[(row - a.h) * a.ld_work + col]);
      if (a.out32)
        static_cast<uint32_t*>(a.out32)[row * a.ld_out + col] = m_to_p(v);
      else
        static_cast<uint16_t*>(a.out)[row * a.ld_out + col] = to_symbol(v, bad);
    }
  }
}

template <int WT, int MODE>
struct StoreLocal {
  KArgs a;
  int col0, j1;
  uint32_t bad;
  static __device__ __forceinline__ StoreLocal make(const KArgs& a, int tx, int ty) {
    return StoreLocal{a, tx * WT, ty, 0u};
  }
  __device__ __forceinline__ void operator()(int j, int c, uint32_t v) {
    const int col = col0 + c;
    if (col >= a.W) return;
    local_store<MODE>(a, j1, j, col, v, bad);
  }
  __device__ __forceinline__ void flush() const {
    if (bad > 65535u) atomicOr(a.status, ST_RANGE);
  }
};

// The same with the mode chosen at run time (a.mode; uniform over the CTA), for
// the persistent kernel, which runs every mode through one tile body.
template <int WT, bool CG>
struct StoreLocalRT {
  KArgs a;
  int col0, j1;
  uint32_t bad;
  static __device__ __forceinline__ StoreLocalRT make(const KArgs& a, int tx, int ty) {
    return StoreLocalRT{a, tx * WT, ty, 0u};
  }
  __device__ __forceinline__ void operator()(int j, int c, uint32_t v) {
    const int col = col0 + c;
    if (col >= a.W) return;
    switch (a.mode) {
      case LM_ENC: local_store<LM_ENC, CG>(a, j1, j, col, v, bad); break;
      case LM_FNT: local_store<LM_FNT, CG>(a, j1, j, col, v, bad); break;
      case LM_WORK: local_store<LM_WORK, CG>(a, j1, j, col, v, bad); break;
      case LM_WORK_AHAT: local_store<LM_WORK_AHAT, CG>(a, j1, j, col, v, bad); break;
      case LM_OUT16: local_store<LM_OUT16, CG>(a, j1, j, col, v, bad); break;
      case LM_SPLIT: local_store<LM_SPLIT, CG>(a, j1, j, col, v, bad); break;
      case LM_X_PARTIAL: local_store<LM_X_PARTIAL, CG>(a, j1, j, col, v, bad); break;
      case LM_ACCUM: local_store<LM_ACCUM, CG>(a, j1, j, col, v, bad); break;
      default: local_store<LM_OUT16_ADD, CG>(a, j1, j, col, v, bad); break;
    }
  }
  __device__ __forceinline__ void flush() const {
    if (bad > 65535u) atomicOr(a.status, ST_RANGE);
  }
};

template <class T>
__device__ __forceinline__ auto flush_if_any(const T& t, int) -> decltype(t.flush(), void()) {
  t.flush();
}
template <class T>
__device__ __forceinline__ void flush_if_any(const T&, long) {}

// ---------------------------------------------------------------------------
// Generic tile transform: DIF passes from a loader to a storer.
// grid = (ceil(W / WT), classes or blocks), dynamic smem = Lay WORDS * 4 bytes.
// ---------------------------------------------------------------------------
template <class S, int WT, int NT, bool INV, class LD, class ST>
__device__ __forceinline__ void tile_body(const KArgs& a, int tx, int ty) {
  extern __shared__ uint4 smem_raw[];
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw);
  LD load = LD::make(a, tx, ty);
  ST store = ST::make(a, tx, ty);
  const uint32_t* tw = INV ? a.twi : a.twf;
  dif_first<S, WT, NT, INV>(sm, tw, load, store);
  if constexpr (S::NP >= 2) {
    __syncthreads();
    if constexpr (S::NP == 3) {
      dif_mid<S, WT, NT, INV>(sm, tw + S::TW2_OFF);
      __syncthreads();
    }
    dif_last<S, WT, NT, INV>(sm, store);
  }
  flush_if_any(store, 0);
}

template <class S, int WT, int NT, bool INV, class LD, class ST>
__global__ void __launch_bounds__(NT) k_tile(KArgs a) {
  dbg_enter(a.status);
  tile_body<S, WT, NT, INV, LD, ST>(a, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Stage hand-over of the one-stage TMA kernels (k_encode_tma, k_decode_tma):
// one producer thread takes over tiles of CTAs not yet launched (cluster
// launch control) and issues each tile's stage loads; the transforming
// threads never wait for that issue.  Issuing a stage takes the producer a
// few thousand cycles (the TMA unit accepts a box only as fast as it works
// through the box's 16-byte rows), time the transforming threads would
// otherwise spend waiting for it at their next barrier.
// kSchedBytes at `bar`: [0] full (the stage has landed; *s_tile, written
// before the producer's arrival, names its tile, ntiles none), [1] cancel
// response barrier, [2] empty (the transforming threads have read the
// stage: `arrivals` arrivals), [3] tables (TABLES below), the 16-byte cancel
// response at byte 32.
// TABLES: between two tiles the stage also carries tables for a later pass:
// once the stage has been read, tables() copies them in (completing
// table_bytes on bar[3]), and the next tile is loaded after a second arrival
// on bar[2] (the tables have been read).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t* tma_empty_bar(uint64_t* bar) { return bar + 2; }
__device__ __forceinline__ uint64_t* tma_tables_bar(uint64_t* bar) { return bar + 3; }

__device__ __forceinline__ void tma_producer_init(uint64_t* bar, uint32_t arrivals = 1) {
  mbar_init(bar, 1);
  mbar_init(bar + 1, 1);
  mbar_init(bar + 2, arrivals);
  mbar_init(bar + 3, 1);
}

// issue(t): the loads of tile t's stage, completing on bar[0]
template <bool TABLES = false, class Issue, class Tables = int>
__device__ __forceinline__ void tma_producer(uint64_t* bar, int* s_tile, int* status, int ntiles,
                                             uint32_t tx_bytes, Issue&& issue,
                                             Tables&& tables = 0, uint32_t table_bytes = 0) {
  uint64_t* cbar = bar + 1;
  uint64_t* ebar = bar + 2;
  uint4* resp = reinterpret_cast<uint4*>(bar + 4);
  auto start = [&](int t) {
    *s_tile = t;
    mbar_expect_tx(bar, tx_bytes);  // this thread's arrival, plus the stage's bytes
    issue(t);
  };
  int tile = blockIdx.x;
  if (tile >= ntiles) {
    *s_tile = ntiles;
    mbar_arrive(bar);
    return;
  }
  start(tile);
  clc_request(resp, cbar);
  uint32_t ephase = 0, cphase = 0, fphase = 0, tphase = 0;
  while (tile < ntiles) {
    if (!mbar_wait(ebar, ephase)) {
      atomicOr(status, ST_TIMEOUT);
      mbar_wait(bar, fphase);  // let the copy in flight land
      mbar_wait(cbar, cphase);
      return;
    }
    ephase ^= 1u;
    fphase ^= 1u;
    if constexpr (TABLES) {
      fence_proxy_async();
      mbar_expect_tx(bar + 3, table_bytes);
      tables();
      if (!mbar_wait(ebar, ephase)) {
        atomicOr(status, ST_TIMEOUT);
        mbar_wait(bar + 3, tphase);  // let the copies in flight land
        mbar_wait(cbar, cphase);
        return;
      }
      ephase ^= 1u;
      tphase ^= 1u;
    }
    int nxt = clc_take(resp, cbar, cphase);
    if (nxt == kClcTimeout) atomicOr(status, ST_TIMEOUT);
    if (nxt >= 0 && nxt < ntiles) {
      fence_proxy_async();
      start(nxt);
      clc_request(resp, cbar);
    } else {
      nxt = ntiles;
      *s_tile = ntiles;
      mbar_arrive(bar);  // no bytes: the phase completes and the transforming threads stop
    }
    tile = nxt;
  }
}

// ---------------------------------------------------------------------------
// Encode with TMA-staged source (n = C * L, C in {1, 2}, k <= L).  One CTA
// per column tile of WT codewords; a running CTA takes over tiles of CTAs not
// yet launched (cluster launch control, see clc_take), and the [k][WT] source
// tile it takes over is brought into shared memory by cp.async.bulk.tensor
// while the current tile is still being transformed.  For C = 2 the tile feeds both output classes:
// class 1 takes x[i] = s_i r_n^i; with i = q*S1 + i2 the factor r_n^(q*S1) is
// a power of two (r_n^S1 has order 2*R1 <= 32) and r_n^i2 rides on the pass-1
// twiddle table twc (all R1 entries).
// smem: work (Lay WORDS u32) | stage (rows_staged * WT u16) | barriers and
// cancel response (kSchedBytes).
// ---------------------------------------------------------------------------
// Roles as in k_decode_tma: NT threads transform, one more warp (its lane 0)
// takes over tiles and issues their stage loads (tma_producer).
template <class S, int WT, int NT, int C>
__global__ void __launch_bounds__(NT + 32, 1)
    k_encode_tma(KArgs a, const uint32_t* __restrict__ twc, int rows_staged, int box_rows,
                 const __grid_constant__ CUtensorMap tsrc) {
  static_assert(S::NP == 3 || S::NP == 2, "");
  static_assert(C == 1 || (C == 2 && 2 * S::R1 <= 32), "");
  dbg_enter(a.status);
  using Y = Lay<S, WT>;
  using Sync = FirstSync<NT>;
  constexpr int R = S::R1, SP = S::S1, B = ilog2(R);
  constexpr int WORK_BYTES = ((Y::WORDS * 4) + 127) / 128 * 128;
  extern __shared__ __align__(128) uint4 smem_raw[];
  uint32_t* work = reinterpret_cast<uint32_t*>(smem_raw);
  uint16_t* stage = reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(smem_raw) + WORK_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(stage) +
                                              (size_t)rows_staged * WT * 2);
  __shared__ int s_tile;
  const int ntiles = (a.W + WT - 1) / WT;
  const int nbox = rows_staged / box_rows;
  const uint32_t tx_bytes = (uint32_t)rows_staged * WT * 2;
  if (threadIdx.x == 0) tma_producer_init(bar);
  __syncthreads();
  if (threadIdx.x >= NT) {
    if (threadIdx.x == NT)
      tma_producer(bar, &s_tile, a.status, ntiles, tx_bytes, [&](int t) {
        for (int bx = 0; bx < nbox; ++bx)
          tma_load_2d(stage + (size_t)bx * box_rows * WT, &tsrc, t * WT, bx * box_rows, bar);
      });
    return;
  }
  uint32_t parity = 0;
  uint32_t* out = static_cast<uint32_t*>(a.out);
  const size_t ld = a.ld_out;
  for (;;) {
    const bool ok = mbar_wait(bar, parity);
    if (first_sync_or<NT>(!ok)) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_TIMEOUT);
      return;
    }
    parity ^= 1u;
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int col0 = tile * WT;
#pragma unroll 1
    for (int cc = 0; cc < C; ++cc) {
      // pass 1 from the staged source
      for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
        const int c = t % WT, i2 = t / WT;
        uint32_t x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int row = q * SP + i2;
          x[q] = row < rows_staged ? (uint32_t)stage[row * WT + c] : 0u;
        }
        if (C == 2 && cc == 1) {
          constexpr int e = Pow2Root<(2 * R > 32 ? 32 : 2 * R)>::e;
#pragma unroll
          for (int q = 1; q < R; ++q) x[q] = m_rot_rt(x[q], (uint32_t)(e * q));
        }
        dft_reg<R, false>(x);
        if (C == 2 && cc == 1) {
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
      Sync::sync();
      // the stage is free for the producer once the last class has read it
      if (cc == C - 1 && threadIdx.x == 0) mbar_arrive(tma_empty_bar(bar));
      if constexpr (S::NP == 3) {
        dif_mid<S, WT, NT, false>(work, a.twf + S::TW2_OFF);
        mid_last_sync<S, WT, NT, Sync>();  // the last pass reads only its group's blocks
      }
      // last pass -> encoded rows cc + C*j
      {
        constexpr int RL = S::RL, BL = ilog2(RL);
        for (int t = threadIdx.x; t < (S::L / RL) * WT; t += NT) {
          const int c = t % WT, b = t / WT;
          if (!dbg_in(cc + C * (S::natural(b * RL) + (RL - 1) * (S::L / RL)), C * S::L) ||
              !dbg_in(b * Y::LAST_B + c + (RL - 1) * WT, Y::WORDS))
            continue;
          const uint32_t* base = work + b * Y::LAST_B + c;
          uint32_t x[RL];
#pragma unroll
          for (int q = 0; q < RL; ++q) x[q] = base[q * WT];
          dft_reg<RL, false>(x);
          const int col = col0 + c;
          if (col < a.W) {
            if (a.wire) {
              // 16-bit symbols: same addressing as below; rows past wire_rows
              // (a punctured code) and escapes take the rare branches
              const uint32_t row0 = (uint32_t)(cc + C * S::natural(b * RL));
              constexpr uint32_t rstep = (uint32_t)(C * (S::L / RL));
              uint16_t* o = static_cast<uint16_t*>(a.out) + (size_t)row0 * ld + col;
              const size_t step = (size_t)rstep * ld;
              const bool all_rows = a.wire_rows >= C * S::L;
#pragma unroll
              for (int q = 0; q < RL; ++q) {
                const uint32_t v = m_to_p(x[q]);
                const uint32_t row = row0 + bitrev(q, BL) * rstep;
                if (all_rows || row < (uint32_t)a.wire_rows) {
                  o[bitrev(q, BL) * step] = (uint16_t)v;
                  if (v == 65536u) WireOut::make(a).escape(row, col);
                }
              }
            } else {
              // streaming stores (evict first): the encoded words are not read
              // again here, so their lines leave L2 while this kernel still
              // computes instead of being written back during the next kernel
              uint32_t* o = out + (size_t)(cc + C * S::natural(b * RL)) * ld + col;
              const size_t step = (size_t)C * (S::L / RL) * ld;
#pragma unroll
              for (int q = 0; q < RL; ++q) __stcs(o + bitrev(q, BL) * step, m_to_p(x[q]));
            }
          }
        }
      }
      Sync::sync();
    }
  }
}

// ---------------------------------------------------------------------------
// Cross pass of a split transform n = C * L (C <= 16): for every i2 < L and
// column, the radix-C DFT over rows i1*L + i2 followed by the twiddle
// r_n^(+-i2*j1); result row j1*L + i2 of the workspace matrix out2.
// ---------------------------------------------------------------------------
// One (i2, column) of the cross pass.  With CG the pattern table and the
// received words are read through L2 only (they may have been written by
// other CTAs of the same launch).  `bad` collects received values above 65536.
template <int C, bool INV, int LOADM, bool CG = false>
__device__ __forceinline__ void cross_one(const KArgs& a, int i2, int col, uint32_t& bad) {
  uint32_t x[C];
#pragma unroll
  for (int q = 0; q < C; ++q) {
    const int row = q * a.L + i2;
    if (!dbg_in(row, a.n, a.status)) {
      x[q] = 0u;
      continue;
    }
    if constexpr (LOADM == CL_SRC16) {
      x[q] = row < a.row_limit
                 ? (uint32_t) static_cast<const uint16_t*>(a.in)[(size_t)row * a.ld_in + col]
                 : 0u;
    } else if constexpr (LOADM == CL_U32) {
      const uint32_t r = a.in_row_mul == 1u
                             ? (uint32_t)row
                             : ((a.in_row_mul * (uint32_t)row) & (uint32_t)(a.n - 1));
      x[q] = row < a.row_limit ? static_cast<const uint32_t*>(a.in)[(size_t)r * a.ld_in + col]
                               : 0u;
    } else {
      const uint2 e = ld_tab<CG>(a.pat + row);
      uint32_t v = 0u;
      if (e.y != 0u && dbg_in(a.slots ? 0 : (long long)e.x, a.k, a.status)) {
        const size_t rr = a.slots ? (size_t)row : (size_t)e.x;
        const uint32_t* src = static_cast<const uint32_t*>(a.in) + rr * a.ld_in + col;
        v = CG ? __ldcg(src) : *src;
      }
      bad |= v > 65536u ? 1u : 0u;
      x[q] = m_mul(v, e.y);
    }
  }
  dft_reg<C, INV>(x);
  const uint32_t* pw = INV ? a.powi : a.powf;
  constexpr int B = ilog2(C);
  uint32_t* out = static_cast<uint32_t*>(a.out2);
#pragma unroll
  for (int q = 0; q < C; ++q) {
    const int j1 = bitrev(q, B);
    uint32_t v = x[q];
    if (j1 != 0) v = m_mul(v, __ldg(pw + (((long long)i2 * j1) & (a.n - 1))));
    out[((size_t)j1 * a.L + i2) * a.ld_work + col] = v;
  }
}

template <int C, bool INV, int LOADM>
__global__ void __launch_bounds__(256) k_cross(KArgs a) {
  const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
  const int col = (int)(t % a.W);
  const long long i2l = t / a.W;
  if (i2l >= a.L) return;
  uint32_t bad = 0u;
  cross_one<C, INV, LOADM>(a, (int)i2l, col, bad);
  if (bad) atomicOr(a.status, ST_RANGE);
}

// ---------------------------------------------------------------------------
// Fused decode for n = L <= tile limit and k <= n/2 (Sec. II.B steps 4-6):
//   T = FNT_n with root r^-1 of u (DIF, slots),  S_j = T_j for j < k,
//   F = FNT_n(S) (DIT, natural),  G = F * ahat  (ahat = n^-1 FNT_n(A mod x^k)),
//   P = FNT_n with root r^-1 of G (DIF), out_j = P_j for j < k.
// The boundary passes of consecutive transforms act on the same register
// groups and are fused.
// ---------------------------------------------------------------------------
// With out32 set the coefficients go there as u32 in [0, p) (all of F_p, as
// the systematic code's intermediate symbols need) instead of 16-bit symbols.
template <int WT>
struct StoreOut16 {
  uint16_t* out;
  uint32_t* out32;
  size_t ld;
  int* status;
  int col0, W, k;
  uint32_t bad;
  bool vec;  // row segments of WT columns start on a boundary of their own size (<= 16 bytes)
  static __device__ __forceinline__ StoreOut16 make(const KArgs& a, int tx, int ty) {
    (void)ty;
    const int vb = a.out32 ? (4 * WT < 16 ? 4 * WT : 16) : (2 * WT < 16 ? 2 * WT : 16);
    const int es = a.out32 ? 4 : 2;
    const uintptr_t base = a.out32 ? (uintptr_t)a.out32 : (uintptr_t)a.out;
    const bool vec = base % vb == 0 && (a.ld_out * es) % vb == 0;
    return StoreOut16{static_cast<uint16_t*>(a.out), static_cast<uint32_t*>(a.out32), a.ld_out,
                      a.status, tx * WT, a.W, a.k, 0u, vec};
  }
  // the WT columns col0.. of row j < k at once, values already in [0, p): one
  // wide store when the segment is aligned and inside the matrix
  // (as operator(): 65536 is out of range only for the 16-bit symbols)
  __device__ __forceinline__ void row(int j, const uint32_t (&v)[WT]) {
    const bool whole = vec && col0 + WT <= W;
    if (out32) {
      uint32_t* p = out32 + (size_t)j * ld + col0;
      if (whole) {
        st_words_cs<WT>(p, v);
      } else {
#pragma unroll
        for (int c = 0; c < WT; ++c)
          if (col0 + c < W) __stcs(p + c, v[c]);
      }
      return;
    }
    uint32_t m = v[0];
#pragma unroll
    for (int c = 1; c < WT; ++c) m = max(m, v[c]);
    bad = max(bad, m);
    uint16_t* p = out + (size_t)j * ld + col0;
    if constexpr (WT >= 2) {
      if (whole) {
        uint32_t h[WT / 2];
#pragma unroll
        for (int u = 0; u < WT / 2; ++u) h[u] = __byte_perm(v[2 * u], v[2 * u + 1], 0x5410);
        st_words_cs<WT / 2>(reinterpret_cast<uint32_t*>(p), h);
        return;
      }
    }
#pragma unroll
    for (int c = 0; c < WT; ++c)
      if (col0 + c < W) __stcs(p + c, (uint16_t)v[c]);
  }
  __device__ __forceinline__ void operator()(int j, int c, uint32_t v) {
    const int col = col0 + c;
    if (col >= W || j >= k) return;
    // streaming stores: the decoded symbols are not read again by this kernel
    if (out32)
      __stcs(out32 + (size_t)j * ld + col, m_to_p(v));
    else
      __stcs(out + (size_t)j * ld + col, to_symbol(v, bad));
  }
  __device__ __forceinline__ void flush() const {
    if (bad > 65535u) atomicOr(status, ST_RANGE);
  }
};

// Lossless decode (nothing erased, Sec. II.B): out row j < k = n^-1-scaled
// inverse transform value j as a 16-bit symbol.
template <int WT>
struct StoreFirstK16 {
  uint16_t* out;
  size_t ld;
  int* status;
  int col0, W, k;
  uint32_t scale, bad;
  static __device__ __forceinline__ StoreFirstK16 make(const KArgs& a, int tx, int ty) {
    (void)ty;
    return StoreFirstK16{static_cast<uint16_t*>(a.out), a.ld_out, a.status, tx * WT, a.W, a.k,
                         a.scale, 0u};
  }
  __device__ __forceinline__ void operator()(int j, int c, uint32_t v) {
    const int col = col0 + c;
    if (col >= W || j >= k) return;
    out[(size_t)j * ld + col] = to_symbol(m_mul(v, scale), bad);
  }
  __device__ __forceinline__ void flush() const {
    if (bad > 65535u) atomicOr(status, ST_RANGE);
  }
};

struct NopStore {
  __device__ __forceinline__ void operator()(int, int, uint32_t) const {}
};

// ---------------------------------------------------------------------------
// Local pass of a split transform fused with the cross pass of the next one
// (n = C * L, L = 4096 as 16 * 16 * 16, C in {4, 8, 16}).  Block j1 of the
// current transform yields X[j1 + C j'] for j' < L; the next transform's cross
// DFT for i2 (inputs at rows q L + i2, q < C) needs exactly the outputs of
// block j1 = i2 mod C at j' = i2 div C + q (L / C).  In the last radix-16 pass
// a task holds the 16 outputs j' = j0 + 256 t (t < 16, j0 < 256), which are
// 16 / C such groups (t = g + (16 / C) u, u < C): the task runs those C-point
// DFTs right away, in registers, instead of writing the local outputs to
// global memory and reading them back in a separate cross pass.  Before the
// cross DFT the values at full indices s >= row_limit are zeroed (the
// truncation to j < k between D1 and D2) and, with AHAT, multiplied by ahat[s]
// (the pointwise product between D2 and D3).  Output: rows j1'' L + i2 of out2
// (ld_work), the same layout the cross pass writes.  Used by the persistent
// ragged kernel's split items, whose cross passes one CTA runs alone (as a
// separate pass each is bound by memory latency); the standalone split path
// keeps separate cross kernels (fused there it measured 1.38 against 1.33 ms
// at k = 32768, n = 65536, W = 1024: its cross kernels are cheap, many small
// CTAs per SM).
// ---------------------------------------------------------------------------
template <class S, int WT, int NT, bool INV_LOCAL, int C, bool INV_CROSS, bool AHAT,
          bool CG = false>
__device__ __forceinline__ void local_cross_last(const uint32_t* sm, const KArgs& a, int j1,
                                                 int col0) {
  static_assert(S::NP == 3 && S::RL == 16 && S::L == 4096 && (C == 4 || C == 8 || C == 16), "");
  using Y = Lay<S, WT>;
  constexpr int R = 16, G = 16 / C, B = 4, BC = ilog2(C);
  const uint32_t* pw = INV_CROSS ? a.powi : a.powf;
  uint32_t* out = static_cast<uint32_t*>(a.out2);
  for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
    const int c = t % WT, b = t / WT;
    const int col = col0 + c;
    if (!dbg_in(b * Y::LAST_B + c + (R - 1) * WT, Y::WORDS)) continue;
    const uint32_t* base = sm + b * Y::LAST_B + c;
    uint32_t x[R];
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = base[q * WT];
    dft_reg<R, INV_LOCAL>(x);
    if (col >= a.W) continue;
    const int j0 = S::natural(b * R);  // register q holds j' = j0 + 256 bitrev(q)
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int m = j0 + 256 * g;   // j' = m + (L / C) u
      const int i2 = j1 + C * m;    // the next transform's cross index
      uint32_t y[C];
#pragma unroll
      for (int u = 0; u < C; ++u) {
        uint32_t v = x[bitrev(g + G * u, B)];
        const int srow = i2 + S::L * u;  // full index of this value
        if constexpr (AHAT) v = m_mul(v, ld_tab<CG>(a.ahat + srow));
        y[u] = srow < a.row_limit ? v : 0u;
      }
      dft_reg<C, INV_CROSS>(y);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const int jn = bitrev(r, BC);  // the next transform's local block
        uint32_t v = y[r];
        if (jn != 0) v = m_mul(v, __ldg(pw + (((long long)i2 * jn) & (a.n - 1))));
        if (!dbg_in((long long)jn * S::L + i2, a.n, a.status)) continue;
        out[((size_t)jn * S::L + i2) * a.ld_work + col] = v;
      }
    }
  }
}



template <class S, int WT, int NT, bool CG = false>
__device__ __forceinline__ void decode_body(const KArgs& a, int tx) {
  extern __shared__ uint4 smem_raw[];
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw);
  using Y = Lay<S, WT>;
  LoadRecv<WT, CG> load = LoadRecv<WT, CG>::make(a, tx, 0);
  StoreOut16<WT> store = StoreOut16<WT>::make(a, tx, 0);
  const uint32_t* __restrict__ ahat = a.ahat;
  if constexpr (S::NP == 1) {
    constexpr int R = S::L, B = ilog2(R);
    for (int c = threadIdx.x; c < WT; c += NT) {
      uint32_t x[R];
#pragma unroll
      for (int i = 0; i < R; ++i) x[i] = load(i, c);
      dft_reg<R, true>(x);
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (bitrev(q, B) >= a.k) x[q] = 0u;
      bitrev_regs<R>(x);
      dft_reg<R, false>(x);
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = m_mul(x[q], ld_tab<CG>(ahat + bitrev(q, B)));
      bitrev_regs<R>(x);
      dft_reg<R, true>(x);
#pragma unroll
      for (int q = 0; q < R; ++q) store(bitrev(q, B), c, x[q]);
    }
  } else {
    const uint32_t* tw1f = a.twf;
    const uint32_t* tw1i = a.twi;
    NopStore nop;
    // D1 passes (root r^-1), natural -> slots
    dif_first<S, WT, NT, true>(sm, tw1i, load, nop);
    __syncthreads();
    if constexpr (S::NP == 3) {
      dif_mid<S, WT, NT, true>(sm, tw1i + S::TW2_OFF);
      __syncthreads();
    }
    // last D1 pass + truncation to j < k + first D2 pass (DIT, root r)
    {
      constexpr int R = S::RL, B = ilog2(R);
      for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
        const int c = t % WT, b = t / WT;
        uint32_t* base = sm + b * Y::LAST_B + c;
        uint32_t x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = base[q * WT];
        dft_reg<R, true>(x);
        const int j0 = S::natural(b * R);
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (j0 + (S::L / R) * bitrev(q, B) >= a.k) x[q] = 0u;
        bitrev_regs<R>(x);
        dft_reg<R, false>(x);
#pragma unroll
        for (int q = 0; q < R; ++q) base[bitrev(q, B) * WT] = x[q];
      }
    }
    __syncthreads();
    if constexpr (S::NP == 3) {
      dit_mid<S, WT, NT, false>(sm, tw1f + S::TW2_OFF);
      __syncthreads();
    }
    // last D2 pass (DIT, natural output) * ahat + first D3 pass (DIF, root r^-1)
    {
      constexpr int R = S::R1, SP = S::S1, B = ilog2(R);
      for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
        const int c = t % WT, i2 = t / WT;
        uint32_t* base = sm + Y::addr(i2, c);
        uint32_t x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = base[bitrev(q, B) * Y::P1_STRIDE];
        twiddle_regs<R>(x, tw1f + i2 * R);
        bitrev_regs<R>(x);
        dft_reg<R, false>(x);
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = m_mul(x[q], ld_tab<CG>(ahat + bitrev(q, B) * SP + i2));
        bitrev_regs<R>(x);
        dft_reg<R, true>(x);
        twiddle_regs<R>(x, tw1i + i2 * R);
#pragma unroll
        for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::P1_STRIDE] = x[q];
      }
    }
    __syncthreads();
    if constexpr (S::NP == 3) {
      dif_mid<S, WT, NT, true>(sm, tw1i + S::TW2_OFF);
      __syncthreads();
    }
    dif_last<S, WT, NT, true>(sm, store);
  }
  load.flush();
  store.flush();
}

template <class S, int WT, int NT>
__global__ void __launch_bounds__(NT) k_decode(KArgs a) {
  dbg_enter(a.status);
  decode_body<S, WT, NT>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Fused decodes of staged received rows (packed layout: row i of recv holds
// the symbols of positions[i]; n = L, k <= n/2), one CTA per tile of WT
// codewords.  Same transform sequence as k_decode.  k_decode_tma (TMA stage,
// tiles of CTAs not yet launched taken over as in k_encode_tma) scatters the
// staged rows into the work buffer through rowtab[i] = (z_i << 17) | c_i;
// k_decode_cpa (cp.async stage) gathers u[z] = v_row(z) * c_z in pass 1
// through pat32[z] = (row << 17) | c_z (c_z = 0: unused).
// smem: work (Lay WORDS u32) | stage (rows_staged * WT u32) | mbarrier.
// ---------------------------------------------------------------------------
// (WT = the stage's row stride; `stage` may point at a column inside the row)
template <int WT>
struct LoadStaged {
  const uint32_t* stage;
  const uint32_t* pat32;
  uint32_t vmax;  // largest received value seen (> 65536 is out of range)
  int rows = 1 << 17;  // staged rows (the debug build checks the row index)
  // unused positions have weight 0 and row 0: the product vanishes, no branch
  __device__ __forceinline__ uint32_t operator()(int z, int c) {
    const uint32_t e = __ldg(pat32 + z);
    if (!dbg_in(e >> 17, rows)) return 0u;
    const uint32_t v = stage[(e >> 17) * WT + c];
    vmax = max(vmax, v);
    return m_mul(v, e & 0x1FFFFu);
  }
};

// Steps 4-6 (Sec. II.B) on one staged tile of WT codewords, n = L, k <= n/2,
// after the first D1 pass (root r^-1) has left its output in the slots:
// the other D1 passes, truncation to j < k, D2 = FNT with root r, * ahat and
// every D3 pass (root r^-1) but the last; boundary passes of consecutive
// transforms fused.
// HALF (k = n/2 exactly): the truncation keeps the even registers of the
// last D1 pass, so the first D2 pass sees a zero upper half, and D3 stores
// only j < n/2; the compiler drops the butterfly halves nobody reads.
// TS: the pass that multiplies by ahat reads its forward twiddles and ahat
// from shared memory, tws = [pass-1 twiddles, chunks permuted (twf_sw) | ahat]
// (L words each); hook(0) runs before that pass (in every thread: the tables
// have landed), hook(1) after the barrier that ends it (they may be
// overwritten).
template <class S, int WT, int NT, bool HALF, class Sync, bool TS, class H>
__device__ __forceinline__ void decode_mid_passes(uint32_t* sm, const KArgs& a,
                                                  const uint32_t* tws, H&& hook) {
  using Y = Lay<S, WT>;
  const uint32_t* tw1f = a.twf;
  const uint32_t* tw1i = a.twi;
  const uint32_t* __restrict__ ahat = a.ahat;
  if constexpr (S::NP == 3) {
    dif_mid<S, WT, NT, true>(sm, tw1i + S::TW2_OFF);
    mid_last_sync<S, WT, NT, Sync>();  // the last pass reads only its group's blocks
  }
  // last D1 pass + truncation to j < k + first D2 pass (DIT, root r)
  {
    constexpr int R = S::RL, B = ilog2(R);
    for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
      const int c = t % WT, b = t / WT;
      uint32_t* base = sm + b * Y::LAST_B + c;
      uint32_t x[R];
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = base[q * WT];
      dft_reg<R, true>(x);
      if constexpr (HALF) {
#pragma unroll
        for (int q = 1; q < R; q += 2) x[q] = 0u;  // j = j0 + (L/R) bitrev(q) >= n/2
        bitrev_regs<R>(x);
        dft_reg_lower<R, false>(x);
      } else {
        const int j0 = S::natural(b * R);
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (j0 + (S::L / R) * bitrev(q, B) >= a.k) x[q] = 0u;
        bitrev_regs<R>(x);
        dft_reg<R, false>(x);
      }
#pragma unroll
      for (int q = 0; q < R; ++q) base[bitrev(q, B) * WT] = x[q];
    }
  }
  if constexpr (S::NP == 3) {
    mid_last_sync<S, WT, NT, Sync>();
    dit_mid<S, WT, NT, false>(sm, tw1f + S::TW2_OFF);
    Sync::sync();
  } else {
    Sync::sync();
  }
  // last D2 pass * ahat + first D3 pass
  if constexpr (TS) hook(0);
  {
    constexpr int R = S::R1, SP = S::S1, B = ilog2(R);
    for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
      const int c = t % WT, i2 = t / WT;
      uint32_t* base = sm + Y::addr(i2, c);
      uint32_t x[R];
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = base[bitrev(q, B) * Y::P1_STRIDE];
      if constexpr (TS)
        twiddle_regs_sw<R>(x, tws + i2 * R, i2);
      else
        twiddle_regs<R>(x, tw1f + i2 * R);
      bitrev_regs<R>(x);
      dft_reg<R, false>(x);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = bitrev(q, B) * SP + i2;
        x[q] = m_mul(x[q], TS ? tws[S::L + i] : __ldg(ahat + i));
      }
      bitrev_regs<R>(x);
      dft_reg<R, true>(x);
      twiddle_regs<R>(x, tw1i + i2 * R);
#pragma unroll
      for (int q = 0; q < R; ++q) base[bitrev(q, B) * Y::P1_STRIDE] = x[q];
    }
  }
  Sync::sync();
  if constexpr (TS) hook(1);
  if constexpr (S::NP == 3) {
    dif_mid<S, WT, NT, true>(sm, tw1i + S::TW2_OFF);
    mid_last_sync<S, WT, NT, Sync>();
  }
}

// The whole decode of one staged tile, the first pass gathering its input
// through `load` (LoadStaged), the last one handing spectrum index j < k to
// `store`.  `freed()` runs (in every thread, after a barrier) once pass 1 has
// read the whole stage.
template <class S, int WT, int NT, bool HALF, class LD, class ST, class F>
__device__ __forceinline__ void decode_staged_tile(uint32_t* sm, LD& load, ST& store,
                                                   const KArgs& a, F&& freed) {
  NopStore nop;
  dif_first<S, WT, NT, true>(sm, a.twi, load, nop);
  __syncthreads();
  freed();
  decode_mid_passes<S, WT, NT, HALF, CtaSync, false>(sm, a, nullptr, [](int) {});
  dif_last_sel<S, WT, NT, true, HALF>(sm, store);
}

// Steps 4 and 5 (Sec. II.B) for a staged tile, row by row: u[z_i] = v_i c_i
// for each of the first k received rows i (z_i, c_i from rowtab[i]), written
// at the natural-order address of position z_i; the other positions of the
// buffer are zero already.  Stage row i: WT words at stage + i * sw.
template <class S, int WT, int NT>
__device__ __forceinline__ void scatter_received(uint32_t* sm, const uint32_t* stage, int sw,
                                                 const uint32_t* __restrict__ rowtab, int k,
                                                 uint32_t& vmax) {
  using Y = Lay<S, WT>;
  // U rows per thread per round, their table entries loaded together (one
  // memory latency per round instead of one per row)
  constexpr int U = WT <= 8 ? 8 : 32 / WT;
  for (int i0 = threadIdx.x; i0 < k; i0 += U * NT) {
    uint32_t e[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * NT;
      e[u] = i < k ? __ldg(rowtab + i) : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + u * NT;
      const int z = (int)(e[u] >> 17);
      const uint32_t w = e[u] & 0x1FFFFu;
      if (i >= k || !dbg_in(z, S::L)) continue;
      uint32_t v[WT];
      ld_words<WT>(stage + (size_t)i * sw, v);
#pragma unroll
      for (int c = 0; c < WT; ++c) {
        vmax = max(vmax, v[c]);
        v[c] = m_mul(v[c], w);
      }
      st_words<WT>(sm + Y::addr(z, 0), v);
    }
  }
}

// Output of a tile after dif_last_reduce: rows j < k, the WT codewords of a
// row read from its slot at once and stored by `store.row`; the slot is
// zeroed again, so that the whole buffer is zero when the next tile's
// received rows are scattered into it.  HALF (k = L/2): the slots with last
// digit below RL/2, taken in order (consecutive threads, consecutive slots).
template <class S, int WT, int NT, bool HALF>
__device__ __forceinline__ void copy_out(uint32_t* sm, StoreOut16<WT>& store, int k) {
  using Y = Lay<S, WT>;
  constexpr int R = S::RL, H = R / 2;
  constexpr int M = HALF ? S::L / 2 : S::L;
  for (int m = threadIdx.x; m < M; m += NT) {
    const int slot = HALF ? (m / H) * R + m % H : m;
    const int j = S::natural(slot);
    if (!HALF && j >= k) continue;
    if (!dbg_in(Y::addr(slot, WT - 1), Y::WORDS)) continue;
    uint32_t* p = sm + Y::addr(slot, 0);
    uint32_t v[WT], zero[WT];
    ld_words<WT>(p, v);
#pragma unroll
    for (int c = 0; c < WT; ++c) zero[c] = 0u;
    st_words<WT>(p, zero);
    store.row(j, v);
  }
}

// The decode of one staged tile with the received rows scattered into the
// (all-zero) work buffer first: `freed()` runs (in every thread, after a
// barrier) as soon as the scatter has read the stage; the first D1 pass then
// works in place, and the last D3 pass writes back reduced values for
// copy_out, which leaves the buffer zero again.
template <class S, int WT, int NT, bool HALF, class Sync, bool TS, class F, class H>
__device__ __forceinline__ void decode_scatter_tile(uint32_t* sm, const uint32_t* stage, int sw,
                                                    const uint32_t* __restrict__ rowtab,
                                                    uint32_t& vmax, StoreOut16<WT>& store,
                                                    const KArgs& a, F&& freed,
                                                    const uint32_t* tws, H&& hook) {
  scatter_received<S, WT, NT>(sm, stage, sw, rowtab, a.k, vmax);
  Sync::sync();
  freed();
  dif_first_inplace<S, WT, NT, true>(sm, a.twi);
  Sync::sync();
  decode_mid_passes<S, WT, NT, HALF, Sync, TS>(sm, a, tws, hook);
  dif_last_reduce<S, WT, NT, true, HALF>(sm, a.k);
  Sync::sync();
  copy_out<S, WT, NT, HALF>(sm, store, a.k);
}

// Tiles: the first `nfull` tiles are WT codewords wide; the columns after them
// are cut into tiles of WT/2 codewords (two per WT-wide TMA box), so that the
// last round of tiles, which would otherwise keep only part of the SMs busy,
// is spread over twice as many CTAs.  With nfull = ceil(W / WT) every tile is
// WT wide.
//
// Roles: the first NT threads decode; one more warp (its lane 0) takes over
// tiles and issues their stage loads (tma_producer).
// TS (k = n/2, L >= 4096, where the tables outgrow the L1 cache that the
// 200 KB of shared memory leave): once a tile's received rows are scattered,
// the producer copies the forward pass-1 twiddles (chunks permuted, twf_sw)
// and ahat into the stage for the pass that multiplies by ahat, and loads the
// next tile after that pass (the passes after it cover the load).
template <class S, int WT, int NT, bool HALF>
__global__ void __launch_bounds__(NT + 32, 1)
    k_decode_tma(KArgs a, const uint32_t* __restrict__ rowtab, int rows_staged, int box_rows,
                 int nfull, const __grid_constant__ CUtensorMap trecv) {
  static_assert(S::NP >= 2, "");
  dbg_enter(a.status);
  using Y = Lay<S, WT>;
  using Sync = FirstSync<NT>;
  constexpr int WH = WT >= 2 ? WT / 2 : 1;
  constexpr int WORK_BYTES = ((Y::WORDS * 4) + 127) / 128 * 128;
  extern __shared__ __align__(128) uint4 smem_raw[];
  __shared__ int s_tile;
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* stage = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(smem_raw) + WORK_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(stage + (size_t)rows_staged * WT);
  const int nwide = (a.W + WT - 1) / WT;
  if (WT < 2 || nfull > nwide) nfull = nwide;
  const int ntiles = nfull + 2 * (nwide - nfull);
  // x coordinate of the WT-wide box that holds tile t's columns
  auto box_x = [&](int t) { return t < nfull ? t * WT : (nfull + ((t - nfull) >> 1)) * WT; };
  const int nbox = rows_staged / box_rows;
  const uint32_t tx_bytes = (uint32_t)rows_staged * WT * 4;
  // (the launch guarantees rows_staged * WT >= 2 L and twf_sw set)
  constexpr bool TS = HALF && S::L >= 4096;
  if (threadIdx.x == 0) tma_producer_init(bar);
  // the work buffer starts all zero (decode_scatter_tile keeps it so)
  for (int i = threadIdx.x; i < WORK_BYTES / 16; i += NT + 32)
    smem_raw[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (threadIdx.x >= NT) {
    if (threadIdx.x == NT)
      tma_producer<TS>(
          bar, &s_tile, a.status, ntiles, tx_bytes,
          [&](int t) {
            for (int bx = 0; bx < nbox; ++bx)
              tma_load_2d(stage + (size_t)bx * box_rows * WT, &trecv, box_x(t), bx * box_rows,
                          bar);
          },
          [&]() {
            bulk_load(stage, a.twf_sw, 4u * S::L, tma_tables_bar(bar));
            bulk_load(stage + S::L, a.ahat, 4u * S::L, tma_tables_bar(bar));
          },
          8u * S::L);
    return;
  }

  // ---- decoding warps
  uint32_t parity = 0;
  uint32_t vmax = 0u;  // largest received value seen (> 65536 is out of range)
  StoreOut16<WT> store = StoreOut16<WT>::make(a, 0, 0);
  StoreOut16<WH> store_h = StoreOut16<WH>::make(a, 0, 0);
  auto freed = [&]() {
    if (threadIdx.x == 0) mbar_arrive(tma_empty_bar(bar));  // the stage is free for the producer
  };
  uint32_t tpar = 0;
  auto tables = [&](int ev) {
    if (ev == 0) {
      if (!mbar_wait(tma_tables_bar(bar), tpar)) atomicOr(a.status, ST_TIMEOUT);
      tpar ^= 1u;
    } else if (threadIdx.x == 0) {
      mbar_arrive(tma_empty_bar(bar));  // the tables have been read
    }
  };
  for (;;) {
    const bool ok = mbar_wait(bar, parity);
    if (first_sync_or<NT>(!ok)) {
      if (threadIdx.x == 0) atomicOr(a.status, ST_TIMEOUT);
      return;
    }
    parity ^= 1u;
    const int tile = s_tile;
    if (tile >= ntiles) break;
    if constexpr (WT >= 2) {
      if (tile >= nfull) {
        // a half tile: columns (tile - nfull) & 1 of its box, WH codewords
        const int h = tile - nfull;
        store_h.col0 = nfull * WT + h * WH;
        decode_scatter_tile<S, WH, NT, HALF, Sync, TS>(sm, stage + (h & 1) * WH, WT, rowtab,
                                                       vmax, store_h, a, freed, stage, tables);
        Sync::sync();
        continue;
      }
    }
    store.col0 = tile * WT;
    decode_scatter_tile<S, WT, NT, HALF, Sync, TS>(sm, stage, WT, rowtab, vmax, store, a, freed,
                                                   stage, tables);
    Sync::sync();
  }
  if (vmax > 65536u) atomicOr(a.status, ST_RANGE);
  store.flush();
  store_h.flush();
}

// ---------------------------------------------------------------------------
// The same decode with half-width tiles staged by cp.async, two CTAs per SM:
// the [k][WT] received tile (WT * 4 = 8 or 16 bytes per row, below TMA's
// 16-byte row minimum for WT = 2) is copied by all threads; while one CTA
// waits at a barrier or on shared memory the other computes.  Tiles are taken
// over as in k_decode_tma.  Received rows must start 8-byte (WT = 2) or
// 16-byte (WT = 4) aligned.
// smem: work (Lay WORDS u32) | stage (k * WT u32) | barriers and cancel response.
// ---------------------------------------------------------------------------
template <class S, int WT, int NT, bool HALF, int MINB = 2>
__global__ void __launch_bounds__(NT, MINB)
    k_decode_cpa(KArgs a, const uint32_t* __restrict__ pat32) {
  dbg_enter(a.status);
  static_assert(S::NP >= 2 && (WT == 1 || WT == 2 || WT == 4), "");
  using Y = Lay<S, WT>;
  constexpr int WORK_BYTES = ((Y::WORDS * 4) + 127) / 128 * 128;
  extern __shared__ __align__(128) uint4 smem_raw[];
  __shared__ int s_next;
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* stage = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(smem_raw) + WORK_BYTES);
  const int k = a.k;
  uint64_t* cbar = reinterpret_cast<uint64_t*>(stage + ((size_t)k * WT + 3) / 4 * 4);
  uint4* resp = reinterpret_cast<uint4*>(cbar + 2);
  const uint32_t* recv = static_cast<const uint32_t*>(a.in);
  const size_t ld = a.ld_in;
  const int ntiles = (a.W + WT - 1) / WT;
  auto issue = [&](int t) {  // all threads: copy tile t's received rows
    const int col0 = t * WT;
    const int valid = min(WT, a.W - col0) * 4;
    for (int r = threadIdx.x; r < k; r += NT)
      cp_async<WT * 4>(stage + (size_t)r * WT, recv + (size_t)r * ld + col0, valid);
    cp_async_commit();
  };
  int tile = blockIdx.x;
  if (threadIdx.x == 0) mbar_init(cbar, 1);
  __syncthreads();
  if (tile < ntiles) {
    issue(tile);
    if (threadIdx.x == 0) clc_request(resp, cbar);
  }
  uint32_t cphase = 0;
  LoadStaged<WT> load{stage, pat32, 0u, k};
  StoreOut16<WT> store = StoreOut16<WT>::make(a, 0, 0);
  while (tile < ntiles) {
    cp_async_wait_all();
    __syncthreads();
    store.col0 = tile * WT;
    decode_staged_tile<S, WT, NT, HALF>(sm, load, store, a, [&]() {
      if (threadIdx.x == 0) {
        int nxt = clc_take(resp, cbar, cphase);
        if (nxt == kClcTimeout) atomicOr(a.status, ST_TIMEOUT);
        s_next = (nxt >= 0 && nxt < ntiles) ? nxt : ntiles;
      }
      __syncthreads();
      // the stage is free: prefetch the taken-over tile, ask for the next one
      if (s_next < ntiles) {
        issue(s_next);
        if (threadIdx.x == 0) clc_request(resp, cbar);
      }
    });
    __syncthreads();
    tile = s_next;
  }
  if (load.vmax > 65536u) atomicOr(a.status, ST_RANGE);
  store.flush();
}

// ---------------------------------------------------------------------------
// Fused decode for n = L and k > n/2: the truncated product of step 6 is
// split at h = n/2 so that only length-n cyclic products occur:
//   P mod x^k = A0 S0 + x^h (A0 S1 + A1 S0),  A = A0 + x^h A1, S = S0 + x^h S1.
// Buffers X (S0 path) and Y (S1 path) in shared memory; ahat = n^-1 FNT(A0),
// ahat2 = n^-1 FNT(A1).  Output P_j = X_j + (j >= h ? Y_(j-h) : 0).
// ---------------------------------------------------------------------------

// One codeword per thread, everything in registers (L <= 32).
template <int L, int WT, int NT, bool CG>
__device__ __forceinline__ void decode_split_regs(const KArgs& a, int tx) {
  constexpr int B = ilog2(L), H = L / 2;
  LoadRecv<WT, CG> load = LoadRecv<WT, CG>::make(a, tx, 0);
  StoreOut16<WT> store = StoreOut16<WT>::make(a, tx, 0);
  for (int c = threadIdx.x; c < WT; c += NT) {
    uint32_t x[L], y[L];
#pragma unroll
    for (int i = 0; i < L; ++i) x[i] = load(i, c);
    dft_reg<L, true>(x);
    bitrev_regs<L>(x);  // x[j] = T_j
#pragma unroll
    for (int j = 0; j < H; ++j) {
      y[j] = (H + j < a.k) ? x[H + j] : 0u;
      y[j + H] = 0u;
      x[j + H] = 0u;
    }
    dft_reg<L, false>(x);
    dft_reg<L, false>(y);
#pragma unroll
    for (int q = 0; q < L; ++q) {
      const int i = bitrev(q, B);
      const uint32_t a0 = ld_tab<CG>(a.ahat + i), a1 = ld_tab<CG>(a.ahat2 + i);
      const uint32_t s0 = m_to_p(x[q]);
      x[q] = m_mul(s0, a0);
      y[q] = m_add(m_mul(y[q], a0), m_mul(s0, a1));
    }
    bitrev_regs<L>(x);
    bitrev_regs<L>(y);
    dft_reg<L, true>(x);
    dft_reg<L, true>(y);
    bitrev_regs<L>(x);
    bitrev_regs<L>(y);
#pragma unroll
    for (int j = 0; j < L; ++j) {
      uint32_t v = x[j];
      if (j >= H) v = m_add(v, y[j - H]);
      store(j, c, v);
    }
  }
  load.flush();
  store.flush();
}

template <class S, int WT, int NT, bool CG>
__device__ __forceinline__ void decode_split_smem(const KArgs& a, int tx) {
  using Y = Lay<S, WT>;
  extern __shared__ uint4 smem_raw[];
  uint32_t* X = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* Yb = X + Y::WORDS;
  LoadRecv<WT, CG> load = LoadRecv<WT, CG>::make(a, tx, 0);
  const uint32_t* tw1f = a.twf;
  const uint32_t* tw1i = a.twi;
  const int k = a.k;
  NopStore nop;
  dif_first<S, WT, NT, true>(X, tw1i, load, nop);
  __syncthreads();
  if constexpr (S::NP == 3) {
    dif_mid<S, WT, NT, true>(X, tw1i + S::TW2_OFF);
    __syncthreads();
  }
  // last D1 pass; split T_j (j < k) into S0 (j < h) and S1 (h <= j < k)
  {
    constexpr int R = S::RL, B = ilog2(R), HR = R / 2;
    for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
      const int c = t % WT, b = t / WT;
      const int off = b * Y::LAST_B + c;
      uint32_t x[R], y[R];
#pragma unroll
      for (int q = 0; q < R; ++q) x[q] = X[off + q * WT];
      dft_reg<R, true>(x);
      bitrev_regs<R>(x);  // x[d] = digit d
      const int j0 = S::natural(b * R);
#pragma unroll
      for (int d = 0; d < HR; ++d) {
        y[d] = (j0 + (S::L / R) * (d + HR) < k) ? x[d + HR] : 0u;
        y[d + HR] = 0u;
        x[d + HR] = 0u;
      }
      dft_reg<R, false>(x);
      dft_reg<R, false>(y);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        X[off + bitrev(q, B) * WT] = x[q];
        Yb[off + bitrev(q, B) * WT] = y[q];
      }
    }
  }
  __syncthreads();
  if constexpr (S::NP == 3) {
    dit_mid<S, WT, NT, false>(X, tw1f + S::TW2_OFF);
    dit_mid<S, WT, NT, false>(Yb, tw1f + S::TW2_OFF);
    __syncthreads();
  }
  // last D2 pass on both, Xf = S0^ A0^, Yf = S1^ A0^ + S0^ A1^, first D3 pass on both
  {
    constexpr int R = S::R1, SP = S::S1, B = ilog2(R);
    for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
      const int c = t % WT, i2 = t / WT;
      const int off = Y::addr(i2, c);
      uint32_t x[R], y[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        x[q] = X[off + bitrev(q, B) * Y::P1_STRIDE];
        y[q] = Yb[off + bitrev(q, B) * Y::P1_STRIDE];
      }
      twiddle_regs<R>(x, tw1f + i2 * R);
      twiddle_regs<R>(y, tw1f + i2 * R);
      bitrev_regs<R>(x);
      bitrev_regs<R>(y);
      dft_reg<R, false>(x);
      dft_reg<R, false>(y);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int i = bitrev(q, B) * SP + i2;
        const uint32_t a0 = ld_tab<CG>(a.ahat + i), a1 = ld_tab<CG>(a.ahat2 + i);
        const uint32_t s0 = m_to_p(x[q]);
        x[q] = m_mul(s0, a0);
        y[q] = m_add(m_mul(y[q], a0), m_mul(s0, a1));
      }
      bitrev_regs<R>(x);
      bitrev_regs<R>(y);
      dft_reg<R, true>(x);
      dft_reg<R, true>(y);
      twiddle_regs<R>(x, tw1i + i2 * R);
      twiddle_regs<R>(y, tw1i + i2 * R);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        X[off + bitrev(q, B) * Y::P1_STRIDE] = x[q];
        Yb[off + bitrev(q, B) * Y::P1_STRIDE] = y[q];
      }
    }
  }
  __syncthreads();
  if constexpr (S::NP == 3) {
    dif_mid<S, WT, NT, true>(X, tw1i + S::TW2_OFF);
    dif_mid<S, WT, NT, true>(Yb, tw1i + S::TW2_OFF);
    __syncthreads();
  }
  // last D3 pass on both; P_j = X_j + (j >= h ? Y_(j-h) : 0)
  uint32_t bad = 0u;
  {
    constexpr int R = S::RL, HR = R / 2;
    uint16_t* out = static_cast<uint16_t*>(a.out);
    const int col0 = tx * WT;
    for (int t = threadIdx.x; t < (S::L / R) * WT; t += NT) {
      const int c = t % WT, b = t / WT;
      const int col = col0 + c;
      const int off = b * Y::LAST_B + c;
      uint32_t x[R], y[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        x[q] = X[off + q * WT];
        y[q] = Yb[off + q * WT];
      }
      dft_reg<R, true>(x);
      dft_reg<R, true>(y);
      bitrev_regs<R>(x);
      bitrev_regs<R>(y);
      const int j0 = S::natural(b * R);
      if (col < a.W) {
#pragma unroll
        for (int d = 0; d < R; ++d) {
          const int j = j0 + (S::L / R) * d;
          uint32_t v = x[d];
          if (d >= HR) v = m_add(v, y[d - HR]);
          if (j < k) {
            if (a.out32)
              static_cast<uint32_t*>(a.out32)[(size_t)j * a.ld_out + col] = m_to_p(v);
            else
              out[(size_t)j * a.ld_out + col] = to_symbol(v, bad);
          }
        }
      }
    }
  }
  load.flush();
  if (bad > 65535u) atomicOr(a.status, ST_RANGE);
}

template <class S, int WT, int NT, bool CG = false>
__device__ __forceinline__ void decode_split_body(const KArgs& a, int tx) {
  if constexpr (S::NP == 1) {
    decode_split_regs<S::L, WT, NT, CG>(a, tx);
  } else {
    decode_split_smem<S, WT, NT, CG>(a, tx);
  }
}

template <class S, int WT, int NT>
__global__ void __launch_bounds__(NT) k_decode_split(KArgs a) {
  dbg_enter(a.status);
  decode_split_body<S, WT, NT>(a, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Log-domain pattern build for n = L <= tile limit, one launch (see pattern.cu
// and logplan.cuh for the identities).  CTA t < D: scatters the first k
// positions into shared memory (received-row index + 1, 0 = erased),
// transforms the indicator 1_R (spec = FNT_n(1_R), every CTA for itself),
// multiplies by the transform of digit t of the reversed log table and writes
// conv[j][t] = (1_R * g'_t)[j], exact integers below p.  CTA 0 also writes the
// position table.  The last CTA to finish (counter `done`, left at zero for the
// next build) turns the digits into weights, pat32 and ahat (or aval).
// smem: work (Lay<S,1> WORDS) | row index / spec (L words).
// ---------------------------------------------------------------------------
// Digit t's part of the build; returns true in the CTA that finished last
// (after it has written the tables).
template <class S, int NT>
__device__ __forceinline__ bool plan_body(const PlanArgs& pa, int t) {
  static_assert(S::NP >= 2, "");
  constexpr int L = S::L, PER = 8;
  extern __shared__ uint4 smem_raw[];
  __shared__ int s_last;
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* ind = sm + Lay<S, 1>::WORDS;
  const int k = pa.k;
  for (int z = threadIdx.x; z < L; z += NT) ind[z] = 0u;
  __syncthreads();
  for (int i0 = 0; i0 < k; i0 += NT * PER) {
    uint32_t zz[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int i = i0 + u * NT + (int)threadIdx.x;
      zz[u] = i < k ? __ldg(pa.pos + i) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (zz[u] < (uint32_t)L) ind[zz[u]] = (uint32_t)(i0 + u * NT + (int)threadIdx.x) + 1u;
  }
  __syncthreads();
  if (t == 0)
    for (int z = threadIdx.x; z < L; z += NT) {
      const uint32_t r = ind[z];
      pa.pat[z] = make_uint2(r ? r - 1u : 0xFFFFFFFFu, 0u);
    }
  // spec = FNT_n(1_R), left in ind[] (natural order) once pass 1 has read it
  struct LoadInd {
    const uint32_t* ind;
    __device__ uint32_t operator()(int i, int) const { return ind[i] != 0u ? 1u : 0u; }
  } ld1{ind};
  struct StoreSpec {
    uint32_t* spec;
    __device__ void operator()(int j, int, uint32_t v) const { spec[j] = m_to_p(v); }
  } st1{ind};
  dif_first<S, 1, NT, false>(sm, pa.twf, ld1, st1);
  __syncthreads();
  if constexpr (S::NP == 3) {
    dif_mid<S, 1, NT, false>(sm, pa.twf + S::TW2_OFF);
    __syncthreads();
  }
  dif_last<S, 1, NT, false>(sm, st1);
  __syncthreads();
  // conv[.][t] = n^-1 IFNT(spec * ghat[.][t])
  struct LoadProd {
    const uint32_t* spec;
    const uint32_t* ghat;
    int D, t;
    __device__ uint32_t operator()(int j, int) const {
      return m_mul(__ldg(ghat + (size_t)j * D + t), spec[j]);
    }
  } ld2{ind, pa.ghat, pa.D, t};
  struct StoreConv {
    uint32_t* conv;
    int D, t;
    uint32_t ninv;
    __device__ void operator()(int j, int, uint32_t v) const {
      conv[(size_t)j * D + t] = m_to_p(m_mul(v, ninv));
    }
  } st2{pa.conv, pa.D, t, pa.ninv};
  dif_first<S, 1, NT, true>(sm, pa.twi, ld2, st2);
  __syncthreads();
  if constexpr (S::NP == 3) {
    dif_mid<S, 1, NT, true>(sm, pa.twi + S::TW2_OFF);
    __syncthreads();
  }
  dif_last<S, 1, NT, true>(sm, st2);
  // the last CTA to get here combines the digits of all CTAs
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(pa.done, 1u) == (uint32_t)pa.D - 1u;
  __syncthreads();
  const bool last = s_last;
  __syncthreads();  // s_last is rewritten by the next build this CTA runs
  if (!last) return false;
  __threadfence();
  const LogFinal f{pa.conv, pa.D, pa.b, L,       k,       pa.exp3, pa.ninv,
                   pa.pat,  pa.pat32, pa.aval, pa.ahat, pa.rowtab};
  lg_final_block<L, NT>(f);
  if (threadIdx.x == 0) *pa.done = 0u;
  return true;
}

template <class S, int NT>
__global__ void __launch_bounds__(NT) k_plan_fused(PlanArgs pa) {
  dbg_enter(pa.status);
  plan_body<S, NT>(pa, blockIdx.x);
}

// ---------------------------------------------------------------------------
// One level of the product tree for A(x) = prod (x - x_i) (step 1 of
// Sec. II.B, divide and conquer with FNT products, "M(n) = 3 FNTs"):
// child nodes of degree <= d are multiplied in pairs with a cyclic product of
// length L = 2d.  Level matrices are [d+1][nodes] (column = node).  Both
// children full (degree d) means the product has degree 2d = L: its leading
// 1 wraps onto coefficient 0 and is moved back.
// ---------------------------------------------------------------------------
template <class S, int WT, int NT>
__global__ void __launch_bounds__(NT) k_poly_level(KArgs a) {
  dbg_enter(a.status);
  static_assert(S::NP >= 2, "");
  using Y = Lay<S, WT>;
  extern __shared__ uint4 smem_raw[];
  uint32_t* X = reinterpret_cast<uint32_t*>(smem_raw);
  uint32_t* Yb = X + Y::WORDS;
  const uint32_t* lvl = static_cast<const uint32_t*>(a.in);
  const size_t ldl = a.ld_in;  // = nodes
  const int d = a.deg_child, nodes = a.nodes, k = a.k;
  const int p0 = blockIdx.x * WT;
  struct LoadChild {
    const uint32_t* lvl;
    size_t ld;
    int d, nodes, p0, side;
    __device__ uint32_t operator()(int i, int c) const {
      const int node = 2 * (p0 + c) + side;
      if (node >= nodes) return (side == 1 && i == 0 && 2 * (p0 + c) < nodes) ? 1u : 0u;
      return i <= d ? lvl[(size_t)i * ld + node] : 0u;
    }
  };
  NopStore nop;
  const uint32_t* twf = a.twf;
  const uint32_t* twi = a.twi;
  LoadChild la{lvl, ldl, d, nodes, p0, 0}, lb{lvl, ldl, d, nodes, p0, 1};
  dif_first<S, WT, NT, false>(X, twf, la, nop);
  dif_first<S, WT, NT, false>(Yb, twf, lb, nop);
  __syncthreads();
  if constexpr (S::NP == 3) {
    dif_mid<S, WT, NT, false>(X, twf + S::TW2_OFF);
    dif_mid<S, WT, NT, false>(Yb, twf + S::TW2_OFF);
    __syncthreads();
  }
  dif_last_inplace<S, WT, NT, false>(X);
  dif_last_inplace<S, WT, NT, false>(Yb);
  __syncthreads();
  dit_last_inplace<S, WT, NT, true, true>(X, Yb);
  __syncthreads();
  if constexpr (S::NP == 3) {
    dit_mid<S, WT, NT, true>(X, twi + S::TW2_OFF);
    __syncthreads();
  }
  struct StoreProd {
    uint32_t* out;
    size_t ld;
    int d, k, p0, npairs;
    uint32_t linv;
    __device__ void operator()(int i, int c, uint32_t v) const {
      const int p = p0 + c;
      if (p >= npairs) return;
      // product degree == 2d only if both children are full
      const bool full = (long long)k >= (long long)(2 * p + 2) * d;
      uint32_t r = m_to_p(m_mul(v, linv));
      if (i == 0 && full) r = r == 0u ? 65536u : r - 1u;
      out[(size_t)i * ld + p] = r;
      if (i == 0) out[(size_t)(2 * d) * ld + p] = full ? 1u : 0u;
    }
  };
  const int npairs = (nodes + 1) / 2;
  StoreProd sp{static_cast<uint32_t*>(a.out), (size_t)npairs, d, k, p0, npairs, a.scale};
  dit_first<S, WT, NT, true>(X, twi, sp);
}

}  // namespace fntrs
