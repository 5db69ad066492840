// Launch arguments shared by the host dispatcher and the kernel templates.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fntrs {

// Status bits ORed into the plan's device status word (ST_BOUNDS: a device
// index check of the debug build failed, dbg.cuh).
enum : int { ST_RANGE = 1, ST_TIMEOUT = 2, ST_BOUNDS = 4 };

// Output modes of the local (in-tile) pass of a split transform n = C * L.
enum LocalMode : int {
  LM_ENC = 0,        // out u32 rows j1 + C*j, reduced to [0, p)
  LM_FNT = 1,        // out u32 rows j1 + C*j, times `scale`, reduced
  LM_WORK = 2,       // out2 u32 rows j1 + C*j < out_limit, raw Z/M values
  LM_WORK_AHAT = 3,  // out2 u32 rows j1 + C*j: value * ahat[row]
  LM_OUT16 = 4,      // out u16 rows j1 + C*j < out_limit, range-checked
  LM_SPLIT = 5,      // rows < h -> out2[row], h <= row < out_limit -> out3[row - h]
  LM_X_PARTIAL = 6,  // out2[row] = v * ahat[row], out3[row] = v * ahat2[row]
  LM_ACCUM = 7,      // out3[row] += v * ahat[row]
  LM_OUT16_ADD = 8   // out u16 rows < out_limit: v + (row >= h ? in2[row - h] : 0)
};

// Input modes of the cross pass (radix-C stage over stride-L rows).
enum CrossLoad : int {
  CL_SRC16 = 0,  // u16 source rows < row_limit
  CL_RECV = 1,   // gathered received rows through the pattern table
  CL_U32 = 2     // u32 rows < row_limit
};

struct KArgs {
  const void* in = nullptr;
  size_t ld_in = 0;
  void* out = nullptr;
  size_t ld_out = 0;
  const void* in2 = nullptr;
  size_t ld_in2 = 0;
  void* out2 = nullptr;
  void* out3 = nullptr;
  size_t ld_work = 0;  // leading dimension of out2/out3/in2 workspace matrices
  int W = 0;           // columns handled by this launch
  int n = 0, k = 0, L = 0, C = 1, h = 0;
  int row_limit = 0;  // input rows >= row_limit read as zero
  int out_limit = 0;  // output rows >= out_limit not written
  void* out32 = nullptr;  // decode: coefficients as u32 in [0, p) here instead of 16-bit symbols
  uint32_t scale = 1;
  const uint32_t* twf = nullptr;   // per-pass tables of the L-schedule, forward root
  const uint32_t* twi = nullptr;   // same, inverse root
  const uint32_t* twf_sw = nullptr;  // pass-1 part of twf, chunks swizzled per row (or null)
  const uint32_t* powf = nullptr;  // r_n^e, e < n
  const uint32_t* powi = nullptr;  // r_n^-e, e < n
  const uint2* pat = nullptr;      // decode gather table, one {row, weight} per position
  const uint32_t* ahat = nullptr;  // pointwise tables (natural order)
  const uint32_t* ahat2 = nullptr;
  int* status = nullptr;
  int mode = 0;
  // non-default root r' = r^u: forward outputs land on row (row_mul * j) mod n,
  // inverse inputs are read from row (in_row_mul * j) mod n (both = u^-1 mod n)
  uint32_t row_mul = 1;
  uint32_t in_row_mul = 1;
  int slots = 0;      // decode input indexed by position (row z = position z)
  int deg_child = 0;  // product-tree level: degree of the child polynomials
  int nodes = 0;      // product-tree level: number of child nodes
  // 16-bit wire output of an encode (wire != 0): `out` is u16, a symbol is
  // stored as its low 16 bits and every symbol equal to 65536 is appended to
  // esc as {row, col_base + column} (*esc_count counts all of them, entries
  // beyond esc_cap are dropped); rows >= wire_rows are not stored.
  int wire = 0;
  int wire_rows = 0;
  int col_base = 0;
  uint32_t esc_cap = 0;
  uint2* esc = nullptr;
  uint32_t* esc_count = nullptr;
};

// Arguments of the one-launch log-domain pattern build (n <= tile limit).
struct PlanArgs {
  int k = 0, D = 0, b = 0;
  uint32_t ninv = 0;
  const uint32_t* twf = nullptr;   // pass tables of the n-schedule, forward root
  const uint32_t* twi = nullptr;   // same, inverse root
  const uint32_t* pos = nullptr;   // first k received positions
  const uint32_t* ghat = nullptr;  // [n][D] transforms of the log-table digits
  const uint32_t* exp3 = nullptr;  // 3^e, e < 65536
  uint32_t* conv = nullptr;        // [n][D] digit convolutions (scratch)
  uint2* pat = nullptr;            // position table (written)
  uint32_t* pat32 = nullptr;
  uint32_t* rowtab = nullptr;  // per received row, or null
  uint32_t* aval = nullptr;        // A(r^j) (split step-6 product) or null
  uint32_t* ahat = nullptr;        // n^-1 FNT(A mod x^k) or null
  uint32_t* done = nullptr;        // CTA completion counter, zero between builds
  int* status = nullptr;           // the plan's status word (debug-build index checks)
};

}  // namespace fntrs
