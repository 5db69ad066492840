// Systematic code and punctured lengths.
//
// Systematic code (the paper's "Toward a systematic code" section): the k
// source values are interpolated at the first k points r^0..r^(k-1), giving k
// intermediate symbols (the coefficients of a polynomial i(x) of degree < k,
// elements of F_p, 65536 included); the codeword is i(r^j), j < n, so its
// first k symbols are the source.  Decoding interpolates the first k
// received points (steps 1-6 of Sec. II.B, coefficients kept in F_p) and
// evaluates at r^0..r^(k-1) with the same forward transform.  When the first
// k received positions are exactly 0..k-1 the source is read off directly.
//
// Puncturing (Sec. II.B, n not a power of two): the code of length n_out < n
// keeps the first n_out positions of the length-n code.
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

// dst[r][c] = src[r][c] for r < rows, c < W
__global__ void k_u16_to_u32(const uint16_t* __restrict__ src, size_t ld_src,
                             uint32_t* __restrict__ dst, size_t ld_dst, int rows, int W) {
  const size_t total = (size_t)rows * W;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / W, c = t % W;
    dst[r * ld_dst + c] = src[r * ld_src + c];
  }
}

// 16-bit symbols from values in [0, p): 65536 has none, becomes 0 and raises
// the range flag (as every decode does)
__global__ void k_u32_to_u16(const uint32_t* __restrict__ src, size_t ld_src,
                             uint16_t* __restrict__ dst, size_t ld_dst, int rows, int W,
                             int* status) {
  const size_t total = (size_t)rows * W;
  bool bad = false;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / W, c = t % W;
    const uint32_t v = src[r * ld_src + c];
    bad |= v > 65535u;
    dst[r * ld_dst + c] = (uint16_t)(v > 65535u ? 0u : v);
  }
  if (bad) atomicOr(status, ST_RANGE);
}

unsigned blocks_for(size_t total) {
  return (unsigned)std::max<size_t>(1, std::min<size_t>((total + 255) / 256, 4096));
}

// Pattern tables of positions 0..k-1, built once per plan.
int sys_pattern(fnt_rs_plan_s* p, cudaStream_t st) {
  if (p->sys_ready) return FNT_RS_OK;
  int rc = alloc_pattern_tables(p->sys, p->n, false);
  if (rc) return rc;
  std::vector<uint32_t> pos(p->k);
  for (uint32_t i = 0; i < p->k; ++i) pos[i] = i;
  if ((rc = cuda_ok(cudaMemcpyAsync(p->sys.pos_d, pos.data(), pos.size() * 4,
                                    cudaMemcpyHostToDevice, st))))
    return rc;
  if ((rc = p->plan_tree ? build_pattern(p, p->sys, st) : build_pattern_log(p, p->sys, st)))
    return rc;
  if ((rc = cuda_ok(cudaStreamSynchronize(st)))) return rc;  // pos is a host vector
  p->sys_ready = true;
  return FNT_RS_OK;
}

struct SysWs {
  uint32_t* Z;  // [n][W] coefficients, rows >= k zero
  uint32_t* T;  // [n][W] values at r^j
  void* rest;   // decode / transform workspace
};

SysWs sys_split(const fnt_rs_plan_s* p, size_t W, void* ws) {
  const size_t zb = align256((size_t)p->n * W * 4);
  uint8_t* b = static_cast<uint8_t*>(ws);
  return SysWs{reinterpret_cast<uint32_t*>(b), reinterpret_cast<uint32_t*>(b + zb), b + 2 * zb};
}

bool aligned_to(const void* ptr, size_t a) { return reinterpret_cast<uintptr_t>(ptr) % a == 0; }

}  // namespace

size_t sys_workspace_bytes(const fnt_rs_plan_s* p, size_t W) {
  if (W == 0) return 0;
  return std::max(2 * align256((size_t)p->n * W * 4) +
                      std::max(dec_ws_max(p, W), fnt_columns_work_bytes(p, W)),
                  direct_ws_bytes(p, W));
}

}  // namespace fntrs

using namespace fntrs;

extern "C" {

int fnt_rs_plan_set_length(fnt_rs_plan p, uint32_t n_out) {
  if (!p || n_out < p->k || n_out > p->n) return FNT_RS_E_ARG;
  p->n_out = n_out;
  return FNT_RS_OK;
}

int fnt_rs_encode_sys(fnt_rs_plan p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                      size_t ld_enc, size_t W, void* workspace, void* stream) {
  if (!p || W == 0) return W == 0 && p ? FNT_RS_OK : FNT_RS_E_ARG;
  if (!src || !enc || ld_src < W || ld_enc < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned_to(src, 2) || !aligned_to(enc, 4)) return FNT_RS_E_ARG;
  if (p->u != 1) return FNT_RS_E_ROOT;  // positions 0..k-1 are those of the default root
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p->sched_sys_enc == FNT_RS_SCHED_DIRECT)
    return direct_encode_sys(p, src, ld_src, enc, ld_enc, W, workspace, st);
  if (!workspace) return FNT_RS_E_WORKSPACE;
  const size_t n = p->n, k = p->k;
  const SysWs w = sys_split(p, W, workspace);
  int rc = sys_pattern(p, st);
  if (rc) return rc;
  // the source as received values at positions 0..k-1 (row z = position z), zeros below
  if (n > k && (rc = cuda_ok(cudaMemsetAsync(w.Z + k * W, 0, (n - k) * W * 4, st)))) return rc;
  k_u16_to_u32<<<blocks_for(k * W), 256, 0, st>>>(src, ld_src, w.Z, W, (int)k, (int)W);
  count_launch();
  // intermediate symbols, in place: each tile reads its rows before writing them
  if ((rc = do_decode_tables(p, p->sys, w.Z, W, nullptr, W, W, w.rest, st, 1, w.Z))) return rc;
  // their values at r^j
  if (p->n_out == p->n) return fnt_columns(p, w.Z, W, enc, ld_enc, W, false, w.rest, st);
  if ((rc = fnt_columns(p, w.Z, W, w.T, W, W, false, w.rest, st))) return rc;
  return cuda_ok(cudaMemcpy2DAsync(enc, ld_enc * 4, w.T, W * 4, W * 4, p->n_out,
                                   cudaMemcpyDeviceToDevice, st));
}

int fnt_rs_decode_sys(fnt_rs_plan p, const uint32_t* recv, size_t ld_recv,
                      const uint32_t* positions, uint32_t npos, uint16_t* out, size_t ld_out,
                      size_t W, void* workspace, void* stream) {
  if (!p) return FNT_RS_E_ARG;
  if ((W && (!recv || !out)) || ld_recv < W || ld_out < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned_to(recv, 4) || !aligned_to(out, 2)) return FNT_RS_E_ARG;
  if (p->u != 1) return FNT_RS_E_ROOT;
  int rc = validate_positions(p, positions, npos);
  if (rc) return rc;
  if (W == 0) return FNT_RS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = p->n, k = p->k;
  bool direct = true;  // the first k received positions are the source positions, in order
  for (uint32_t i = 0; i < p->k && direct; ++i) direct = positions[i] == i;
  if (direct) {
    k_u32_to_u16<<<blocks_for(k * W), 256, 0, st>>>(recv, ld_recv, out, ld_out, (int)k, (int)W,
                                                    p->status);
    count_launch();
    return cuda_ok(cudaGetLastError());
  }
  if (p->sched_sys_dec == FNT_RS_SCHED_DIRECT)
    return direct_decode_sys(p, recv, ld_recv, positions, out, ld_out, W, workspace, st);
  if (!workspace) return FNT_RS_E_WORKSPACE;
  const SysWs w = sys_split(p, W, workspace);
  if (n > k && (rc = cuda_ok(cudaMemsetAsync(w.Z + k * W, 0, (n - k) * W * 4, st)))) return rc;
  if ((rc = prepare_pattern(p, positions, npos, st))) return rc;
  if ((rc = do_decode_tables(p, p->slots[p->current], recv, ld_recv, nullptr, W, W, w.rest, st,
                             0, w.Z)))
    return rc;
  if ((rc = fnt_columns(p, w.Z, W, w.T, W, W, false, w.rest, st))) return rc;
  k_u32_to_u16<<<blocks_for(k * W), 256, 0, st>>>(w.T, W, out, ld_out, (int)k, (int)W,
                                                  p->status);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

}  // extern "C"
