// 16-bit wire format of the encoded symbols.
//
// Sec. II.B ("Design of the code on GF(65537)"): every element of F_65537
// but 65536 fits in 16 bits, so a symbol travels as 16 bits and the
// positions where the value 65536 occurs are sent beside the packets (in
// their headers).  Encoding straight into that format halves the bytes an
// encode writes (4 -> 2 per symbol) and the bytes a decode reads.
//
// Encode: the encode kernels' storers write the low 16 bits and append each
// 65536 to an escape array (KArgs::wire).  Decode: the received 16-bit rows
// are widened to u32 in the workspace, the escapes are written back as
// 65536, and the ordinary decode runs on that copy.  The host-buffer
// variants are in hostpipe.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/fnt_rs.h"
#include "internal.h"
#include "kargs.h"

namespace fntrs {

void count_launch();

namespace {

static_assert(sizeof(fnt_rs_escape) == sizeof(uint2), "escape = {row, col} u32 pair");

// dst[r][c] = src[r][c] for r < rows, c < W; eight symbols per thread when
// every row starts on a 16-byte boundary (vec), else one.
__global__ void k_widen16(const uint16_t* __restrict__ src, size_t ld_src,
                          uint32_t* __restrict__ dst, size_t ld_dst, int rows, int W, int vec) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  if (vec) {
    const int W8 = W / 8;
    const size_t total = (size_t)rows * W8;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
      const size_t r = t / W8, c8 = t % W8;
      const uint4 v = __ldcs(reinterpret_cast<const uint4*>(src + r * ld_src) + c8);
      uint4* d = reinterpret_cast<uint4*>(dst + r * ld_dst) + 2 * c8;
      d[0] = make_uint4(v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16);
      d[1] = make_uint4(v.z & 0xFFFFu, v.z >> 16, v.w & 0xFFFFu, v.w >> 16);
    }
  } else {
    const size_t total = (size_t)rows * W;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
      const size_t r = t / W, c = t % W;
      dst[r * ld_dst + c] = src[r * ld_src + c];
    }
  }
}

// Escapes of the received rows: row < rows (rows at or beyond `rows`, which
// the decode never reads, are skipped), column in [c_lo, c_hi).  An escape
// outside [0, nrecv) x [0, W), or one whose 16-bit symbol is not 0, is not
// valid wire data and raises the range flag.
__global__ void k_apply_escapes(const uint2* __restrict__ esc, uint32_t nesc, uint32_t* dst,
                                size_t ld_dst, uint32_t rows, uint32_t nrecv, uint32_t W,
                                uint32_t c_lo, uint32_t c_hi, int* status) {
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nesc; i += gridDim.x * blockDim.x) {
    const uint2 e = esc[i];
    if (e.x >= nrecv || e.y >= W) {
      bad = true;
    } else if (e.x < rows && e.y >= c_lo && e.y < c_hi) {
      uint32_t* v = dst + (size_t)e.x * ld_dst + e.y;
      bad |= *v != 0u;
      *v = 65536u;
    }
  }
  if (bad) atomicOr(status, ST_RANGE);
}

unsigned grid_for(const fnt_rs_plan_s* p, size_t work) {
  const size_t want = (work + 255) / 256;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(want, (size_t)p->sms * 8));
}

bool aligned_to(const void* ptr, size_t a) { return reinterpret_cast<uintptr_t>(ptr) % a == 0; }

size_t dec_copy_bytes(const fnt_rs_plan_s* p, size_t W) { return align256((size_t)p->k * W * 4); }

}  // namespace

int wire_widen(fnt_rs_plan_s* p, const uint16_t* recv, size_t ld_recv, uint32_t* dst,
               size_t ld_dst, size_t W, cudaStream_t st) {
  const bool vec = W % 8 == 0 && ld_recv % 8 == 0 && ld_dst % 4 == 0 && aligned_to(recv, 16) &&
                   aligned_to(dst, 16);
  const size_t work = (size_t)p->k * (vec ? W / 8 : W);
  k_widen16<<<grid_for(p, work), 256, 0, st>>>(recv, ld_recv, dst, ld_dst, (int)p->k, (int)W,
                                               vec ? 1 : 0);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

int wire_escapes(fnt_rs_plan_s* p, const uint2* esc, uint32_t nesc, uint32_t nrecv,
                 uint32_t* dst, size_t ld_dst, size_t W, size_t c_lo, size_t c_hi,
                 cudaStream_t st) {
  if (nesc == 0) return FNT_RS_OK;
  k_apply_escapes<<<grid_for(p, nesc), 256, 0, st>>>(esc, nesc, dst, ld_dst, p->k, nrecv,
                                                    (uint32_t)W, (uint32_t)c_lo, (uint32_t)c_hi,
                                                    p->status);
  count_launch();
  return cuda_ok(cudaGetLastError());
}

size_t wire_workspace_bytes(const fnt_rs_plan_s* p, size_t W, int op) {
  switch (op) {
    case FNT_RS_OP_ENCODE_WIRE: return ws_bytes(p, W, enc_nbuf_max(p));
    case FNT_RS_OP_DECODE_WIRE: return dec_copy_bytes(p, W) + dec_ws_max(p, W);
    default: return 0;
  }
}

}  // namespace fntrs

using namespace fntrs;

extern "C" {

size_t fnt_rs_wire_escape_cap(fnt_rs_plan p, size_t W) {
  if (!p) return 0;
  return (size_t)p->n_out * W / 64 + 1024;
}

int fnt_rs_encode_wire(fnt_rs_plan p, const uint16_t* src, size_t ld_src, uint16_t* enc,
                       size_t ld_enc, size_t W, fnt_rs_escape* esc, uint32_t esc_cap,
                       uint32_t* esc_count, void* workspace, void* stream) {
  if (!p || !esc_count || (esc_cap && !esc)) return FNT_RS_E_ARG;
  if (!aligned_to(esc_count, 4) || !aligned_to(esc, 8)) return FNT_RS_E_ARG;
  if (W && (!src || !enc || ld_src < W || ld_enc < W || W > (1u << 30))) return FNT_RS_E_ARG;
  if (!aligned_to(src, 2) || !aligned_to(enc, 2)) return FNT_RS_E_ARG;
  if (W && ws_bytes(p, W, enc_nbuf(p)) && !workspace) return FNT_RS_E_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = cuda_ok(cudaMemsetAsync(esc_count, 0, 4, st));
  if (rc || W == 0) return rc;
  const WireSpec w{enc, ld_enc, reinterpret_cast<uint2*>(esc), esc_count, esc_cap, p->n_out, 0};
  return do_encode(p, src, ld_src, nullptr, ld_enc, W, workspace, st, &w);
}

int fnt_rs_decode_wire(fnt_rs_plan p, const uint16_t* recv, size_t ld_recv,
                       const uint32_t* positions, uint32_t npos, const fnt_rs_escape* esc,
                       uint32_t nesc, uint16_t* out, size_t ld_out, size_t W, void* workspace,
                       void* stream) {
  if (!p) return FNT_RS_E_ARG;
  if ((W && (!recv || !out)) || ld_recv < W || ld_out < W || W > (1u << 30)) return FNT_RS_E_ARG;
  if (!aligned_to(recv, 2) || !aligned_to(out, 2) || (nesc && !esc) || !aligned_to(esc, 8))
    return FNT_RS_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = prepare_pattern(p, positions, npos, st);
  if (rc || W == 0) return rc;
  if (!workspace) return FNT_RS_E_WORKSPACE;
  uint32_t* copy = static_cast<uint32_t*>(workspace);
  void* rest = static_cast<uint8_t*>(workspace) + dec_copy_bytes(p, W);
  if ((rc = wire_widen(p, recv, ld_recv, copy, W, W, st))) return rc;
  if ((rc = wire_escapes(p, reinterpret_cast<const uint2*>(esc), nesc, npos, copy, W, W, 0, W,
                         st)))
    return rc;
  return do_decode_tables(p, p->slots[p->current], copy, W, out, ld_out, W, rest, st, 0);
}

}  // extern "C"
