// Host-buffer entry points: encode and decode with the data in host memory.
//
// The batch is cut into column chunks (codewords are independent, Sec. II.B)
// that flow through three streams: the host-to-device copy of chunk c+1, the
// kernels of chunk c and the device-to-host copy of chunk c-1 run at the same
// time, so the transfer over the host link (the slowest stage) is no longer
// followed by the kernels and then by the other transfer.  Chunks are at least
// 512 codewords wide so that each chunk's kernels still fill most of the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "../../include/fnt_rs.h"
#include "internal.h"

namespace fntrs {

int pipe_init(HostPipe& h) {
  if (cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h.out_done, cudaEventDisableTiming) != cudaSuccess)
    return FNT_RS_E_CUDA;
  for (int c = 0; c < kPipeChunks; ++c)
    if (cudaEventCreateWithFlags(&h.in_done[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h.comp_done[c], cudaEventDisableTiming) != cudaSuccess)
      return FNT_RS_E_CUDA;
  return FNT_RS_OK;
}

void pipe_free(HostPipe& h) {
  for (int c = 0; c < kPipeChunks; ++c) {
    if (h.in_done[c]) cudaEventDestroy(h.in_done[c]);
    if (h.comp_done[c]) cudaEventDestroy(h.comp_done[c]);
  }
  if (h.start) cudaEventDestroy(h.start);
  if (h.out_done) cudaEventDestroy(h.out_done);
  if (h.in) cudaStreamDestroy(h.in);
  if (h.out) cudaStreamDestroy(h.out);
  h = HostPipe{};
}

namespace {

constexpr size_t kChunkMin = 512;  // codewords per chunk, at least
constexpr int kChunksMax = 4;
constexpr uint32_t kEscPrefix = 4096;  // escapes read back with the encoded symbols

struct Chunking {
  int n;
  size_t w;
};

// FNTRS_HOST_CHUNKS (1..8) overrides the chunk count cap (for measurements)
int chunks_max() {
  static const int v = [] {
    const char* e = std::getenv("FNTRS_HOST_CHUNKS");
    const int x = e ? std::atoi(e) : 0;
    return x >= 1 && x <= kPipeChunks ? x : kChunksMax;
  }();
  return v;
}

Chunking chunking(size_t W) {
  const int want = (int)std::min<size_t>((size_t)chunks_max(),
                                         std::max<size_t>(1, W / (chunks_max() > kChunksMax
                                                                      ? kChunkMin / 2
                                                                      : kChunkMin)));
  size_t w = (W + want - 1) / want;
  w = (w + 63) / 64 * 64;  // chunk starts stay 128-byte aligned
  return Chunking{(int)((W + w - 1) / w), w};
}

// Runs pre(st) once, then in(c0, w, s_in), comp(c0, w, st), out(c0, w, s_out)
// for every chunk, each stage after the previous one of its chunk and the
// copies after the work queued on st before the call (not after pre, so the
// first copy overlaps it); st waits for everything and is synchronised.
template <class Pre, class In, class Comp, class Out>
int run_chunks(fnt_rs_plan_s* p, cudaStream_t st, size_t W, Pre pre, In in, Comp comp, Out out,
               Chunking ch) {
  HostPipe& h = p->pipe;
  int rc = cuda_ok(cudaEventRecord(h.start, st));
  if (!rc) rc = cuda_ok(cudaStreamWaitEvent(h.in, h.start, 0));
  if (!rc) rc = cuda_ok(cudaStreamWaitEvent(h.out, h.start, 0));
  if (!rc) rc = pre(st);
  for (int c = 0; c < ch.n && !rc; ++c) {
    const size_t c0 = (size_t)c * ch.w, w = std::min(ch.w, W - c0);
    if ((rc = in(c0, w, h.in))) break;
    if ((rc = cuda_ok(cudaEventRecord(h.in_done[c], h.in)))) break;
    if ((rc = cuda_ok(cudaStreamWaitEvent(st, h.in_done[c], 0)))) break;
    if ((rc = comp(c0, w, st))) break;
    if ((rc = cuda_ok(cudaEventRecord(h.comp_done[c], st)))) break;
    if ((rc = cuda_ok(cudaStreamWaitEvent(h.out, h.comp_done[c], 0)))) break;
    rc = out(c0, w, h.out);
  }
  // join the copy streams whatever happened, so that nothing is left in flight
  int jr = cuda_ok(cudaEventRecord(h.out_done, h.out));
  if (!jr) jr = cuda_ok(cudaStreamWaitEvent(st, h.out_done, 0));
  if (jr) {
    cudaStreamSynchronize(h.in);
    cudaStreamSynchronize(h.out);
  }
  const int sr = cuda_ok(cudaStreamSynchronize(st));
  return rc ? rc : (jr ? jr : sr);
}

// 2-D copy of columns [c0, c0 + w) of a [rows][W] matrix of `es`-byte elements
int copy_cols(void* dst, const void* src, size_t rows, size_t W, size_t c0, size_t w, size_t es,
              cudaMemcpyKind kind, cudaStream_t s) {
  if (rows == 0) return FNT_RS_OK;
  return cuda_ok(cudaMemcpy2DAsync(static_cast<char*>(dst) + c0 * es, W * es,
                                   static_cast<const char*>(src) + c0 * es, W * es, w * es, rows,
                                   kind, s));
}

struct Carve {
  uint8_t* b;
  template <class T>
  T* take(size_t bytes) {
    T* r = reinterpret_cast<T*>(b);
    b += align256(bytes);
    return r;
  }
};

}  // namespace

size_t host_workspace_bytes(fnt_rs_plan_s* p, size_t W, int op) {
  const size_t k = p->k, n_out = p->n_out;
  switch (op) {
    case FNT_RS_OP_ENCODE_HOST:
      return align256(k * W * 2) + align256(n_out * W * 4) +
             fnt_rs_workspace_bytes(p, W, FNT_RS_OP_ENCODE);
    case FNT_RS_OP_DECODE_HOST:
      return align256(k * W * 4) + align256(k * W * 2) + dec_ws_max(p, W);
    case FNT_RS_OP_ENCODE_WIRE_HOST:
      return align256(k * W * 2) + align256(n_out * W * 2) +
             align256(fnt_rs_wire_escape_cap(p, W) * 8) + 256 + ws_bytes(p, W, enc_nbuf_max(p));
    case FNT_RS_OP_DECODE_WIRE_HOST:
      return align256(k * W * 2) + align256((size_t)kEscStage * 8) + align256(k * W * 2) +
             align256(k * W * 4) + dec_ws_max(p, W);
    default: return 0;
  }
}

}  // namespace fntrs

using namespace fntrs;

extern "C" {

int fnt_rs_encode_host(fnt_rs_plan p, const uint16_t* h_src, uint32_t* h_enc, size_t W,
                       void* workspace, void* stream) {
  if (!p || !h_src || !h_enc || !workspace) return FNT_RS_E_ARG;
  if (W == 0) return FNT_RS_OK;
  if (W > (1u << 30)) return FNT_RS_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Carve cv{static_cast<uint8_t*>(workspace)};
  uint16_t* d_src = cv.take<uint16_t>((size_t)p->k * W * 2);
  uint32_t* d_enc = cv.take<uint32_t>((size_t)p->n_out * W * 4);
  void* rest = cv.b;
  return run_chunks(
      p, st, W, [](cudaStream_t) { return 0; },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return copy_cols(d_src, h_src, p->k, W, c0, w, 2, cudaMemcpyHostToDevice, s);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return fnt_rs_encode(p, d_src + c0, W, d_enc + c0, W, w, rest, s);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return copy_cols(h_enc, d_enc, p->n_out, W, c0, w, 4, cudaMemcpyDeviceToHost, s);
      },
      chunking(W));
}

int fnt_rs_decode_host(fnt_rs_plan p, const uint32_t* h_recv, const uint32_t* positions,
                       uint32_t npos, uint16_t* h_out, size_t W, void* workspace, void* stream) {
  if (!p || !h_recv || !h_out || !workspace) return FNT_RS_E_ARG;
  if (W > (1u << 30)) return FNT_RS_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (W == 0) return prepare_pattern(p, positions, npos, st);
  int rc = validate_positions(p, positions, npos);
  if (rc) return rc;
  Carve cv{static_cast<uint8_t*>(workspace)};
  uint32_t* d_recv = cv.take<uint32_t>((size_t)p->k * W * 4);
  uint16_t* d_out = cv.take<uint16_t>((size_t)p->k * W * 2);
  void* rest = cv.b;
  return run_chunks(
      p, st, W, [&](cudaStream_t s) { return prepare_pattern(p, positions, npos, s); },
      [&](size_t c0, size_t w, cudaStream_t s) {
        // only the first k received rows enter the decode
        return copy_cols(d_recv, h_recv, p->k, W, c0, w, 4, cudaMemcpyHostToDevice, s);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return do_decode_tables(p, p->slots[p->current], d_recv + c0, W, d_out + c0, W, w, rest,
                                s, 0);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return copy_cols(h_out, d_out, p->k, W, c0, w, 2, cudaMemcpyDeviceToHost, s);
      },
      chunking(W));
}

int fnt_rs_encode_wire_host(fnt_rs_plan p, const uint16_t* h_src, uint16_t* h_enc, size_t W,
                            fnt_rs_escape* h_esc, uint32_t esc_cap, uint32_t* nesc,
                            void* workspace, void* stream) {
  if (!p || !h_src || !h_enc || !nesc || (esc_cap && !h_esc) || !workspace) return FNT_RS_E_ARG;
  *nesc = 0;
  if (W == 0) return FNT_RS_OK;
  if (W > (1u << 30)) return FNT_RS_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t cap = fnt_rs_wire_escape_cap(p, W);
  Carve cv{static_cast<uint8_t*>(workspace)};
  uint16_t* d_src = cv.take<uint16_t>((size_t)p->k * W * 2);
  uint16_t* d_enc = cv.take<uint16_t>((size_t)p->n_out * W * 2);
  uint2* d_esc = cv.take<uint2>(cap * 8);
  uint32_t* d_count = cv.take<uint32_t>(4);
  void* rest = cv.b;
  uint32_t count_h[1] = {0};
  std::vector<fnt_rs_escape> pre_h(kEscPrefix);
  int rc = run_chunks(
      p, st, W, [&](cudaStream_t s) { return cuda_ok(cudaMemsetAsync(d_count, 0, 4, s)); },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return copy_cols(d_src, h_src, p->k, W, c0, w, 2, cudaMemcpyHostToDevice, s);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        const WireSpec ws{d_enc + c0, W, d_esc, d_count,
                          (uint32_t)std::min<size_t>(cap, 0xFFFFFFFFu), p->n_out, (uint32_t)c0};
        return do_encode(p, d_src + c0, W, nullptr, W, w, rest, s, &ws);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        int r = copy_cols(h_enc, d_enc, p->n_out, W, c0, w, 2, cudaMemcpyDeviceToHost, s);
        if (!r && c0 + w == W) {  // after the last chunk's kernels
          r = cuda_ok(cudaMemcpyAsync(count_h, d_count, 4, cudaMemcpyDeviceToHost, s));
          if (!r)
            r = cuda_ok(cudaMemcpyAsync(pre_h.data(), d_esc,
                                        std::min<size_t>(kEscPrefix, cap) * 8,
                                        cudaMemcpyDeviceToHost, s));
        }
        return r;
      },
      chunking(W));
  if (rc) return rc;
  // the count and the first kEscPrefix escapes come back with the symbols'
  // last copy (one synchronisation); the rest, if any, after the count is known
  *nesc = count_h[0];
  const uint32_t count = count_h[0];
  if (count > cap) return FNT_RS_E_WORKSPACE;  // more escapes than the staging holds
  if (count > esc_cap) return FNT_RS_E_ARG;    // the caller's array is too short
  if (count == 0) return FNT_RS_OK;
  std::vector<fnt_rs_escape> e(count);
  std::copy(pre_h.begin(), pre_h.begin() + std::min(count, kEscPrefix), e.begin());
  if (count > kEscPrefix) {
    if ((rc = cuda_ok(cudaMemcpyAsync(e.data() + kEscPrefix, d_esc + kEscPrefix,
                                      (size_t)(count - kEscPrefix) * 8, cudaMemcpyDeviceToHost,
                                      st))))
      return rc;
    if ((rc = cuda_ok(cudaStreamSynchronize(st)))) return rc;
  }
  std::sort(e.begin(), e.end(), [](const fnt_rs_escape& a, const fnt_rs_escape& b) {
    return a.row != b.row ? a.row < b.row : a.col < b.col;
  });
  std::copy(e.begin(), e.end(), h_esc);
  return FNT_RS_OK;
}

int fnt_rs_decode_wire_host(fnt_rs_plan p, const uint16_t* h_recv, const uint32_t* positions,
                            uint32_t npos, const fnt_rs_escape* h_esc, uint32_t nesc,
                            uint16_t* h_out, size_t W, void* workspace, void* stream) {
  if (!p || !h_recv || !h_out || (nesc && !h_esc) || !workspace) return FNT_RS_E_ARG;
  if (W > (1u << 30)) return FNT_RS_E_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (W == 0) return prepare_pattern(p, positions, npos, st);
  int rc = validate_positions(p, positions, npos);
  if (rc) return rc;
  Carve cv{static_cast<uint8_t*>(workspace)};
  uint16_t* d_recv = cv.take<uint16_t>((size_t)p->k * W * 2);
  uint2* d_esc = cv.take<uint2>((size_t)kEscStage * 8);
  uint16_t* d_out = cv.take<uint16_t>((size_t)p->k * W * 2);
  uint32_t* copy = cv.take<uint32_t>((size_t)p->k * W * 4);
  void* rest = cv.b;
  const auto* esc = reinterpret_cast<const uint2*>(h_esc);
  // escapes: staged once when they fit, else in batches inside a single chunk
  const bool staged = nesc <= kEscStage;
  return run_chunks(
      p, st, W,
      [&](cudaStream_t s) {
        int r = prepare_pattern(p, positions, npos, s);
        if (!r && staged && nesc)
          r = cuda_ok(cudaMemcpyAsync(d_esc, esc, (size_t)nesc * 8, cudaMemcpyHostToDevice, s));
        return r;
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        // only the first k received rows enter the decode
        return copy_cols(d_recv, h_recv, p->k, W, c0, w, 2, cudaMemcpyHostToDevice, s);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        int r = wire_widen(p, d_recv + c0, W, copy + c0, W, w, s);
        if (r) return r;
        if (staged) {
          r = wire_escapes(p, d_esc, nesc, npos, copy, W, W, c0, c0 + w, s);
        } else {
          for (uint32_t i0 = 0; i0 < nesc && !r; i0 += kEscStage) {
            const uint32_t m = std::min(kEscStage, nesc - i0);
            r = cuda_ok(cudaMemcpyAsync(d_esc, esc + i0, (size_t)m * 8, cudaMemcpyHostToDevice,
                                        s));
            if (!r) r = wire_escapes(p, d_esc, m, npos, copy, W, W, c0, c0 + w, s);
          }
        }
        if (r) return r;
        return do_decode_tables(p, p->slots[p->current], copy + c0, W, d_out + c0, W, w, rest,
                                s, 0);
      },
      [&](size_t c0, size_t w, cudaStream_t s) {
        return copy_cols(h_out, d_out, p->k, W, c0, w, 2, cudaMemcpyDeviceToHost, s);
      },
      staged ? chunking(W) : Chunking{1, W});
}

}  // extern "C"
