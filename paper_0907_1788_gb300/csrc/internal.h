// Internal declarations shared by the host modules of libfntrs (plans,
// ragged batches, the serving loop).  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/fnt_rs.h"

namespace fntrs {

// Device tables per transform length L: per-pass schedule tables and the
// powers r_L^e, r_L^-e (default root).
struct Tables {
  uint32_t* twf = nullptr;
  uint32_t* twi = nullptr;
  uint32_t* twf_sw = nullptr;  // pass-1 part of twf, 16-byte chunks of row i2 rotated (decode_tw_sw)
  uint32_t* powf = nullptr;
  uint32_t* powi = nullptr;
};

// Per-pattern device tables (steps 1-3 of the interpolation, Sec. II.B).
struct PatternSlot {
  std::vector<uint32_t> key;
  uint64_t last_use = 0;
  bool valid = false;
  uint2* pat = nullptr;
  uint32_t* ahat = nullptr;
  uint32_t* ahat2 = nullptr;
  uint32_t* pat32 = nullptr;  // (row << 17) | weight per position
  uint32_t* rowtab = nullptr;  // (position << 17) | weight per received row (first k rows)
  uint32_t* pos_d = nullptr;  // first k positions (device)
  uint32_t* pos_h = nullptr;  // pinned staging of the upload
  const uint32_t* pos_map = nullptr;  // pos_h as seen from the device (mapped pinned memory)
  cudaEvent_t staged = nullptr;  // recorded once the device has read pos_h
  uint32_t* done = nullptr;   // completion counter of the one-launch build (zero at rest)
};

// Device tables of one erasure pattern for length n (and, with `staging`, the
// pinned upload buffer and its event); release with free_pattern_tables.
int alloc_pattern_tables(PatternSlot& sl, size_t n, bool staging);
void free_pattern_tables(PatternSlot& sl);

// Streams and events of the host-buffer entry points, which overlap the
// host-to-device copies, the kernels and the device-to-host copies of
// successive column chunks (hostpipe.cu).
constexpr int kPipeChunks = 8;
struct HostPipe {
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, out_done = nullptr;
  cudaEvent_t in_done[kPipeChunks] = {};
  cudaEvent_t comp_done[kPipeChunks] = {};
};
int pipe_init(HostPipe& h);
void pipe_free(HostPipe& h);

constexpr int kPatternSlots = 4;
struct PaperState;   // paper_route.cu
struct DirectState;  // direct.cu
constexpr size_t kChunkBudget = 96ull << 20;  // bytes of split-transform workspace per chunk

}  // namespace fntrs

struct fnt_rs_plan_s {
  int dev = 0;
  uint32_t n = 0, k = 0, root = 0;
  uint32_t u = 1, uinv = 1;  // root = default^u; spectrum index j -> row uinv*j
  uint32_t ninv = 1;
  bool split = false;  // n > tile limit: n = C * kLocalL
  int C = 1;
  bool blocked = false;  // k > n/2
  fntrs::Tables tn;             // tables of length n (pow tables; schedule tables if n <= tile)
  fntrs::Tables tl;             // tables of the local length (n > 8192)
  int C_local = 1;              // n / kLocalL (n > 8192)
  fntrs::Tables tenc;           // schedule tables of the TMA encode's tile length
  uint32_t* twc = nullptr;  // TMA encode, class 1 of n = 2L: pass-1 twiddles times r_n^i2
  // log-domain pattern build: digits of g[d] = log_3(1 - r^d), b bits each
  bool plan_tree = false;   // use the product tree instead
  int lg_b = 4, lg_D = 4;
  uint32_t* ghat = nullptr;  // [n][D] transforms of the reversed digit vectors
  uint32_t* exp3 = nullptr;  // shared table
  int enc_L = 0, enc_C = 0;  // TMA encode shape (0: not applicable)
  bool enc_fold = false;     // n = 8192, k > 4096: the classes fold two source rows
  bool no_tma = false;
  int sched_enc = 0, sched_dec = 0;  // fnt_rs_sched of encode / decode (0: automatic)
  int sms = 1;
  int* status = nullptr;
  uint32_t* pscratch = nullptr;
  size_t pscratch_words = 0;
  fntrs::PatternSlot slots[fntrs::kPatternSlots];
  int current = -1;
  uint64_t clock = 0;
  uint32_t n_out = 0;         // code length after puncturing (k <= n_out <= n)
  fntrs::PatternSlot sys;     // pattern of positions 0..k-1 (systematic code), built on first use
  bool sys_ready = false;
  fntrs::HostPipe pipe;       // host-buffer entry points
  fntrs::PaperState* paper = nullptr;  // decode schedule FNT_RS_SCHED_PAPER, once selected
  fntrs::DirectState* direct = nullptr;  // FNT_RS_SCHED_DIRECT of the systematic ops
  int sched_sys_enc = 0, sched_sys_dec = 0;  // 0 (FNT route) or FNT_RS_SCHED_DIRECT
};

namespace fntrs {

int cuda_ok(cudaError_t e);
size_t split_chunk(uint32_t n, int nbuf);
// workspace buffers of the schedule in use / the most any candidate schedule needs
int enc_nbuf(const fnt_rs_plan_s* p);
int dec_nbuf(const fnt_rs_plan_s* p);
int enc_nbuf_max(const fnt_rs_plan_s* p);
int dec_nbuf_max(const fnt_rs_plan_s* p);
// schedules (fnt_rs_sched) an op can run with, and the one it runs with now
bool sched_available(const fnt_rs_plan_s* p, int op, int sched);
int sched_effective(const fnt_rs_plan_s* p, int op);
int fnt_nbuf(const fnt_rs_plan_s* p);
size_t ws_bytes(const fnt_rs_plan_s* p, size_t W, int nbuf);
inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// workspace of the systematic encode / decode (systematic.cu)
size_t sys_workspace_bytes(const fnt_rs_plan_s* p, size_t W);
// workspace of the 16-bit wire-format device calls (wire.cu) and of the
// host-buffer calls (hostpipe.cu)
size_t wire_workspace_bytes(const fnt_rs_plan_s* p, size_t W, int op);
size_t host_workspace_bytes(fnt_rs_plan_s* p, size_t W, int op);
int get_tables(int L, Tables* out);
uint32_t hinv(uint32_t a);
int validate_positions(const fnt_rs_plan_s* p, const uint32_t* pos, uint32_t npos);
// find or build the pattern of the first k positions (p->current)
int prepare_pattern(fnt_rs_plan_s* p, const uint32_t* positions, uint32_t npos, cudaStream_t st);
// length-n transform of W columns (forward or n^-1-scaled inverse), in column
// chunks through `work` (fnt_columns_work_bytes) when n exceeds the tile limit
int fnt_columns(fnt_rs_plan_s* p, const uint32_t* in, size_t ld_in, uint32_t* out,
                size_t ld_out, size_t W, bool inverse, void* work, cudaStream_t st);
size_t fnt_columns_work_bytes(const fnt_rs_plan_s* p, size_t W);
// build the pattern of the positions already uploaded to sl.pos_d (or, for
// the one-launch build, of the device-readable positions `pos`)
int build_pattern_log(fnt_rs_plan_s* p, PatternSlot& sl, cudaStream_t st,
                      uint32_t* scratch = nullptr, const uint32_t* pos = nullptr);
// the log-domain build of this plan runs as one launch (k_plan_fused)
bool fused_plan_applies(const fnt_rs_plan_s* p);
size_t pattern_scratch_words(uint32_t n, uint32_t k);
int build_pattern(fnt_rs_plan_s* p, PatternSlot& sl, cudaStream_t st);
// 16-bit wire output of an encode (see KArgs::wire): symbols to enc as u16,
// escapes of the value 65536 to esc (count on the device), rows < rows kept.
struct WireSpec {
  uint16_t* enc;
  size_t ld;
  uint2* esc;
  uint32_t* count;
  uint32_t cap;
  uint32_t rows;
  uint32_t col0;  // column of enc[.][0] in the escapes' numbering
};
// Widens rows [0, k) x columns [0, W) of 16-bit received symbols to u32 (dst,
// ld_dst) and writes 65536 at the escapes that fall in columns [c_lo, c_hi)
// of rows < k (escape columns are absolute: dst column = escape column).
int wire_widen(fnt_rs_plan_s* p, const uint16_t* recv, size_t ld_recv, uint32_t* dst,
               size_t ld_dst, size_t W, cudaStream_t st);
int wire_escapes(fnt_rs_plan_s* p, const uint2* esc, uint32_t nesc, uint32_t nrecv,
                 uint32_t* dst, size_t ld_dst, size_t W, size_t c_lo, size_t c_hi,
                 cudaStream_t st);
constexpr uint32_t kEscStage = 65536;  // escapes staged at once by the host decode

// Encode of n > 8192 in two passes (radix-n/4096 cross pass, 4096-point
// local transforms) through `work` of ws_bytes(p, W, enc_nbuf(p)) bytes.
// With `wire` the output goes there instead of enc (which may be null).
int do_encode_two_pass(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                       size_t ld_enc, size_t W, uint32_t* work, cudaStream_t st,
                       const WireSpec* wire = nullptr);
int do_encode(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc, size_t ld_enc,
              size_t W, void* workspace, cudaStream_t st, const WireSpec* wire = nullptr);
// decode with explicit pattern tables (slots != 0: row z of recv is position z);
// with out32 the coefficients go there as u32 (ld_out) and `out` is unused
int do_decode_tables(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv,
                     size_t ld_recv, uint16_t* out, size_t ld_out, size_t W, void* workspace,
                     cudaStream_t st, int slots, uint32_t* out32 = nullptr);
// decode workspace: of the schedule in use / of every schedule the plan can run
size_t dec_ws_now(const fnt_rs_plan_s* p, size_t W);
size_t dec_ws_max(const fnt_rs_plan_s* p, size_t W);

// The paper's decode route (paper_route.cu): chirp step 3 and middle-product
// step 5 at length 2n, step 6 by FNT_2n.
bool paper_available(const fnt_rs_plan_s* p);
int paper_enable(fnt_rs_plan_s* p, cudaStream_t st);
void paper_free(fnt_rs_plan_s* p);
size_t paper_ws_bytes(const fnt_rs_plan_s* p, size_t W);
int paper_decode(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv, size_t ld_recv,
                 uint16_t* out, size_t ld_out, size_t W, void* workspace, cudaStream_t st,
                 int slots, uint32_t* out32);

// The direct (quadratic) systematic encoder and decoder (direct.cu).
bool direct_available(const fnt_rs_plan_s* p);
int direct_enable(fnt_rs_plan_s* p, int op);  // op: FNT_RS_OP_ENCODE / _DECODE / _ENCODE_SYS / _DECODE_SYS
bool direct_ready(const fnt_rs_plan_s* p, int op);
void direct_free(fnt_rs_plan_s* p);
int direct_encode(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                  size_t ld_enc, size_t W, void* workspace, cudaStream_t st);
int direct_decode(fnt_rs_plan_s* p, const PatternSlot& sl, const uint32_t* recv, size_t ld_recv,
                  uint16_t* out, size_t ld_out, size_t W, void* workspace, cudaStream_t st,
                  int slots, uint32_t* out32);
size_t direct_ws_bytes(const fnt_rs_plan_s* p, size_t W);
int direct_encode_sys(fnt_rs_plan_s* p, const uint16_t* src, size_t ld_src, uint32_t* enc,
                      size_t ld_enc, size_t W, void* workspace, cudaStream_t st);
int direct_decode_sys(fnt_rs_plan_s* p, const uint32_t* recv, size_t ld_recv,
                      const uint32_t* positions, uint16_t* out, size_t ld_out, size_t W,
                      void* workspace, cudaStream_t st);

}  // namespace fntrs
