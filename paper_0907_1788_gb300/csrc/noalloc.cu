// Encode for long codes (n > 8192) that allocates nothing at call time.
//
// Codes longer than one CTA's tile are encoded in two passes that meet in a
// scratch matrix of n * W words, and a punctured code is first encoded at full
// length into a buffer of n * W words.  fnt_rs_encode takes that scratch from
// the caller; fnt_rs_encode_noalloc takes it from the fixed device array below,
// which every GPU that loads this library keeps until the process exits.
// Calls share the array: two calls that overlap on the GPU (different
// streams, or graphs replayed concurrently) race on it.  Nothing in it has to
// start at zero: the first pass writes every word the second pass reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/fnt_rs.h"
#include "kargs.h"
#include "sched.h"

namespace fntrs {

constexpr size_t kNoAllocScratchWords = FNT_RS_NOALLOC_SCRATCH_BYTES / 4;

// Device-side scratch.  Host code may not use this name as an address: on
// the host it is only a stand-in symbol, so its device address is looked up
// with cudaGetSymbolAddress (once per device) and passed to the kernels.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchWords];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {};

// Address of the scratch array on the current device; set up on first use.
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FNT_RS_E_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FNT_RS_E_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return FNT_RS_OK;
}

}  // namespace fntrs

extern "C" int fnt_rs_encode_noalloc(fnt_rs_plan plan, const uint16_t* src, size_t ld_src,
                                     uint32_t* enc, size_t ld_enc, size_t W, void* stream) {
  using namespace fntrs;
  if (!plan) return FNT_RS_E_ARG;
  // everything the regular call may use from its workspace: the split scratch
  // and, for a punctured code, the full-length codeword buffer in front of it
  const size_t need = fnt_rs_workspace_bytes(plan, W, FNT_RS_OP_ENCODE);
  if (need == 0)  // short codes use no scratch: the regular entry point allocates nothing
    return fnt_rs_encode(plan, src, ld_src, enc, ld_enc, W, nullptr, stream);
  if (need > FNT_RS_NOALLOC_SCRATCH_BYTES) return FNT_RS_E_WORKSPACE;
  void* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  return fnt_rs_encode(plan, src, ld_src, enc, ld_enc, W, scratch, stream);
}
