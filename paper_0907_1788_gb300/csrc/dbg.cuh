// Debug build: device index checks (compile with -DFNTRS_DEBUG_BOUNDS=1; the
// build script's debug_bounds option puts that library in a folder of its
// own).  Every shared-memory index of the tile engine's passes and every
// global index of the loaders, storers and staged tiles goes through dbg_in;
// a failed check ORs ST_BOUNDS into the status word (the caller's, or the one
// the kernel registered with dbg_enter) and the access is skipped, so the
// kernel neither faults nor traps and the host reads FNT_RS_E_BOUNDS from
// fnt_rs_status.  In the release build dbg_in is the constant true and the
// checks compile away.
#pragma once
#include <stdint.h>

#include "kargs.h"

#ifndef FNTRS_DEBUG_BOUNDS
#define FNTRS_DEBUG_BOUNDS 0
#endif

namespace fntrs {

constexpr bool kDebugBounds = FNTRS_DEBUG_BOUNDS != 0;

#if FNTRS_DEBUG_BOUNDS
// status word of the running work, for checks that have no KArgs at hand
__shared__ int* fntrs_dbg_status;
#endif

// Registers the status word that failed checks report to (all threads call it
// at the same point; it synchronises the CTA in the debug build only).
__device__ __forceinline__ void dbg_enter(int* status) {
#if FNTRS_DEBUG_BOUNDS
  __syncthreads();
  if (threadIdx.x == 0) fntrs_dbg_status = status;
  __syncthreads();
#else
  (void)status;
#endif
}

// 0 <= i < n: true.  Otherwise (debug build only) the fault is recorded and
// false tells the caller to skip the access.
__device__ __forceinline__ bool dbg_in(long long i, long long n, int* status = nullptr) {
#if FNTRS_DEBUG_BOUNDS
  if (i >= 0 && i < n) return true;
  int* s = status ? status : fntrs_dbg_status;
  if (s) atomicOr(s, ST_BOUNDS);
  return false;
#else
  (void)i;
  (void)n;
  (void)status;
  return true;
#endif
}

}  // namespace fntrs
