// Work list of the ragged persistent kernel (k_ragged): every group with
// 256 <= n <= 8192 contributes encode tiles, pattern digit builds (decode
// groups) and decode tiles; one launch of k_ragged runs them all, each CTA
// taking work items in list order from an atomic counter.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kargs.h"

namespace fntrs {

enum RaggedItemKind : int { RI_ENC = 0, RI_PLAN = 1, RI_DEC = 2 };

struct RaggedItem {
  int kind;   // RaggedItemKind
  int group;  // index into RaggedArgs::groups
  int tile;   // column tile (encode, decode) or digit (pattern build)
};

struct RaggedGroupDev {
  KArgs enc;      // generic encode: C = 1, L = n
  KArgs dec;      // generic decode from the encoded rows (slots mode)
  KArgs tail_inv; // k > n/2: coefficients of A, n^-1 IFNT of the values (one column)
  KArgs tail_fwd; // k > n/2: transforms of the two coefficient halves (two columns)
  PlanArgs plan;  // one-launch pattern build
  uint32_t* halves;  // [n][2] coefficient halves (k > n/2)
  int L;          // n
  int blocked;    // k > n/2: two-buffer decode, tables from the coefficient split
  int enc_tiles;  // encode tiles this group contributes (its decode waits for all of them)
  int enc_need;   // encode tiles a decode item waits for (= enc_tiles; see FNTRS_TEST_STALL_GROUP)
  int has_plan;   // decode group
};

struct RaggedArgs {
  const RaggedItem* items;
  int nitems;
  const RaggedGroupDev* groups;
  unsigned* next;       // work counter (zero before the launch)
  unsigned* enc_done;   // [groups] finished encode tiles (zero before the launch)
  unsigned* plan_done;  // [groups] 1 once the pattern tables are written (zero before)
};

// Tile lengths the ragged kernel handles, all with 512 threads per CTA.
constexpr int kRaggedMinL = 256;
constexpr int kRaggedMaxL = 8192;
constexpr int kRaggedNT = 512;

// Dynamic shared memory of k_ragged (the largest body it runs).
int ragged_smem_bytes();
// Launch on `st` with `grid` persistent CTAs; -1 if the kernel cannot be set up.
int launch_ragged(const RaggedArgs& ra, int grid, cudaStream_t st);
// Columns per encode tile / per decode tile of length L (k <= n/2, k > n/2).
int ragged_wt_enc(int L);
int ragged_wt_dec(int L, bool blocked);

}  // namespace fntrs
