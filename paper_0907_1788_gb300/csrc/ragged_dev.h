// Work list of the ragged persistent kernel (k_ragged): every group with
// n >= 256 contributes encode tiles, pattern-build items (decode groups) and
// decode tiles; one launch of k_ragged runs them all, each CTA taking work
// items in list order from an atomic counter.
//
// How a group's work is cut depends on its length:
//   tile  (encode n <= 16384; decode n <= 16384, or n = 32768 with k <= n/2):
//         one CTA holds a whole codeword tile in shared memory, as the
//         standalone tile kernels do;
//   split (encode n >= 32768; decode n = 65536, or n = 32768 with k > n/2): a
//         work item is a tile of up to 8 columns, and its CTA runs the whole
//         split transform of those columns itself (radix-n/4096 cross pass
//         into its own global scratch, then the n/4096 local 4096-point
//         passes), so the items of a group never wait on one another;
//   pattern build, n <= 16384: the one-launch build's D digit items;
//   pattern build, n >= 32768: one spectrum item (the transform of the
//         received-position indicator), then D digit items that wait for it,
//         the last of which finishes the tables.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kargs.h"

namespace fntrs {

enum RaggedItemKind : int { RI_ENC = 0, RI_PLAN = 1, RI_DEC = 2, RI_SPEC = 3 };

// Scratch of a long pattern build (n >= 32768), all in the group's own buffer.
struct LongPlanDev {
  uint32_t* ind;   // [n] received-position indicator (row + 1, then 0/1)
  uint32_t* spec;  // [n] its transform
  uint32_t* prod;  // [D][n] spectrum times each digit's table
  uint32_t* aval;  // [n] A(r^j) (k > n/2)
  uint32_t* coef;  // [n] coefficients of A (k > n/2)
  uint32_t* M2;    // [n][2] coefficient halves
  uint32_t* E2;    // [n][2] their transforms
};

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
  int split_enc;  // encode items run the in-CTA split transform (n = 65536)
  int split_dec;  // decode items run the in-CTA split transform
  int long_plan;  // pattern build by a spectrum item + digit items (n >= 32768)
  int C;          // n / 4096 (split transforms)
  KArgs xenc;     // split encode base: L = 4096, C, powers of r_n, 4096-point tables
  KArgs xdec;     // split decode base: the same plus pattern tables, slots = the encoded rows
  KArgs colf;     // one-column transforms of the long build: forward (tables of n or of 4096)
  KArgs coli;     // the same, inverse
  LongPlanDev lp;
};

struct RaggedArgs {
  const RaggedItem* items;
  int nitems;
  const RaggedGroupDev* groups;
  unsigned* next;       // work counter (zero before the launch)
  unsigned* enc_done;   // [groups] finished encode tiles (zero before the launch)
  unsigned* plan_done;  // [groups] 1 once the pattern tables are written (zero before)
  unsigned* spec_done;  // [groups] 1 once a long build's spectrum is written (zero before)
  uint32_t* cta_scratch;      // per CTA: split-transform buffers (blockIdx.x * cta_words)
  size_t cta_words;
};

// Code lengths the ragged kernel handles, all with 512 threads per CTA.
constexpr int kRaggedMinL = 256;
constexpr int kRaggedMaxL = 65536;
constexpr int kRaggedNT = 512;
// Columns of a split-transform work item (the 4096-point local tile's width)
// and the split buffers one CTA needs per column of length n (decode with
// k > n/2: four n x 8 buffers).
constexpr int kRaggedSplitWT = 8;
constexpr int kRaggedSplitBufs = 4;

// Dynamic shared memory of k_ragged (the largest body it runs).
int ragged_smem_bytes();
// Launch on `st` with `grid` persistent CTAs; -1 if the kernel cannot be set up.
int launch_ragged(const RaggedArgs& ra, int grid, cudaStream_t st);
// Columns per encode tile / per decode tile of length L (k <= n/2, k > n/2).
int ragged_wt_enc(int L);
int ragged_wt_dec(int L, bool blocked);
// Which groups run the in-CTA split transform, and which build long patterns.
inline bool ragged_split_enc(int L) { return L >= 32768; }
inline bool ragged_split_dec(int L, bool blocked) { return L > 32768 || (L == 32768 && blocked); }
inline bool ragged_long_plan(int L) { return L >= 32768; }

}  // namespace fntrs
