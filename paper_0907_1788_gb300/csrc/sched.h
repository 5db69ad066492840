// Radix schedules of the tile transform and the launch registry.
#pragma once
#include "kargs.h"

namespace fntrs {

// Largest transform held by one CTA (u32 words, at most 128 KB of shared
// memory per buffer); codes that do not fit split n = C * kLocalL.
constexpr int kTileMaxL = 32768;
constexpr int kLocalL = 4096;
// Largest tile length of the product-tree route's pairwise products.
constexpr int kTreeTileL = 8192;

// radix factorisation of each tile length (each radix <= 32)
inline void sched_radices(int L, int r[3]) {
  r[0] = L; r[1] = 1; r[2] = 1;
  switch (L) {
    case 64: r[0] = 8; r[1] = 8; break;
    case 128: r[0] = 16; r[1] = 8; break;
    case 256: r[0] = 16; r[1] = 16; break;
    case 512: r[0] = 32; r[1] = 16; break;
    case 1024: r[0] = 32; r[1] = 32; break;
    case 2048: r[0] = 16; r[1] = 16; r[2] = 8; break;
    case 4096: r[0] = 16; r[1] = 16; r[2] = 16; break;
    case 8192: r[0] = 32; r[1] = 16; r[2] = 16; break;
    case 16384: r[0] = 32; r[1] = 32; r[2] = 16; break;
    case 32768: r[0] = 32; r[1] = 32; r[2] = 32; break;
    default: break;  // L <= 32: one pass
  }
}

// Codewords per CTA for one-buffer kernels (encode, FNT, decode) and for
// two-buffer kernels (split decode, product-tree level): L * WT * 4 bytes of
// shared memory per buffer, at most 128 KB in all.
constexpr int wt_one(int L) { return L <= 32 ? 128 : (L >= 1024 ? 32768 / L : 32); }
constexpr int wt_two(int L) { return L <= 32 ? 128 : (L >= 512 ? 16384 / L : 32); }
constexpr int nt_for(int L) { return L <= 32 ? 128 : (L >= 256 ? 512 : 256); }

using Launch = void (*)(const KArgs&, int grid_y, cudaStream_t);

struct TileOps {
  int L = 0, wt1 = 0, wt2 = 0, nt = 0;
  Launch encode = nullptr;      // fold-load source, rows cc + C*j
  Launch fnt_fwd = nullptr;     // rows -> rows, scaled
  Launch fnt_inv = nullptr;
  Launch lossless = nullptr;    // inverse transform, first k rows as 16-bit symbols
  Launch decode = nullptr;      // fused decode, k <= n/2
  Launch decode_split = nullptr;  // fused decode, k > n/2
  Launch poly_level = nullptr;  // product-tree level (L = 2d)
  // log-domain pattern build (n = L) in one launch of D CTAs
  void (*plan_fused)(const PlanArgs&, cudaStream_t) = nullptr;
  // decode with half-width tiles staged by cp.async, two CTAs per SM (k <= n/2)
  int (*decode_cpa)(const KArgs&, const uint32_t* pat32, cudaStream_t) = nullptr;
  int wt_cpa = 0;
};

// Registry filled by the instantiation units.
const TileOps& tile_ops(int L);
void register_tile_ops_small();
void register_tile_ops_mid();
void register_tile_ops_big();
void register_tile_ops_huge();

// TMA-staged encode for tile length L (C = 1) or n = 2L (C = 2).
// Returns -1 if the configuration has no instantiation.
struct TmaEncodeArgs {
  const uint32_t* twc;
  int rows_staged, box_rows, grid;
  const void* map;  // CUtensorMap*
};
int launch_encode_tma(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st);

// TMA-staged decode (n = L <= tile limit, k <= n/2, packed rows).
struct TmaDecodeArgs {
  const uint32_t* pat32;
  const uint32_t* rowtab;  // (position << 17) | weight of received row i < k
  int rows_staged, box_rows;
  int sms;          // SMs of the device (the launch sizes its last round of tiles by it)
  const void* map;  // CUtensorMap*
};
int launch_decode_tma(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st);

// Split-transform passes (n = C * kLocalL).
Launch local_launcher(bool inverse, int mode);
Launch cross_launcher(int C, bool inverse, int load_mode);

}  // namespace fntrs
