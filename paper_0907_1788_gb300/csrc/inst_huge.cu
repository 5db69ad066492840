// Tile kernels for L = 16384 and 32768 (one CTA holds the whole transform of
// two codewords, respectively one).
#include "inst.cuh"

namespace fntrs {
void register_tile_ops_huge() {
  register_ops(make_tile_ops<16384>());
  register_ops(make_tile_ops<32768>());
}
}  // namespace fntrs
