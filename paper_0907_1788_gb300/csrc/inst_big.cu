// Tile kernels for L = 4096 and 8192.
#include "inst.cuh"

namespace fntrs {
void register_tile_ops_big() {
  register_ops(make_tile_ops<4096>());
  register_ops(make_tile_ops<8192>());
}
}  // namespace fntrs
