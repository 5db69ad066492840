// Tile kernels for L = 512 .. 2048.
#include "inst.cuh"

namespace fntrs {
void register_tile_ops_mid() {
  register_ops(make_tile_ops<512>());
  register_ops(make_tile_ops<1024>());
  register_ops(make_tile_ops<2048>());
}
}  // namespace fntrs
