// Tile kernels for L = 2 .. 256.
#include "inst.cuh"

namespace fntrs {
void register_tile_ops_small() {
  register_ops(make_tile_ops<2>());
  register_ops(make_tile_ops<4>());
  register_ops(make_tile_ops<8>());
  register_ops(make_tile_ops<16>());
  register_ops(make_tile_ops<32>());
  register_ops(make_tile_ops<64>());
  register_ops(make_tile_ops<128>());
  register_ops(make_tile_ops<256>());
}
}  // namespace fntrs
