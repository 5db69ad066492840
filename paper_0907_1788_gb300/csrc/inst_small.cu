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

namespace fntrs {
template <int L>
static int tma_c1(const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  using S = typename SchedFor<L>::type;
  return launch_encode_tma_t<S, wt_one(L), nt_for(L), 1>(
      a, t.twc, t.rows_staged, t.box_rows, *static_cast<const CUtensorMap*>(t.map), t.grid, st);
}
int launch_encode_tma_small(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  if (C != 1) return -1;
  switch (L) {
    case 64: return tma_c1<64>(a, t, st);
    case 128: return tma_c1<128>(a, t, st);
    case 256: return tma_c1<256>(a, t, st);
    default: return -1;
  }
}
}  // namespace fntrs

namespace fntrs {
int launch_decode_tma_small(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  switch (L) {
    case 64: return decode_tma_for<64>(a, t, st);
    case 128: return decode_tma_for<128>(a, t, st);
    case 256: return decode_tma_for<256>(a, t, st);
    default: return -1;
  }
}
}  // namespace fntrs
