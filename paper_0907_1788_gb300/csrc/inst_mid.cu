// Tile kernels for L = 512 .. 2048.
#include "inst.cuh"

namespace fntrs {
void register_tile_ops_mid() {
  register_ops(make_tile_ops<512>());
  register_ops(make_tile_ops<1024>());
  register_ops(make_tile_ops<2048>());
}
}  // namespace fntrs

namespace fntrs {
template <int L>
static int tma_c1(const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  using S = typename SchedFor<L>::type;
  return launch_encode_tma_t<S, wt_one(L), nt_for(L), 1>(
      a, t.twc, t.rows_staged, t.box_rows, *static_cast<const CUtensorMap*>(t.map), t.grid, st);
}
int launch_encode_tma_mid(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  if (C != 1) return -1;
  switch (L) {
    case 512: return tma_c1<512>(a, t, st);
    case 1024: return tma_c1<1024>(a, t, st);
    case 2048: return tma_c1<2048>(a, t, st);
    default: return -1;
  }
}
}  // namespace fntrs

namespace fntrs {
int launch_decode_tma_mid(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  switch (L) {
    case 512: return decode_tma_for<512>(a, t, st);
    case 1024: return decode_tma_for<1024>(a, t, st);
    case 2048: return decode_tma_for<2048>(a, t, st);
    default: return -1;
  }
}
}  // namespace fntrs
