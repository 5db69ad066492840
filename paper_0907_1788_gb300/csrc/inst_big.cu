// Tile kernels for L = 4096 and 8192.
#include "inst.cuh"

namespace fntrs {
void register_tile_ops_big() {
  register_ops(make_tile_ops<4096>());
  register_ops(make_tile_ops<8192>());
}
}  // namespace fntrs

namespace fntrs {
int launch_encode_tma_big(int L, int C, const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  using S = SchedFor<4096>::type;
  constexpr int W = wt_one(4096), NT = nt_for(4096);
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(t.map);
  if (L != 4096) return -1;
  if (C == 1) return launch_encode_tma_t<S, W, NT, 1>(a, t.twc, t.rows_staged, t.box_rows, m, t.grid, st);
  if (C == 2) return launch_encode_tma_t<S, W, NT, 2>(a, t.twc, t.rows_staged, t.box_rows, m, t.grid, st);
  return -1;
}
}  // namespace fntrs

namespace fntrs {
int launch_decode_tma_big(int L, const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  switch (L) {
    case 4096: return decode_tma_for<4096>(a, t, st);
    case 8192: return decode_tma_for<8192>(a, t, st);
    default: return -1;
  }
}
}  // namespace fntrs
