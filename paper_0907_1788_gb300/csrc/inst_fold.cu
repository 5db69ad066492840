// TMA-staged encode of n = 8192 codes with k > 4096 (k_encode_tma_fold).
#include <cuda.h>
#include <cuda_runtime.h>

#include "encode_fold.cuh"
#include "inst.cuh"

namespace fntrs {

int launch_encode_tma_fold(const KArgs& a, const TmaEncodeArgs& t, cudaStream_t st) {
  using S = SchedFor<4096>::type;
  auto kern = k_encode_tma_fold<S, 512>;
  constexpr int work = ((Lay<S, 4>::WORDS * 4) + 127) / 128 * 128;
  auto bytes = [&](int rows) { return work + rows * 8 * 2 + kSchedBytes; };
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes(8192)) !=
        cudaSuccess)
      return -1;
    done[dev & 63] = true;
  }
  kern<<<t.grid, 512, bytes(t.rows_staged), st>>>(
      a, t.twc, t.rows_staged, t.box_rows, *static_cast<const CUtensorMap*>(t.map));
  count_launch();
  return 0;
}

}  // namespace fntrs
