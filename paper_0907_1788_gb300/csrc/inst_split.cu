// Passes of split transforms n = C * 4096 (n = 8192 .. 65536):
// cross passes (radix C over stride-4096 rows) and local passes (length-4096
// tile transforms of each block with the output modes of kargs.h).
#include "inst.cuh"

namespace fntrs {

namespace {
using SL = SchedFor<kLocalL>::type;
constexpr int kWT = wt_one(kLocalL);
constexpr int kNT = nt_for(kLocalL);

template <bool INV, int MODE>
void launch_local(const KArgs& a, int gy, cudaStream_t st) {
  launch_tile<SL, kWT, kNT, INV, LoadRows32<kWT>, StoreLocal<kWT, MODE>>(a, gy, st);
}

template <int C, bool INV, int LOADM>
void launch_cross(const KArgs& a, int, cudaStream_t st) {
  const long long tasks = (long long)a.L * a.W;
  const unsigned blocks = (unsigned)((tasks + 255) / 256);
  k_cross<C, INV, LOADM><<<blocks, 256, 0, st>>>(a);
  count_launch();
}

template <int C>
Launch cross_for(bool inverse, int load_mode) {
  if (!inverse && load_mode == CL_SRC16) return &launch_cross<C, false, CL_SRC16>;
  if (inverse && load_mode == CL_RECV) return &launch_cross<C, true, CL_RECV>;
  if (!inverse && load_mode == CL_U32) return &launch_cross<C, false, CL_U32>;
  if (inverse && load_mode == CL_U32) return &launch_cross<C, true, CL_U32>;
  return nullptr;
}
}  // namespace

Launch local_launcher(bool inverse, int mode) {
  if (!inverse) {
    switch (mode) {
      case LM_ENC: return &launch_local<false, LM_ENC>;
      case LM_FNT: return &launch_local<false, LM_FNT>;
      case LM_WORK_AHAT: return &launch_local<false, LM_WORK_AHAT>;
      case LM_X_PARTIAL: return &launch_local<false, LM_X_PARTIAL>;
      case LM_ACCUM: return &launch_local<false, LM_ACCUM>;
      default: return nullptr;
    }
  }
  switch (mode) {
    case LM_FNT: return &launch_local<true, LM_FNT>;
    case LM_WORK: return &launch_local<true, LM_WORK>;
    case LM_OUT16: return &launch_local<true, LM_OUT16>;
    case LM_SPLIT: return &launch_local<true, LM_SPLIT>;
    case LM_OUT16_ADD: return &launch_local<true, LM_OUT16_ADD>;
    default: return nullptr;
  }
}

Launch cross_launcher(int C, bool inverse, int load_mode) {
  switch (C) {
    case 2: return cross_for<2>(inverse, load_mode);
    case 4: return cross_for<4>(inverse, load_mode);
    case 8: return cross_for<8>(inverse, load_mode);
    case 16: return cross_for<16>(inverse, load_mode);
    default: return nullptr;
  }
}

}  // namespace fntrs
