// Launch wrappers for the kernel templates (included by the instantiation units).
#pragma once
#include <cuda_runtime.h>

#include <cuda.h>

#include "kernels.cuh"
#include "sched.h"

namespace fntrs {

void count_launch();

template <int L> struct SchedFor { using type = Sched<L, L>; };
template <> struct SchedFor<64> { using type = Sched<64, 8, 8>; };
template <> struct SchedFor<128> { using type = Sched<128, 16, 8>; };
template <> struct SchedFor<256> { using type = Sched<256, 16, 16>; };
template <> struct SchedFor<512> { using type = Sched<512, 32, 16>; };
template <> struct SchedFor<1024> { using type = Sched<1024, 32, 32>; };
template <> struct SchedFor<2048> { using type = Sched<2048, 16, 16, 8>; };
template <> struct SchedFor<4096> { using type = Sched<4096, 16, 16, 16>; };
template <> struct SchedFor<8192> { using type = Sched<8192, 32, 16, 16>; };
template <> struct SchedFor<16384> { using type = Sched<16384, 32, 32, 16>; };
template <> struct SchedFor<32768> { using type = Sched<32768, 32, 32, 32>; };

// Opt a kernel into more than 48 KB of dynamic shared memory, once per device.
template <class Tag, class F>
inline void ensure_smem(F* kern, int bytes) {
  static bool done[64] = {};
  if (bytes <= 48 * 1024) return;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done[dev & 63] = true;
  }
}

template <class S, int WT, int NT, bool INV, class LD, class ST>
void launch_tile(const KArgs& a, int gy, cudaStream_t st) {
  auto kern = k_tile<S, WT, NT, INV, LD, ST>;
  const int smem = smem_words<S, WT>() * 4;
  struct Tag {};
  ensure_smem<Tag>(kern, smem);
  dim3 grid((a.W + WT - 1) / WT, gy);
  kern<<<grid, NT, smem, st>>>(a);
  count_launch();
}

template <class S, int WT, int NT>
void launch_decode(const KArgs& a, int, cudaStream_t st) {
  auto kern = k_decode<S, WT, NT>;
  const int smem = smem_words<S, WT>() * 4;
  struct Tag {};
  ensure_smem<Tag>(kern, smem);
  dim3 grid((a.W + WT - 1) / WT, 1);
  kern<<<grid, NT, smem, st>>>(a);
  count_launch();
}

template <class S, int WT, int NT>
void launch_decode_split(const KArgs& a, int, cudaStream_t st) {
  auto kern = k_decode_split<S, WT, NT>;
  const int smem = 2 * smem_words<S, WT>() * 4;
  struct Tag {};
  ensure_smem<Tag>(kern, smem);
  dim3 grid((a.W + WT - 1) / WT, 1);
  kern<<<grid, NT, smem, st>>>(a);
  count_launch();
}

template <class S, int WT, int NT>
void launch_poly_level(const KArgs& a, int, cudaStream_t st) {
  auto kern = k_poly_level<S, WT, NT>;
  const int smem = 2 * smem_words<S, WT>() * 4;
  struct Tag {};
  ensure_smem<Tag>(kern, smem);
  const int npairs = (a.nodes + 1) / 2;
  dim3 grid((npairs + WT - 1) / WT, 1);
  kern<<<grid, NT, smem, st>>>(a);
  count_launch();
}

template <class S, int NT>
void launch_plan_fused(const PlanArgs& pa, cudaStream_t st) {
  auto kern = k_plan_fused<S, NT>;
  const int smem = (Lay<S, 1>::WORDS + S::L) * 4;
  struct Tag {};
  ensure_smem<Tag>(kern, smem);
  kern<<<pa.D, NT, smem, st>>>(pa);
  count_launch();
}

template <class S, int WT, int NT, bool HALF, int MINB>
int launch_decode_cpa_h(const KArgs& a, const uint32_t* pat32, cudaStream_t st) {
  auto kern = k_decode_cpa<S, WT, NT, HALF, MINB>;
  constexpr int work = ((Lay<S, WT>::WORDS * 4) + 127) / 128 * 128;
  auto bytes = [&](int k) { return work + ((k * WT + 3) / 4 * 4) * 4 + kSchedBytes; };
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes(S::L / 2)) !=
        cudaSuccess)
      return -1;
    done[dev & 63] = true;
  }
  kern<<<(a.W + WT - 1) / WT, NT, bytes(a.k), st>>>(a, pat32);
  count_launch();
  return 0;
}

template <class S, int WT, int NT, int MINB = 2>
int launch_decode_cpa_t(const KArgs& a, const uint32_t* pat32, cudaStream_t st) {
  if (2 * a.k == S::L) return launch_decode_cpa_h<S, WT, NT, true, MINB>(a, pat32, st);
  return launch_decode_cpa_h<S, WT, NT, false, MINB>(a, pat32, st);
}

template <int L>
TileOps make_tile_ops() {
  using S = typename SchedFor<L>::type;
  constexpr int W1 = wt_one(L), W2 = wt_two(L), NT = nt_for(L);
  TileOps ops;
  ops.L = L;
  ops.wt1 = W1;
  ops.wt2 = W2;
  ops.nt = NT;
  ops.encode = &launch_tile<S, W1, NT, false, LoadSrcFold<W1>, StoreRows32<W1>>;
  ops.fnt_fwd = &launch_tile<S, W1, NT, false, LoadRows32<W1>, StoreRows32<W1>>;
  ops.fnt_inv = &launch_tile<S, W1, NT, true, LoadRows32<W1>, StoreRows32<W1>>;
  ops.lossless = &launch_tile<S, W1, NT, true, LoadRows32<W1>, StoreFirstK16<W1>>;
  ops.decode = &launch_decode<S, W1, NT>;
  // two-buffer kernels need one codeword of two L-word buffers per CTA
  if constexpr (W2 > 0) {
    ops.decode_split = &launch_decode_split<S, W2, NT>;
    if constexpr (S::NP >= 2) ops.poly_level = &launch_poly_level<S, W2, NT>;
  }
  if constexpr (L >= 64 && (Lay<S, 1>::WORDS + L) * 4 <= 227 * 1024) {
    ops.plan_fused = &launch_plan_fused<S, 512>;
  }
  if constexpr (L == 4096 || L == 8192) {
    ops.decode_cpa = &launch_decode_cpa_t<S, W1 / 2, 256>;
    ops.wt_cpa = W1 / 2;
  } else if constexpr (L == 16384 || L == 32768) {
    // the one-CTA tile's two (one) codewords, rows staged by 8-byte (4-byte)
    // copies (a TMA row would need 16 bytes); one CTA per SM
    ops.decode_cpa = &launch_decode_cpa_t<S, W1, 512, 1>;
    ops.wt_cpa = W1;
  }
  return ops;
}

void register_ops(const TileOps& ops);

// TMA-staged encode (k_encode_tma): dynamic shared memory bytes.
template <class S, int WT>
constexpr int encode_tma_smem(int rows_staged) {
  return ((Lay<S, WT>::WORDS * 4) + 127) / 128 * 128 + rows_staged * WT * 2 + kSchedBytes;
}

template <class S, int WT, int NT, int C>
int launch_encode_tma_t(const KArgs& a, const uint32_t* twc, int rows_staged, int box_rows,
                        const CUtensorMap& map, int grid, cudaStream_t st) {
  auto kern = k_encode_tma<S, WT, NT, C>;
  const int smem = encode_tma_smem<S, WT>(rows_staged);
  static bool done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             encode_tma_smem<S, WT>(S::L)) != cudaSuccess)
      return -1;
    done[dev & 63] = true;
  }
  kern<<<grid, NT + 32, smem, st>>>(a, twc, rows_staged, box_rows, map);  // + producer warp
  count_launch();
  return 0;
}

}  // namespace fntrs

namespace fntrs {
constexpr int decode_tma_max_rows(int L) { return L <= 256 ? L : L / 2; }

// Number of WT-wide tiles kept when the last round of a one-CTA-per-tile
// launch (nwide tiles over `resident` CTAs at a time) is cut into half-width
// tiles: only when the remainder r fills at most half the CTAs, so that its
// 2r half tiles still form a single round.
inline int tail_full_tiles(int nwide, int resident, int wt) {
  if (wt < 2 || resident <= 0) return nwide;
  const int r = nwide % resident;
  return (r != 0 && 2 * r <= resident) ? nwide - r : nwide;
}

template <class S, int WT, int NT, bool HALF>
int launch_decode_tma_h(const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  auto kern = k_decode_tma<S, WT, NT, HALF>;
  // the staged tables (HALF, L >= 4096) need the stage to hold 2 L words
  if (HALF && S::L >= 4096 && (!a.twf_sw || (size_t)t.rows_staged * WT < 2 * (size_t)S::L))
    return -1;
  constexpr int work = ((Lay<S, WT>::WORDS * 4) + 127) / 128 * 128;
  const int smem = work + t.rows_staged * WT * 4 + kSchedBytes;
  static bool done[64] = {};
  static int occ[64] = {};  // CTAs resident per SM at the largest stage
  int dev = 0;
  cudaGetDevice(&dev);
  if (!done[dev & 63]) {
    const int max_smem = work + decode_tma_max_rows(S::L) * WT * 4 + kSchedBytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) !=
        cudaSuccess)
      return -1;
    int o = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT + 32, max_smem) !=
        cudaSuccess)
      o = 1;
    occ[dev & 63] = o > 0 ? o : 1;
    done[dev & 63] = true;
  }
  const int nwide = (a.W + WT - 1) / WT;
  const int nfull = tail_full_tiles(nwide, t.sms * occ[dev & 63], WT);
  const int grid = nfull + 2 * (nwide - nfull);  // one CTA per tile (see clc_take)
  // NT decoding threads and one producer warp
  kern<<<grid, NT + 32, smem, st>>>(a, t.rowtab, t.rows_staged, t.box_rows, nfull,
                               *static_cast<const CUtensorMap*>(t.map));
  count_launch();
  return 0;
}

// k = n/2 exactly takes the pruned (HALF) variant
template <class S, int WT, int NT>
int launch_decode_tma_t(const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  if (2 * a.k == S::L) return launch_decode_tma_h<S, WT, NT, true>(a, t, st);
  return launch_decode_tma_h<S, WT, NT, false>(a, t, st);
}

template <int L>
int decode_tma_for(const KArgs& a, const TmaDecodeArgs& t, cudaStream_t st) {
  using S = typename SchedFor<L>::type;
  return launch_decode_tma_t<S, wt_one(L), nt_for(L)>(a, t, st);
}
}  // namespace fntrs
