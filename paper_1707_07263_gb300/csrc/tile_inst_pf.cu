// tile_inst_pf.cu -- compiled persistent single-pass kernels with an L2
// prefetch of the next transform (tile_fft_pf_kernel), lengths 2^12..2^14;
// kernel signature void(TileArgs, long long ntiles).
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_PF(LG) \
  {(const void*)&tile_fft_pf_kernel<LG>, TileCfg<LG, 1, false, false>::T, TileCfg<LG, 1, false, false>::SMEM_BYTES, LG, 1, MAP_JJ}

const TileKernelInfo* tile_kernel_pf(int lg) {
  static const TileKernelInfo tab[] = {GBFFT_PF(12), GBFFT_PF(13), GBFFT_PF(14)};
  if (lg < 12 || lg > 14) return nullptr;
  return &tab[lg - 12];
}

}  // namespace gbfft
