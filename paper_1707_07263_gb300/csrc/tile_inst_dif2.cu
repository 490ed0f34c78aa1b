// tile_inst_dif2.cu -- compiled two-CTA radix-2 split kernels (tile_fft_dif2_kernel),
// half lengths 2^11..2^13 (transform lengths 2^12..2^14).
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_DIF2(LG)                                                                                   \
  {(const void*)&tile_fft_dif2_kernel<LG>, TileCfg<LG, 1, false, false>::T,                               \
   TileCfg<LG, 1, false, false>::SMEM_BYTES, LG, 1, MAP_JJ}

const TileKernelInfo* tile_kernel_dif2(int lg) {
  static const TileKernelInfo tab[] = {GBFFT_DIF2(11), GBFFT_DIF2(12), GBFFT_DIF2(13)};
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg) return &k;
  return nullptr;
}

}  // namespace gbfft
