// tile_inst_rc.cu -- compiled fused range-compression kernels (forward
// transform, filter product, inverse transform in one pass over each row),
// one per length 2^1..2^14 with jj_cols(lg) rows per CTA.
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_RC(LG)                                                                            \
  {(const void*)&tile_rc_kernel<LG, jj_cols(LG)>, TileCfg<LG, jj_cols(LG), false, false>::T,    \
   jj_cols(LG) * TileCfg<LG, jj_cols(LG), false, false>::LP * 8, LG, jj_cols(LG), MAP_JJ}

const TileKernelInfo* tile_kernel_rc(int lg) {
  static const TileKernelInfo tab[] = {
      GBFFT_RC(1),  GBFFT_RC(2),  GBFFT_RC(3),  GBFFT_RC(4),  GBFFT_RC(5),  GBFFT_RC(6),  GBFFT_RC(7),
      GBFFT_RC(8),  GBFFT_RC(9),  GBFFT_RC(10), GBFFT_RC(11), GBFFT_RC(12), GBFFT_RC(13), GBFFT_RC(14),
  };
  if (lg < 1 || lg > 14) return nullptr;
  return &tab[lg - 1];
}

}  // namespace gbfft
