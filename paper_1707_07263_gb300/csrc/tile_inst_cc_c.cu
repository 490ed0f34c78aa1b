// tile_inst_cc_c.cu -- compiled column-pass (c-fast in, c-fast out) tile-FFT variants (lengths 2^11..2^14).
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tile_kernel_cc_c(int lg, int C) {
  static const TileKernelInfo tab[] = {
      GBFFT_TK(11, 1, true, true, MAP_CC),
      GBFFT_TK(11, 2, true, true, MAP_CC),
      GBFFT_TK(11, 4, true, true, MAP_CC),
      GBFFT_TK(11, 8, true, true, MAP_CC),
      GBFFT_TK(12, 1, true, true, MAP_CC),
      GBFFT_TK(12, 2, true, true, MAP_CC),
      GBFFT_TK(12, 4, true, true, MAP_CC),
      GBFFT_TK(13, 1, true, true, MAP_CC),
      GBFFT_TK(13, 2, true, true, MAP_CC),
      GBFFT_TK(14, 1, true, true, MAP_CC),
  };
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

}  // namespace gbfft
