// tile_inst_cc_b.cu -- compiled column-pass (c-fast in, c-fast out) tile-FFT variants (lengths 2^8..2^10).
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tile_kernel_cc_b(int lg, int C) {
  static const TileKernelInfo tab[] = {
      GBFFT_TK(8, 1, true, true, MAP_CC),
      GBFFT_TK(8, 2, true, true, MAP_CC),
      GBFFT_TK(8, 4, true, true, MAP_CC),
      GBFFT_TK(8, 8, true, true, MAP_CC),
      GBFFT_TK(8, 16, true, true, MAP_CC),
      GBFFT_TK(8, 32, true, true, MAP_CC),
      GBFFT_TK(8, 64, true, true, MAP_CC),
      GBFFT_TK(9, 1, true, true, MAP_CC),
      GBFFT_TK(9, 2, true, true, MAP_CC),
      GBFFT_TK(9, 4, true, true, MAP_CC),
      GBFFT_TK(9, 8, true, true, MAP_CC),
      GBFFT_TK(9, 16, true, true, MAP_CC),
      GBFFT_TK(9, 32, true, true, MAP_CC),
      GBFFT_TK(10, 1, true, true, MAP_CC),
      GBFFT_TK(10, 2, true, true, MAP_CC),
      GBFFT_TK(10, 4, true, true, MAP_CC),
      GBFFT_TK(10, 8, true, true, MAP_CC),
      GBFFT_TK(10, 16, true, true, MAP_CC),
  };
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

}  // namespace gbfft
