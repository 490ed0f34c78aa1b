// tile_inst_cc_a.cu -- compiled column-pass (c-fast in, c-fast out) tile-FFT variants (lengths 2^1..2^7).
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tile_kernel_cc_a(int lg, int C) {
  static const TileKernelInfo tab[] = {
      GBFFT_TK(1, 1, true, true, MAP_CC),
      GBFFT_TK(1, 2, true, true, MAP_CC),
      GBFFT_TK(1, 4, true, true, MAP_CC),
      GBFFT_TK(1, 8, true, true, MAP_CC),
      GBFFT_TK(1, 16, true, true, MAP_CC),
      GBFFT_TK(2, 1, true, true, MAP_CC),
      GBFFT_TK(2, 2, true, true, MAP_CC),
      GBFFT_TK(2, 4, true, true, MAP_CC),
      GBFFT_TK(2, 8, true, true, MAP_CC),
      GBFFT_TK(2, 16, true, true, MAP_CC),
      GBFFT_TK(3, 1, true, true, MAP_CC),
      GBFFT_TK(3, 2, true, true, MAP_CC),
      GBFFT_TK(3, 4, true, true, MAP_CC),
      GBFFT_TK(3, 8, true, true, MAP_CC),
      GBFFT_TK(3, 16, true, true, MAP_CC),
      GBFFT_TK(4, 1, true, true, MAP_CC),
      GBFFT_TK(4, 2, true, true, MAP_CC),
      GBFFT_TK(4, 4, true, true, MAP_CC),
      GBFFT_TK(4, 8, true, true, MAP_CC),
      GBFFT_TK(4, 16, true, true, MAP_CC),
      GBFFT_TK(5, 1, true, true, MAP_CC),
      GBFFT_TK(5, 2, true, true, MAP_CC),
      GBFFT_TK(5, 4, true, true, MAP_CC),
      GBFFT_TK(5, 8, true, true, MAP_CC),
      GBFFT_TK(5, 16, true, true, MAP_CC),
      GBFFT_TK(5, 32, true, true, MAP_CC),
      GBFFT_TK(5, 64, true, true, MAP_CC),
      GBFFT_TK(6, 1, true, true, MAP_CC),
      GBFFT_TK(6, 2, true, true, MAP_CC),
      GBFFT_TK(6, 4, true, true, MAP_CC),
      GBFFT_TK(6, 8, true, true, MAP_CC),
      GBFFT_TK(6, 16, true, true, MAP_CC),
      GBFFT_TK(6, 32, true, true, MAP_CC),
      GBFFT_TK(6, 64, true, true, MAP_CC),
      GBFFT_TK(7, 1, true, true, MAP_CC),
      GBFFT_TK(7, 2, true, true, MAP_CC),
      GBFFT_TK(7, 4, true, true, MAP_CC),
      GBFFT_TK(7, 8, true, true, MAP_CC),
      GBFFT_TK(7, 16, true, true, MAP_CC),
      GBFFT_TK(7, 32, true, true, MAP_CC),
      GBFFT_TK(7, 64, true, true, MAP_CC),
  };
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

}  // namespace gbfft
