// tile_inst_jc_a.cu -- compiled row-pass (j-fast in, c-fast out) tile-FFT variants (lengths 2^5..2^8).
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tile_kernel_jc_a(int lg, int C) {
  static const TileKernelInfo tab[] = {
      GBFFT_TK(5, 1, false, true, MAP_JC),
      GBFFT_TK(5, 2, false, true, MAP_JC),
      GBFFT_TK(5, 4, false, true, MAP_JC),
      GBFFT_TK(5, 8, false, true, MAP_JC),
      GBFFT_TK(5, 16, false, true, MAP_JC),
      GBFFT_TK(5, 32, false, true, MAP_JC),
      GBFFT_TK(5, 64, false, true, MAP_JC),
      GBFFT_TK(6, 1, false, true, MAP_JC),
      GBFFT_TK(6, 2, false, true, MAP_JC),
      GBFFT_TK(6, 4, false, true, MAP_JC),
      GBFFT_TK(6, 8, false, true, MAP_JC),
      GBFFT_TK(6, 16, false, true, MAP_JC),
      GBFFT_TK(6, 32, false, true, MAP_JC),
      GBFFT_TK(6, 64, false, true, MAP_JC),
      GBFFT_TK(7, 1, false, true, MAP_JC),
      GBFFT_TK(7, 2, false, true, MAP_JC),
      GBFFT_TK(7, 4, false, true, MAP_JC),
      GBFFT_TK(7, 8, false, true, MAP_JC),
      GBFFT_TK(7, 16, false, true, MAP_JC),
      GBFFT_TK(7, 32, false, true, MAP_JC),
      GBFFT_TK(7, 64, false, true, MAP_JC),
      GBFFT_TK(8, 1, false, true, MAP_JC),
      GBFFT_TK(8, 2, false, true, MAP_JC),
      GBFFT_TK(8, 4, false, true, MAP_JC),
      GBFFT_TK(8, 8, false, true, MAP_JC),
      GBFFT_TK(8, 16, false, true, MAP_JC),
      GBFFT_TK(8, 32, false, true, MAP_JC),
      GBFFT_TK(8, 64, false, true, MAP_JC),
  };
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

}  // namespace gbfft
