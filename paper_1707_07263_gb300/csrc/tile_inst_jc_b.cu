// tile_inst_jc_b.cu -- compiled row-pass (j-fast in, c-fast out) tile-FFT variants (lengths 2^9..2^14).
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tile_kernel_jc_b(int lg, int C) {
  static const TileKernelInfo tab[] = {
      GBFFT_TK(9, 1, false, true, MAP_JC),
      GBFFT_TK(9, 2, false, true, MAP_JC),
      GBFFT_TK(9, 4, false, true, MAP_JC),
      GBFFT_TK(9, 8, false, true, MAP_JC),
      GBFFT_TK(9, 16, false, true, MAP_JC),
      GBFFT_TK(9, 32, false, true, MAP_JC),
      GBFFT_TK(10, 1, false, true, MAP_JC),
      GBFFT_TK(10, 2, false, true, MAP_JC),
      GBFFT_TK(10, 4, false, true, MAP_JC),
      GBFFT_TK(10, 8, false, true, MAP_JC),
      GBFFT_TK(10, 16, false, true, MAP_JC),
      GBFFT_TK(11, 1, false, true, MAP_JC),
      GBFFT_TK(11, 2, false, true, MAP_JC),
      GBFFT_TK(11, 4, false, true, MAP_JC),
      GBFFT_TK(11, 8, false, true, MAP_JC),
      GBFFT_TK(12, 1, false, true, MAP_JC),
      GBFFT_TK(12, 2, false, true, MAP_JC),
      GBFFT_TK(12, 4, false, true, MAP_JC),
      GBFFT_TK(13, 1, false, true, MAP_JC),
      GBFFT_TK(13, 2, false, true, MAP_JC),
      GBFFT_TK(14, 1, false, true, MAP_JC),
  };
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

}  // namespace gbfft
