// tile_inst_jj.cu -- compiled batched single-pass tile-FFT variants (contiguous in and out),
// one per length 2^1..2^14 with jj_cols(lg) transforms per CTA.
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tile_kernel_jj(int lg) {
  static const TileKernelInfo tab[] = {
      GBFFT_TK(1, jj_cols(1), false, false, MAP_JJ),
      GBFFT_TK(2, jj_cols(2), false, false, MAP_JJ),
      GBFFT_TK(3, jj_cols(3), false, false, MAP_JJ),
      GBFFT_TK(4, jj_cols(4), false, false, MAP_JJ),
      GBFFT_TK(5, jj_cols(5), false, false, MAP_JJ),
      GBFFT_TK(6, jj_cols(6), false, false, MAP_JJ),
      GBFFT_TK(7, jj_cols(7), false, false, MAP_JJ),
      GBFFT_TK(8, jj_cols(8), false, false, MAP_JJ),
      GBFFT_TK(9, jj_cols(9), false, false, MAP_JJ),
      GBFFT_TK(10, jj_cols(10), false, false, MAP_JJ),
      GBFFT_TK(11, jj_cols(11), false, false, MAP_JJ),
      GBFFT_TK(12, jj_cols(12), false, false, MAP_JJ),
      GBFFT_TK(13, jj_cols(13), false, false, MAP_JJ),
      GBFFT_TK(14, jj_cols(14), false, false, MAP_JJ),
  };
  if (lg < 1 || lg > 14) return nullptr;
  return &tab[lg - 1];
}

}  // namespace gbfft
