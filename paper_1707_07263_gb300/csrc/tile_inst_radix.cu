// tile_inst_radix.cu -- compiled batched single-pass variants (contiguous in
// and out, jj_cols(lg) transforms per CTA) whose Stockham passes use a smaller
// largest radix: radix-8 passes with 8 points per thread (2^5..2^13) and
// radix-4 passes with 4 points per thread (2^5..2^12).  With the same tile,
// the CTA has 2x / 4x the threads of the radix-16 kernel.  These are the
// autotuner's radix, points-per-thread and threads-per-CTA choices for one
// on-chip pass (the paper fixes radix 2 and one thread per butterfly,
// Sec. 2.3.3).
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_TKR(LG, LGM)                                                                         \
  {(const void*)&tile_fft_kernel<LG, jj_cols(LG), false, false, LGM>,                              \
   TileCfg<LG, jj_cols(LG), false, false, 0, LGM>::T, TileCfg<LG, jj_cols(LG), false, false, 0, LGM>::SMEM_BYTES, \
   LG, jj_cols(LG), MAP_JJ}

const TileKernelInfo* tile_kernel_radix(int lg, int lgm) {
  static const TileKernelInfo r8[] = {
      GBFFT_TKR(5, 3),  GBFFT_TKR(6, 3),  GBFFT_TKR(7, 3),  GBFFT_TKR(8, 3), GBFFT_TKR(9, 3),
      GBFFT_TKR(10, 3), GBFFT_TKR(11, 3), GBFFT_TKR(12, 3), GBFFT_TKR(13, 3),
  };
  static const TileKernelInfo r4[] = {
      GBFFT_TKR(5, 2),  GBFFT_TKR(6, 2),  GBFFT_TKR(7, 2),  GBFFT_TKR(8, 2),
      GBFFT_TKR(9, 2),  GBFFT_TKR(10, 2), GBFFT_TKR(11, 2), GBFFT_TKR(12, 2),
  };
  if (lgm == 3 && lg >= 5 && lg <= 13) return &r8[lg - 5];
  if (lgm == 2 && lg >= 5 && lg <= 12) return &r4[lg - 5];
  return nullptr;
}

}  // namespace gbfft
