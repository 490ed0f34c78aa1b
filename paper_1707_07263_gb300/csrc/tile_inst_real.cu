// tile_inst_real.cu -- compiled fused real-to-complex and complex-to-real
// kernels, one per half length L = 2^1..2^14 (N = 2L reals) with
// jj_cols(lg) rows per CTA.
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_REAL(KERNEL, LG)                                                                 \
  {(const void*)&KERNEL<LG, jj_cols(LG)>, TileCfg<LG, jj_cols(LG), false, false>::T,           \
   jj_cols(LG) * TileCfg<LG, jj_cols(LG), false, false>::LP * 8, LG, jj_cols(LG), MAP_JJ}

const TileKernelInfo* tile_kernel_r2c(int lg) {
  static const TileKernelInfo tab[] = {
      GBFFT_REAL(tile_r2c_kernel, 1),  GBFFT_REAL(tile_r2c_kernel, 2),  GBFFT_REAL(tile_r2c_kernel, 3),
      GBFFT_REAL(tile_r2c_kernel, 4),  GBFFT_REAL(tile_r2c_kernel, 5),  GBFFT_REAL(tile_r2c_kernel, 6),
      GBFFT_REAL(tile_r2c_kernel, 7),  GBFFT_REAL(tile_r2c_kernel, 8),  GBFFT_REAL(tile_r2c_kernel, 9),
      GBFFT_REAL(tile_r2c_kernel, 10), GBFFT_REAL(tile_r2c_kernel, 11), GBFFT_REAL(tile_r2c_kernel, 12),
      GBFFT_REAL(tile_r2c_kernel, 13), GBFFT_REAL(tile_r2c_kernel, 14),
  };
  if (lg < 1 || lg > 14) return nullptr;
  return &tab[lg - 1];
}

const TileKernelInfo* tile_kernel_c2r(int lg) {
  static const TileKernelInfo tab[] = {
      GBFFT_REAL(tile_c2r_kernel, 1),  GBFFT_REAL(tile_c2r_kernel, 2),  GBFFT_REAL(tile_c2r_kernel, 3),
      GBFFT_REAL(tile_c2r_kernel, 4),  GBFFT_REAL(tile_c2r_kernel, 5),  GBFFT_REAL(tile_c2r_kernel, 6),
      GBFFT_REAL(tile_c2r_kernel, 7),  GBFFT_REAL(tile_c2r_kernel, 8),  GBFFT_REAL(tile_c2r_kernel, 9),
      GBFFT_REAL(tile_c2r_kernel, 10), GBFFT_REAL(tile_c2r_kernel, 11), GBFFT_REAL(tile_c2r_kernel, 12),
      GBFFT_REAL(tile_c2r_kernel, 13), GBFFT_REAL(tile_c2r_kernel, 14),
  };
  if (lg < 1 || lg > 14) return nullptr;
  return &tab[lg - 1];
}

}  // namespace gbfft
