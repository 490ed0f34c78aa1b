// tc_inst_bf16s.cu -- tensor-core tile-FFT variants, precision code 3 (bf16s).
#include "tc_fft.cuh"
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_TC(LG, C, ICF, OCF, MAP, PREC) \
  {(const void*)&tc_fft_kernel<LG, C, ICF, OCF, PREC>, TileCfg<LG, C, ICF, OCF, 1>::T, \
   TileCfg<LG, C, ICF, OCF, 1>::SMEM_BYTES, LG, C, MAP}

const TileKernelInfo* tc_kernel_bf16s(int map, int lg, int C) {
  static const TileKernelInfo tab[] = {
      GBFFT_TC(8, jj_cols(8), false, false, MAP_JJ, 3),
      GBFFT_TC(10, jj_cols(10), false, false, MAP_JJ, 3),
      GBFFT_TC(12, jj_cols(12), false, false, MAP_JJ, 3),
      GBFFT_TC(8, 16, true, true, MAP_CC, 3),
      GBFFT_TC(8, 16, false, true, MAP_JC, 3),
      GBFFT_TC(10, 8, true, true, MAP_CC, 3),
      GBFFT_TC(10, 8, false, true, MAP_JC, 3),
      GBFFT_TC(12, 2, true, true, MAP_CC, 3),
      GBFFT_TC(12, 2, false, true, MAP_JC, 3),
  };
  for (const TileKernelInfo& k : tab)
    if (k.map == map && k.lg == lg && k.C == C) return &k;
  return nullptr;
}

}  // namespace gbfft
