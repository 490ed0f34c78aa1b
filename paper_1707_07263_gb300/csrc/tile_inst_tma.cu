// tile_inst_tma.cu -- compiled persistent TMA-staged batched tile-FFT variants,
// one per length 2^1..2^14 (jj_cols(lg) transforms per tile).
#include "tile_fft_tma.cuh"
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_TMA(LG)                                                                                       \
  {(const void*)&tile_fft_tma_kernel<LG, jj_cols(LG), tma_exchange_width(LG)>,                              \
   TmaCfg<LG, jj_cols(LG), tma_exchange_width(LG)>::T, TmaCfg<LG, jj_cols(LG), tma_exchange_width(LG)>::SMEM_BYTES, \
   LG, jj_cols(LG), MAP_JJ}

const TileKernelInfo* tile_kernel_tma(int lg) {
  static const TileKernelInfo tab[] = {
      GBFFT_TMA(1),  GBFFT_TMA(2),  GBFFT_TMA(3),  GBFFT_TMA(4),  GBFFT_TMA(5),  GBFFT_TMA(6),  GBFFT_TMA(7),
      GBFFT_TMA(8),  GBFFT_TMA(9),  GBFFT_TMA(10), GBFFT_TMA(11), GBFFT_TMA(12), GBFFT_TMA(13), GBFFT_TMA(14),
  };
  if (lg < 1 || lg > 14) return nullptr;
  return &tab[lg - 1];
}

}  // namespace gbfft
