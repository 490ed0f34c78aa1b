// tile_inst_pf.cu -- compiled persistent single-pass kernels that fetch the
// next transform while computing one, lengths 2^12..2^14:
//   tile_fft_pf_kernel  (L2 prefetch; signature void(TileArgs, long long ntiles))
//   tile_fft_pfs_kernel (L2 prefetch and a bulk copy into the exchange buffer;
//                        signature void(TileArgs, long long ntiles, int* status))
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_PF(LG) \
  {(const void*)&tile_fft_pf_kernel<LG>, TileCfg<LG, 1, false, false>::T, TileCfg<LG, 1, false, false>::SMEM_BYTES, LG, 1, MAP_JJ}

const TileKernelInfo* tile_kernel_pf(int lg) {
  static const TileKernelInfo tab[] = {GBFFT_PF(12), GBFFT_PF(13), GBFFT_PF(14)};
  if (lg < 12 || lg > 14) return nullptr;
  return &tab[lg - 12];
}

#define GBFFT_PFS(LG) \
  {(const void*)&tile_fft_pfs_kernel<LG>, TileCfg<LG, 1, false, false>::T, pfs_smem_bytes<LG>(), LG, 1, MAP_JJ}

const TileKernelInfo* tile_kernel_pfs(int lg) {
  static const TileKernelInfo tab[] = {GBFFT_PFS(12), GBFFT_PFS(13), GBFFT_PFS(14)};
  if (lg < 12 || lg > 14) return nullptr;
  return &tab[lg - 12];
}

}  // namespace gbfft
