// tile_registry.h -- lookup of the compiled tile-FFT kernel variants.
#pragma once
#include <cuda_runtime.h>

#include "tile_fft.cuh"

namespace gbfft {

// Thread mappings of the first / last pass (see tile_fft.cuh):
//   MAP_JJ: contiguous transforms in, contiguous out (batched single pass, 2-D rows)
//   MAP_CC: adjacent columns in and out (four-step column pass, 2-D columns)
//   MAP_JC: contiguous rows in, adjacent columns out (four-step row pass)
enum TileMap { MAP_JJ = 0, MAP_CC = 1, MAP_JC = 2 };

struct TileKernelInfo {
  const void* fn;   // __global__ void(TileArgs)
  int threads;      // CTA size
  int smem_bytes;   // dynamic shared memory
  int lg, C, map;
};

// Columns per CTA the JJ variant is compiled with for length 2^lg.
constexpr int jj_cols(int lg) { return lg >= 12 ? 1 : (lg >= 4 ? (4096 >> lg) : 256); }

// Persistent TMA-staged variant of MAP_JJ (tile_fft_tma.cuh), one per length;
// kernel signature void(TileArgs, long long ntiles, int* status).
const TileKernelInfo* tile_kernel_tma(int lg);
constexpr int tma_exchange_width(int lg) { return lg >= 13 ? 4 : 8; }

// Persistent tensor-TMA column kernels (tile_fft_tma2d.cuh), lengths 2^6..2^8.
const TileKernelInfo* tile_kernel_coltma(int lg, int C);
bool coltma_usable(const TileKernelInfo* k, const TileArgs& a, const void* in);
int coltma_launch(const TileKernelInfo* k, const TileArgs& a, long long ntiles, int grid, int* status,
                  cudaStream_t s);

// Row-pass kernels (MAP_JC) whose output tile is written by tensor TMA
// (row_tmas.cu), rows of 2^10 and 2^11 points, four per CTA; signature
// void(CUtensorMap, TileArgs).
const TileKernelInfo* tile_kernel_rowtmas(int lg, int C);
bool rowtmas_usable(const TileKernelInfo* k, const TileArgs& a, const void* out, long long ntiles);
int rowtmas_launch(const TileKernelInfo* k, const TileArgs& a, long long ntiles, cudaStream_t s);

// MAP_JJ single-pass variants with radix-8 (lgm = 3, 2^5..2^13) or radix-4
// (lgm = 2, 2^5..2^12) passes and as many points per thread, jj_cols(lg)
// transforms per CTA; NULL where not compiled.
const TileKernelInfo* tile_kernel_radix(int lg, int lgm);

// Two-CTA radix-2 split kernels (tile_fft_dif2_kernel) for half length 2^lg.
const TileKernelInfo* tile_kernel_dif2(int lg);

// Persistent single-pass kernels with an L2 prefetch of the next transform,
// lengths 2^12..2^14 (one transform per CTA); signature void(TileArgs, long long).
const TileKernelInfo* tile_kernel_pf(int lg);
// Persistent 2^12..2^14 kernels staging the next transform into the exchange
// buffer by a bulk copy (tile_fft_pfs_kernel); signature void(TileArgs, long long, int* status).
const TileKernelInfo* tile_kernel_pfs(int lg);

// Fused real-to-complex / complex-to-real kernels for half length 2^lg
// (N = 2^(lg+1) reals), 2^1..2^14, jj_cols(lg) rows per CTA.
const TileKernelInfo* tile_kernel_r2c(int lg);
const TileKernelInfo* tile_kernel_c2r(int lg);

// Fused range-compression kernels (tile_rc_kernel), lengths 2^1..2^14 with
// jj_cols(lg) rows per CTA.
const TileKernelInfo* tile_kernel_rc(int lg);

// Returns NULL when (map, lg, C) was not compiled.
const TileKernelInfo* tile_kernel(int map, int lg, int C);

// per-file tables (tile_inst_*.cu)
const TileKernelInfo* tile_kernel_jj(int lg);
const TileKernelInfo* tile_kernel_cc_a(int lg, int C);
const TileKernelInfo* tile_kernel_cc_b(int lg, int C);
const TileKernelInfo* tile_kernel_cc_c(int lg, int C);
const TileKernelInfo* tile_kernel_jc_a(int lg, int C);
const TileKernelInfo* tile_kernel_jc_b(int lg, int C);

#define GBFFT_TK(LG, C, ICF, OCF, MAP)                                                         \
  {(const void*)&tile_fft_kernel<LG, C, ICF, OCF>, TileCfg<LG, C, ICF, OCF>::T,                 \
   TileCfg<LG, C, ICF, OCF>::SMEM_BYTES, LG, C, MAP}

}  // namespace gbfft
