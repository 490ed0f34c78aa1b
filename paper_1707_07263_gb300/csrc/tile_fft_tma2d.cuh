// tile_fft_tma2d.cuh -- persistent column-pass kernel staged by tensor TMA.
//
// The column passes of the multi-pass plans (four-step pass 1, the first two
// passes of the three-pass split, the 2-D column passes) read C adjacent
// columns of L rows that lie far apart in memory.  Here each CTA loops over
// tiles; one thread issues cp.async.bulk.tensor for the C x L box of the next
// tile (a 4-D tensor map: columns, rows, inner batch, outer batch) into a
// staging buffer while the CTA computes the current one, completion on an
// mbarrier with a bounded wait.  The first pass reads the staged box [n][c]
// from shared memory; the remaining passes, the four-step twiddle and the
// stores are those of tile_fft.cuh.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tile_fft_tma.cuh"

namespace gbfft {

template <int LG, int C>
struct ColTmaCfg {
  using Tile = TileCfg<LG, C, true, true>;
  static constexpr int L = Tile::L;
  static constexpr int T = Tile::T;
  static constexpr int S_ELEMS = C * L;  // staged box
  static constexpr int SMEM_BYTES = S_ELEMS * 8 + Tile::SMEM_BYTES;
  static constexpr int MIN_BLOCKS = T <= 256 ? 3 : 1;
};

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint32_t bytes, uint64_t* mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(mbar))
      : "memory");
}

template <int LG, int C>
__global__ void __launch_bounds__(ColTmaCfg<LG, C>::T, ColTmaCfg<LG, C>::MIN_BLOCKS)
    col_tma_kernel(const __grid_constant__ CUtensorMap tmap, const TileArgs a, long long ntiles, int* status) {
  using Cfg = ColTmaCfg<LG, C>;
  using Tile = typename Cfg::Tile;
  static_assert(Tile::NST >= 2, "the staged pass is followed by at least one more");
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  float2* S = (float2*)smraw;
  float2* X = S + Cfg::S_ELEMS;
  float2* epi = X + Tile::SM_TILE;
  const int tid = threadIdx.x;

  auto split = [&](long long t, long long& b2, long long& b, long long& g) {
    b = t / a.tiles_per_batch;
    g = t - b * a.tiles_per_batch;
    b2 = 0;
    if (a.nb1) {
      b2 = b / a.nb1;
      b -= b2 * a.nb1;
    }
  };
  auto issue = [&](long long t) {
    long long b2, b, g;
    split(t, b2, b, g);
    tma_load_4d(S, &tmap, (int)(g * C), 0, (int)b, (int)b2, (uint32_t)(Cfg::S_ELEMS * 8), &mbar);
  };

  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  long long tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue(tile);
  uint32_t parity = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    long long b2, b, g;
    split(tile, b2, b, g);
    const long long col0 = g * C;
    float2* gout = a.out + b2 * a.out_b2stride + b * a.out_bstride + g * a.out_gstride;
    __syncthreads();  // the previous tile's last pass has finished reading X and epi
    if (a.ft_lgN) {
      constexpr int NS_LAST = 1 << radix_lgns(LG, Tile::NST - 1);
      for (int e = tid; e < C * 16; e += Cfg::T) {
        const int q = e / C, c = e - q * C;   // entry q*C + c (q-major, as tile_pass reads it)
        const unsigned n2 = a.ft_by_batch ? (unsigned)b : (unsigned)(col0 + c);
        const unsigned m = (n2 * (unsigned)NS_LAST * (unsigned)q) & ((1u << a.ft_lgN) - 1u);
        const unsigned mask = (1u << a.ft_s) - 1u;
        epi[e] = cmul(__ldg(a.ft_lo + (m & mask)), __ldg(a.ft_hi + (m >> a.ft_s)));
      }
    }
    if (!mbar_wait(&mbar, parity)) {
      if (tid == 0) atomicExch(status, FFT_ERR_TIMEOUT);
      mbar_wait(&mbar, parity);  // second bounded wait for the copy in flight
      return;
    }
    parity ^= 1u;
    float2 v[Tile::P];
    // pass 0 from the staged box; its closing barrier frees the staging buffer
    tile_pass<LG, C, true, true, 0, false, 2>(v, X, a, S, gout, col0, b, epi);
    if (tid == 0 && tile + gridDim.x < ntiles) {
      fence_proxy_async();
      issue(tile + gridDim.x);
    }
    tile_stage<LG, C, true, true, 1, false, 0>(v, X, a, S, gout, col0, b, epi);
  }
}

}  // namespace gbfft
