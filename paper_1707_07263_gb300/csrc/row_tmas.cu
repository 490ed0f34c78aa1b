// row_tmas.cu -- the last (row) pass of the multi-pass 1-D plans with its
// output written by tensor TMA.
//
// A row pass reads C contiguous rows of L points (rows g*C + c of the
// workspace) and writes output k of row c to X[(g*C + c) + ncols*k]: C
// adjacent elements at a stride of ncols, i.e. a C x L box of the output
// viewed as a matrix of ncols columns and batch*L rows.  Stored from
// registers, that is R scalar 8-byte stores per thread into runs of only C
// elements (32 bytes at C = 4), and the global store queue becomes the
// binding stall (ncu at 2^20 = 2^8 x 2^12: `lg_throttle` the top stall).
// Here the last pass leaves the scaled outputs as a dense [k][c] tile in
// shared memory (tile_fft.cuh, last-pass mode 7) and one thread stores the
// tile with L/256 tensor-TMA copies of C x 256 boxes; the CTA waits for the
// copies to have read shared memory before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gbfft_internal.h"
#include "tile_fft.cuh"
#include "tile_registry.h"

namespace gbfft {

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
}

template <int LG, int C>
__global__ void __launch_bounds__(TileCfg<LG, C, false, true>::T)
    row_tmas_kernel(const __grid_constant__ CUtensorMap omap, const TileArgs a) {
  static_assert((1 << LG) >= 256 && (C % 2) == 0, "boxes of C x 256 elements, 16-byte rows");
  constexpr int L = 1 << LG;
  extern __shared__ __align__(128) float2 rt_smem[];
  const long long tile = blockIdx.x;
  tile_body<LG, C, false, true, false, 0, 7>(a, tile, rt_smem);
  // the dense [k][c] tile is complete (mode 7 ends with a barrier)
  if (threadIdx.x == 0) {
    const long long b = tile / a.tiles_per_batch;
    const long long g = tile - b * a.tiles_per_batch;
    fence_proxy_async();   // generic-proxy writes of the tile before the async-proxy reads
#pragma unroll 1
    for (int i = 0; i < L / 256; ++i)
      tma_store_2d(&omap, (int)(g * C), (int)(b * L + i * 256), rt_smem + (long long)i * 256 * C);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  }
}

#define GBFFT_ROWTMAS(LG, C) \
  {(const void*)&row_tmas_kernel<LG, C>, TileCfg<LG, C, false, true>::T, TileCfg<LG, C, false, true>::SMEM_BYTES, \
   LG, C, MAP_JC}

// Rows of 2^10 and 2^11 points, four per CTA (256 / 512 threads), and of
// 2^10 with eight (512 threads), where the plain store path is queue-bound.
// Measured per 2^26 points against it: 2^18 = 2^8 x 2^10 373.8 -> 335.5 us,
// 2^19 398.0 -> 365.2, 2^21 = 2^10 x 2^11 482.0 -> 449.2, the transposed 2-D
// 1024 x 1024 plan 411 -> 388.  Not compiled where it did not pay: every
// 1024-thread tile (rows of 2^11 with eight, 2^12 with four, 2^13 with two:
// one CTA per SM idles while its stores drain; 2^20 as 2^8 x 2^12 435.9 ->
// 442.0 us, 2048^2 506 -> 536, 4096^2 543 -> 564) and the 16-row tiles of 2^8
// / 2^9 (64- and 128-byte runs, no change).
const TileKernelInfo* tile_kernel_rowtmas(int lg, int C) {
  static const TileKernelInfo tab[] = {GBFFT_ROWTMAS(10, 4), GBFFT_ROWTMAS(11, 4), GBFFT_ROWTMAS(10, 8)};
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn_rt() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    cudaGetLastError();
  });
  return fn;
}

// The pass writes X[(g*C + c) + ncols*k] of batch b at b * L * ncols: dense
// rows of ncols columns, 16-byte aligned, no filter, no outer batch.
// (TMA coordinates are 32-bit: at most 2^31 output rows.)
bool rowtmas_usable(const TileKernelInfo* k, const TileArgs& a, const void* out, long long ntiles) {
  if (!k || !encode_fn_rt() || ((uintptr_t)out & 15) || a.tiles_per_batch < 1) return false;
  const long long L = 1LL << k->lg;
  return a.out_sc == 1 && a.out_gstride == k->C && a.out_sn == a.ncols && a.out_bstride == L * a.ncols &&
         (a.ncols & 1) == 0 && a.tiles_per_batch * k->C == a.ncols && !a.filt && !a.nb1 && !a.col_off &&
         ntiles % a.tiles_per_batch == 0 && (ntiles / a.tiles_per_batch) * L < 0x7fffffffLL;
}

int rowtmas_launch(const TileKernelInfo* k, const TileArgs& a, long long ntiles, cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn_rt();
  if (!enc) return FFT_ERR_UNSUPPORTED;
  if (ntiles <= 0) return FFT_OK;
  if (ntiles > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
  const long long L = 1LL << k->lg;
  const long long batches = ntiles / a.tiles_per_batch;
  const cuuint64_t dims[2] = {(cuuint64_t)a.ncols, (cuuint64_t)(batches * L)};
  const cuuint64_t strides[1] = {(cuuint64_t)a.ncols * 8};
  const cuuint32_t box[2] = {(cuuint32_t)k->C, 256};
  const cuuint32_t estr[2] = {1, 1};
  CUtensorMap map;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)a.out, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return FFT_ERR_UNSUPPORTED;
  void* args[] = {(void*)&map, (void*)&a};
  return cudaLaunchKernel(k->fn, dim3((unsigned)ntiles), dim3(k->threads), args, (size_t)k->smem_bytes, s) ==
                 cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace gbfft
