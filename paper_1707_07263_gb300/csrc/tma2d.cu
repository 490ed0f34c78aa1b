// tma2d.cu -- host side of the tensor-TMA column kernels: the tensor map for a
// column pass (encoded per exec, since it holds the data pointer) and the
// compiled variants.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gbfft_internal.h"
#include "tile_fft_tma2d.cuh"
#include "tile_registry.h"

namespace gbfft {

#define GBFFT_COLTMA(LG, C) \
  {(const void*)&col_tma_kernel<LG, C>, ColTmaCfg<LG, C>::T, ColTmaCfg<LG, C>::SMEM_BYTES, LG, C, MAP_CC}

const TileKernelInfo* tile_kernel_coltma(int lg, int C) {
  static const TileKernelInfo tab[] = {GBFFT_COLTMA(6, 16), GBFFT_COLTMA(6, 32), GBFFT_COLTMA(7, 8),
                                       GBFFT_COLTMA(7, 16), GBFFT_COLTMA(7, 32), GBFFT_COLTMA(8, 8),
                                       GBFFT_COLTMA(8, 16), GBFFT_COLTMA(8, 32)};
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg && k.C == C) return &k;
  return nullptr;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// Whether a column pass can be staged by tensor TMA: 16-byte aligned base,
// even element strides (16-byte row pitch), x = g*C a multiple of 2.
bool coltma_usable(const TileKernelInfo* k, const TileArgs& a, const void* in) {
  if (!k || !encode_fn()) return false;
  if (((uintptr_t)in & 15) || (a.in_sn & 1) || (a.in_bstride & 1) || (a.in_b2stride & 1)) return false;
  if (a.in_sc != 1 || a.in_gstride != k->C || (k->C & 1) || (1 << k->lg) > 256) return false;
  return true;
}

// Launch the persistent tensor-TMA column kernel for the pass described by a
// (a.in is the base of the tensor).  ntiles = tiles of the pass, grid =
// resident CTAs.
int coltma_launch(const TileKernelInfo* k, const TileArgs& a, long long ntiles, int grid, int* status,
                  cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return FFT_ERR_UNSUPPORTED;
  const long long nb_total = ntiles / a.tiles_per_batch;
  const long long nz = a.nb1 ? a.nb1 : nb_total;
  const long long nw = a.nb1 ? nb_total / a.nb1 : 1;
  const cuuint64_t dims[4] = {(cuuint64_t)a.ncols, (cuuint64_t)(1 << k->lg), (cuuint64_t)nz, (cuuint64_t)nw};
  const cuuint64_t zs = (cuuint64_t)a.in_bstride * 8;
  const cuuint64_t strides[3] = {(cuuint64_t)a.in_sn * 8, zs, a.nb1 ? (cuuint64_t)a.in_b2stride * 8 : zs * nz};
  const cuuint32_t box[4] = {(cuuint32_t)k->C, (cuuint32_t)(1 << k->lg), 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUtensorMap map;
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)a.in, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return FFT_ERR_UNSUPPORTED;
  const long long g = grid < ntiles ? grid : ntiles;
  void* args[] = {(void*)&map, (void*)&a, (void*)&ntiles, (void*)&status};
  return cudaLaunchKernel(k->fn, dim3((unsigned)g), dim3(k->threads), args, (size_t)k->smem_bytes, s) == cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace gbfft
