// mixed4_f32.cu -- FP32 (complex64) instances of the strided mixed-radix
// pass (mixed4.cuh): 1..16 columns per CTA, padded shared-memory index, and
// the unpadded one-column form for sub-lengths whose padded buffers do not
// fit.  256 threads, up to four CTAs per SM (64 registers).
#include <cuda_runtime.h>

#include "mixed4.cuh"

namespace gbfft {

template <int CSH, bool PAD>
__global__ void __launch_bounds__(256, 4) mixed4_kernel32(const Mixed4Args a) {
  extern __shared__ __align__(16) unsigned char m4_smem32[];
  m4_tiles<float2, CSH, PAD>(a, (float2*)m4_smem32);
}

const void* mixed4_kernel_fn32(int csh, bool pad) {
  if (!pad) return csh == 0 ? (const void*)&mixed4_kernel32<0, false> : nullptr;
  switch (csh) {
    case 0: return (const void*)&mixed4_kernel32<0, true>;
    case 1: return (const void*)&mixed4_kernel32<1, true>;
    case 2: return (const void*)&mixed4_kernel32<2, true>;
    case 3: return (const void*)&mixed4_kernel32<3, true>;
    case 4: return (const void*)&mixed4_kernel32<4, true>;
    default: return nullptr;
  }
}

}  // namespace gbfft
