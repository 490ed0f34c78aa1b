// mixed4_f64.cu -- FP64 (complex128) instances of the strided mixed-radix
// pass (mixed4.cuh): 1..8 columns per CTA, padded shared-memory index, and
// the unpadded one-column form for sub-lengths whose padded buffers do not
// fit.  256 threads, up to two CTAs per SM (128 registers: a radix-16
// butterfly holds 16 complex128 values).
#include <cuda_runtime.h>

#include "mixed4.cuh"

namespace gbfft {

template <int CSH, bool PAD>
__global__ void __launch_bounds__(256, 2) mixed4_kernel64(const Mixed4Args a) {
  extern __shared__ __align__(16) unsigned char m4_smem64[];
  m4_tiles<double2, CSH, PAD>(a, (double2*)m4_smem64);
}

const void* mixed4_kernel_fn64(int csh, bool pad) {
  if (!pad) return csh == 0 ? (const void*)&mixed4_kernel64<0, false> : nullptr;
  switch (csh) {
    case 0: return (const void*)&mixed4_kernel64<0, true>;
    case 1: return (const void*)&mixed4_kernel64<1, true>;
    case 2: return (const void*)&mixed4_kernel64<2, true>;
    case 3: return (const void*)&mixed4_kernel64<3, true>;
    default: return nullptr;
  }
}

}  // namespace gbfft
