// hostmem.cu -- which pointers fft_exec may take: device memory of the
// current device, managed memory, or page-locked host memory that unified
// addressing maps into the device at the same address.  On a host whose CPU
// shares a coherent link with the GPU the kernels then transform host-resident
// data in place of a copy in and a copy out.
#include <cuda_runtime.h>

#include <cstdint>

#include "gbfft.h"

namespace gbfft {

int set_err(int code);

static int usable_at(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // an unknown pointer is an answer, not a sticky error
    return 0;
  }
  switch (a.type) {
    case cudaMemoryTypeDevice: {
      int dev = -1;
      if (cudaGetDevice(&dev) != cudaSuccess) return FFT_ERR_CUDA;
      return a.device == dev ? 1 : 0;
    }
    case cudaMemoryTypeManaged:
      return 1;
    case cudaMemoryTypeHost:
      return a.devicePointer == p ? 1 : 0;
    default:
      return 0;
  }
}

}  // namespace gbfft

extern "C" GBFFT_API int fft_pointer_usable(const void* ptr, size_t bytes) {
  using namespace gbfft;
  if (!ptr || bytes == 0) return set_err(FFT_ERR_INVALID_ARG);
  const int a = usable_at(ptr);
  if (a != 1) return a < 0 ? set_err(a) : 0;
  const int b = usable_at((const char*)ptr + (bytes - 1));
  if (b < 0) return set_err(b);
  return b;
}
