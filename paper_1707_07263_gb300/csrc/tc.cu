// tc.cu -- tensor-core radix-16 passes (placeholder).
#include "gbfft_internal.h"

namespace gbfft {
int tc_plan_init(fft_plan*) { return FFT_ERR_UNSUPPORTED; }
int tc_exec(fft_plan*, const float2*, float2*, int, cudaStream_t) { return FFT_ERR_UNSUPPORTED; }
}  // namespace gbfft
