// many.cu -- uneven-length batches (placeholder until the persistent kernel lands).
#include "gbfft_internal.h"

namespace gbfft {
struct ManyPlan {};
int many_plan_init(fft_plan*, const int64_t*, int64_t) { return FFT_ERR_UNSUPPORTED; }
void many_plan_free(fft_plan* p) { delete p->many; p->many = nullptr; }
int many_exec(fft_plan*, const float2*, float2*, int, cudaStream_t) { return FFT_ERR_UNSUPPORTED; }
}  // namespace gbfft
