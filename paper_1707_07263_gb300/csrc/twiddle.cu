// twiddle.cu -- device-side generation of the twiddle look-up tables
// (paper Sec. 2.3.1: the sine/cosine values are computed once, before the FFT,
// and kept in a table the butterflies read).  Every entry is evaluated in FP64
// with sincospi of -2m/M, the exponent m reduced mod M first (Eq. 3), and
// rounded once to FP32 (kept in FP64 for FP64 transforms).  For M a power of
// two the argument -2m/M is exact; for the mixed-radix lengths it carries one
// FP64 rounding (relative 2^-53), far below either table precision.
#include <cuda_runtime.h>

#include "gbfft_internal.h"
#include "tile_fft.cuh"

namespace gbfft {

__device__ __forceinline__ float2 w_entry(long long m, long long M) {
  m %= M;
  double s, c;
  sincospi(-2.0 * (double)m / (double)M, &s, &c);
  return make_float2((float)c, (float)s);
}

// Stage table of length L = 2^lg: for pass s with Ns > 1, row e, column k
// holds W_{Ns*R}^{2^e * k} at stage_tw_off(lg, s, rev, lgm) + e*Ns + k (rev:
// the remainder-last schedule; lgm: log2 of the largest radix).
__global__ void gen_stage_twiddles(float2* tab, int lg, bool rev, int lgm) {
  const int total = stage_tw_size(lg, rev, lgm);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int s = 1;
    while (s + 1 < radix_nst(lg, lgm) && idx >= stage_tw_off(lg, s + 1, rev, lgm)) ++s;
    const int local = idx - stage_tw_off(lg, s, rev, lgm);
    const int lgns = radix_lgns(lg, s, rev, lgm), lgr = radix_lgr(lg, s, rev, lgm);
    const int NS = 1 << lgns;
    const int e = local / NS, k = local % NS;
    const long long M = 1LL << (lgns + lgr);
    tab[idx] = w_entry((1LL << e) * (long long)k, M);
  }
}

// tab[i] = W_N^{i * step}, i < count, N = 2^lgN.
__global__ void gen_power_twiddles(float2* tab, int lgN, long long count, long long step) {
  const long long N = 1LL << lgN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    tab[i] = w_entry((i * step) % N, N);
}

// tab[m] = W_N^m, m < count, for any N (mixed-radix lengths).
__global__ void gen_twiddles_n(float2* tab, long long N, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    tab[i] = w_entry(i % N, N);
}

cudaError_t launch_gen_twiddles_n(float2* tab, long long N, long long count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const long long blocks = (count + 255) / 256;
  gen_twiddles_n<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(tab, N, count);
  return cudaGetLastError();
}

// tab[m] = W_N^m in FP64, m < count (FP64 transforms).
__global__ void gen_twiddles_n64(double2* tab, long long N, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)(i % N) / (double)N, &sn, &cs);
    tab[i] = make_double2(cs, sn);
  }
}

cudaError_t launch_gen_twiddles_n64(double2* tab, long long N, long long count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const long long blocks = (count + 255) / 256;
  gen_twiddles_n64<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(tab, N, count);
  return cudaGetLastError();
}

// tab[i] = W_N^{(i * step) mod N}, i < count, for any N (the strided
// mixed-radix plans: sub-length tables with step 1, and the high level of a
// two-level four-step table with step 2^s); FP64 entries, or rounded once to
// FP32.
template <typename T>
__global__ void gen_twiddles_step(T* tab, long long N, long long count, long long step) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)((i * step) % N) / (double)N, &sn, &cs);
    if constexpr (sizeof(T) == 16)
      tab[i] = make_double2(cs, sn);
    else
      tab[i] = make_float2((float)cs, (float)sn);
  }
}

cudaError_t launch_gen_twiddles_step(void* tab, bool fp64, long long N, long long count, long long step,
                                     cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const long long blocks = (count + 255) / 256;
  const unsigned g = (unsigned)(blocks < 4096 ? blocks : 4096);
  if (fp64)
    gen_twiddles_step<double2><<<g, 256, 0, s>>>((double2*)tab, N, count, step);
  else
    gen_twiddles_step<float2><<<g, 256, 0, s>>>((float2*)tab, N, count, step);
  return cudaGetLastError();
}

cudaError_t launch_gen_stage_twiddles(float2* tab, int lg, cudaStream_t s, bool rev, int lgm) {
  const int total = stage_tw_size(lg, rev, lgm);
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const int blocks = (total + threads - 1) / threads;
  gen_stage_twiddles<<<blocks, threads, 0, s>>>(tab, lg, rev, lgm);
  return cudaGetLastError();
}

cudaError_t launch_gen_power_twiddles(float2* tab, int lgN, long long count, long long step, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int threads = 256;
  const long long blocks = (count + threads - 1) / threads;
  gen_power_twiddles<<<(unsigned)(blocks < 4096 ? blocks : 4096), threads, 0, s>>>(tab, lgN, count, step);
  return cudaGetLastError();
}

}  // namespace gbfft
