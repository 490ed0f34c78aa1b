// mixed_ct.cu -- mixed-radix transforms (N = 2^a 3^b 5^c) with the radix
// schedule fixed at compile time for common lengths, in three passes of
// composite register radices.
//
// The run-time kernel (mixed.cu) takes one pass per prime factor or radix-16
// block: N = 1000 = 8*5*5*5 costs four passes, 12000 seven, each a round trip
// through shared memory plus run-time index divisions.  Sec. 2.1's split
// holds for any factorisation, so here N = R0 * R1 * R2 with composite
// radices of 10..25 points kept in registers (a radix R = A * B is itself a
// Cooley-Tukey split: A-point DFTs, the inner twiddles W_R^{n2 k1} as
// compile-time constants, B-point DFTs).  Every length below takes three
// passes, two exchanges through shared memory; N, the radices and every
// divisor are template parameters, so the index arithmetic folds to
// multiplications and shifts.
//
// Passes follow the same Stockham recurrence as mixed.cu (natural order in
// and out): butterfly j of a pass with radix R and Ns = the product of the
// earlier radices reads a[j + r N/R], multiplies by W_{Ns R}^{r (j mod Ns)}
// (powers of one W_N table entry), runs the R-point DFT and writes
// b[(j div Ns) Ns R + (j mod Ns) + q Ns].  FP32 only; other lengths, and
// FP64, take the run-time kernel.
#include <cuda_runtime.h>

#include "gbfft_internal.h"
#include "mixed_ct.cuh"

namespace gbfft {

// One pass over the tile's C transforms: radix R, Ns = NS.
template <int N, int R, int NS, bool PAD, bool FIRST, bool LAST>
__device__ __forceinline__ void ct_pass(const MixedArgs& a, const float2* src, float2* dst, long long col0) {
  constexpr int NB = N / R;
  constexpr int STRIDE = N / (NS * R);
  static_assert(N % (NS * R) == 0, "schedule");
  const float2* tw = (const float2*)a.tw;
  const int total = a.C * NB;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int c = b / NB, j = b - c * NB;
    const bool ok = col0 + c < a.batch;
    float2 v[R];
    const int n0 = c * N + j;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if constexpr (FIRST)
        v[r] = ok ? __ldcs(src + n0 + r * NB) : make_float2(0.f, 0.f);
      else
        v[r] = src[msidx<PAD>(n0 + r * NB)];
    }
    if (FIRST && a.conj_in) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
    }
    const int jq = j / NS, k = j - jq * NS;
    if constexpr (NS > 1) ct_twiddles<R>(v, tw, k * STRIDE);
    ct_dft<R>(v);
    const int m0 = c * N + jq * NS * R + k;
    if constexpr (LAST) {
      if (!ok) continue;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        float2 y = v[q];
        if (a.scale_out) y = make_float2(y.x * a.fsx, y.y * a.fsy);
        __stcs(dst + m0 + q * NS, y);
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) dst[msidx<PAD>(m0 + q * NS)] = v[q];
    }
  }
}

// The tile of C transforms: three passes R0, R1, R2 (in == out is safe: the
// first pass reads the whole tile into shared memory before the last writes).
template <int N, int R0, int R1, int R2, bool PAD, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS <= 256 ? 2 : 1) mixed_ct_kernel(const MixedArgs a) {
  static_assert(R0 * R1 * R2 == N, "schedule");
  extern __shared__ __align__(16) unsigned char ct_smem[];
  float2* const buf0 = (float2*)ct_smem;
  float2* const buf1 = buf0 + msidx<PAD>(a.C * N - 1) + 1;
  const long long col0 = (long long)blockIdx.x * a.C;
  const float2* in = (const float2*)a.in + col0 * N;
  float2* out = (float2*)a.out + col0 * N;
  ct_pass<N, R0, 1, PAD, true, false>(a, in, buf0, col0);
  __syncthreads();
  ct_pass<N, R1, R0, PAD, false, false>(a, buf0, buf1, col0);
  __syncthreads();
  ct_pass<N, R2, R0 * R1, PAD, false, true>(a, buf1, out, col0);
}

// Compiled schedules, each the fastest of the orders and factorisations
// measured on GB300 for its length (radix 25 first, then 8 or 16; e.g.
// N = 1000: [25, 8, 5] 203 us against 312 for [10, 10, 10] and 420 for the
// run-time kernel's [8, 5, 5, 5], per 2^26 points), the transforms per CTA,
// C = floor(4096 / N) as for the run-time kernel, and the threads per CTA
// (512 where one CTA fills an SM's shared memory, 8000 and up: 12000 350 -> 324
// us; 256 below, where two or three CTAs share an SM).
// (Tiles chosen instead to spread every pass's butterflies evenly over the
// threads -- N = 1000: 5 transforms, 3000: 2 -- measured slower: the larger
// tiles cost resident CTAs.)  The padded layout where the first pass writes at
// an even stride.
#define GBFFT_CT(N, R0, R1, R2, C, T) \
  {N, R0, R1, R2, C, T, (R0 % 2 == 0), (const void*)&mixed_ct_kernel<N, R0, R1, R2, (R0 % 2 == 0), T>}

const MixedCtInfo* mixed_ct_lookup(long long N) {
  static const MixedCtInfo tab[] = {
      GBFFT_CT(1000, 25, 8, 5, 4, 256),    GBFFT_CT(1200, 25, 16, 3, 3, 256),   GBFFT_CT(1500, 25, 12, 5, 2, 256),
      GBFFT_CT(2000, 25, 16, 5, 2, 256),   GBFFT_CT(2400, 25, 8, 12, 1, 256),   GBFFT_CT(3000, 25, 8, 15, 1, 256),
      GBFFT_CT(4000, 25, 16, 10, 1, 256),  GBFFT_CT(5000, 25, 8, 25, 1, 256),   GBFFT_CT(6000, 25, 16, 15, 1, 256),
      GBFFT_CT(8000, 25, 16, 20, 1, 512),  GBFFT_CT(10000, 25, 16, 25, 1, 512), GBFFT_CT(12000, 25, 24, 20, 1, 512),
  };
  for (const MixedCtInfo& t : tab)
    if (t.N == N) return &t;
  return nullptr;
}

}  // namespace gbfft
