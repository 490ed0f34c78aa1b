// mixed4_ct.cu -- the strided mixed-radix pass (mixed4.cuh) with the
// sub-length, its radix schedule and the columns per CTA fixed at compile
// time, for the sub-lengths that the two-pass FP32 plans meet most (FP32).
//
// Same recurrence, layout and thread mapping as the run-time kernel: a tile
// of C = 2^CSH adjacent columns of length L, threads column-fastest, element
// (c, n) in shared memory at sidx(n) * C + c with one pad row every 16.  The
// radices are the composite register radices of mixed_ct.cuh (up to 25
// points as Cooley-Tukey splits inside the register file), two or three
// passes per sub-transform, so L, every radix, Ns and every divisor are
// template parameters and the index arithmetic folds.  The last pass applies
// the four-step twiddle W_Nt^{col k} (two table entries) when the plan has
// one, and the output scale.
#include <cuda_runtime.h>

#include "gbfft_internal.h"
#include "mixed_ct.cuh"

namespace gbfft {

template <int L, int R, int NS, int CSH, bool FIRST, bool LAST>
__device__ __forceinline__ void m4ct_pass(const Mixed4Args& a, const float2* gin, const float2* src, float2* dst,
                                          float2* gout, long long col0, int valid) {
  constexpr int C = 1 << CSH;
  constexpr int NB = L / R;
  constexpr int STRIDE = L / (NS * R);
  static_assert(L % (NS * R) == 0, "schedule");
  const MixedArgs& m = a.m;
  const float2* tw = (const float2*)m.tw;
  const float2* ft_lo = (const float2*)a.ft_lo;
  const float2* ft_hi = (const float2*)a.ft_hi;
  const unsigned long long ft_mask = (1ULL << a.ft_s) - 1ULL;
  for (int b = threadIdx.x; b < (NB << CSH); b += blockDim.x) {
    const int c = b & (C - 1), j = b >> CSH;
    const bool ok = c < valid;
    float2 v[R];
    if constexpr (FIRST) {
      const float2* p = gin + c * a.in_cs + (long long)j * a.in_ns;
      const long long step = (long long)NB * a.in_ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = ok ? __ldcs(p + r * step) : make_float2(0.f, 0.f);
      if (m.conj_in) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = src[msidx<true>(j + r * NB) * C + c];
    }
    const int jq = j / NS, k = j - jq * NS;
    if constexpr (NS > 1) ct_twiddles<R>(v, tw, k * STRIDE);
    ct_dft<R>(v);
    const int m0 = jq * NS * R + k;
    if constexpr (LAST) {
      if (!ok) continue;
      const unsigned long long col = (unsigned long long)(col0 + c);
      float2* p = gout + c * a.out_cs + (long long)m0 * a.out_ns;
      const long long step = (long long)NS * a.out_ns;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        float2 y = v[q];
        if (ft_lo) {
          const unsigned long long e = col * (unsigned long long)(m0 + q * NS);
          y = cmul(y, cmul(__ldg(ft_lo + (e & ft_mask)), __ldg(ft_hi + (e >> a.ft_s))));
        }
        if (m.scale_out) y = make_float2(y.x * m.fsx, y.y * m.fsy);
        __stcs(p + q * step, y);
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) dst[msidx<true>(m0 + q * NS) * C + c] = v[q];
    }
  }
}

// Two passes (R2 == 1) or three.
template <int L, int R0, int R1, int R2, int CSH>
__global__ void __launch_bounds__(256, 2) mixed4_ct_kernel(const Mixed4Args a) {
  static_assert(R0 * R1 * R2 == L, "schedule");
  constexpr int C = 1 << CSH;
  extern __shared__ __align__(16) unsigned char m4ct_smem[];
  float2* const buf0 = (float2*)m4ct_smem;
  float2* const buf1 = buf0 + (msidx<true>(L - 1) + 1) * C;
  for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const long long bt = t / a.tiles_per_batch;
    const long long col0 = (t - bt * a.tiles_per_batch) * C;
    const int valid = (int)(a.ncols - col0 < C ? a.ncols - col0 : C);
    const float2* gin = (const float2*)a.m.in + bt * a.in_bs + col0 * a.in_cs;
    float2* gout = (float2*)a.m.out + bt * a.out_bs + col0 * a.out_cs;
    m4ct_pass<L, R0, 1, CSH, true, false>(a, gin, nullptr, buf0, gout, col0, valid);
    __syncthreads();
    if constexpr (R2 == 1) {
      m4ct_pass<L, R1, R0, CSH, false, true>(a, gin, buf0, nullptr, gout, col0, valid);
    } else {
      m4ct_pass<L, R1, R0, CSH, false, false>(a, gin, buf0, buf1, gout, col0, valid);
      __syncthreads();
      m4ct_pass<L, R2, R0 * R1, CSH, false, true>(a, gin, buf1, nullptr, gout, col0, valid);
    }
    __syncthreads();
  }
}

// Sub-length, schedule (radix 25 or the largest first, as for the one-pass
// compiled schedules), columns per CTA (a tile of about 2048..4096 points,
// at most 16).
#define GBFFT_M4CT(L, R0, R1, R2, CSH) {L, R0, R1, R2, CSH, (const void*)&mixed4_ct_kernel<L, R0, R1, R2, CSH>}

const Mixed4CtInfo* mixed4_ct_lookup(long long L) {
  static const Mixed4CtInfo tab[] = {
      GBFFT_M4CT(64, 16, 4, 1, 4),      GBFFT_M4CT(100, 25, 4, 1, 4),    GBFFT_M4CT(120, 15, 8, 1, 4),
      GBFFT_M4CT(125, 25, 5, 1, 4),     GBFFT_M4CT(128, 16, 8, 1, 4),    GBFFT_M4CT(160, 16, 10, 1, 4),
      GBFFT_M4CT(200, 25, 8, 1, 4),     GBFFT_M4CT(240, 16, 15, 1, 4),   GBFFT_M4CT(250, 25, 10, 1, 4),
      GBFFT_M4CT(256, 16, 16, 1, 4),    GBFFT_M4CT(320, 20, 16, 1, 3),   GBFFT_M4CT(400, 25, 16, 1, 3),
      GBFFT_M4CT(500, 25, 20, 1, 3),    GBFFT_M4CT(512, 16, 8, 4, 3),    GBFFT_M4CT(625, 25, 25, 1, 2),
      GBFFT_M4CT(1000, 25, 8, 5, 2),    GBFFT_M4CT(1024, 16, 16, 4, 2),  GBFFT_M4CT(1250, 25, 10, 5, 1),
      GBFFT_M4CT(2000, 25, 16, 5, 1),   GBFFT_M4CT(2048, 16, 16, 8, 1),  GBFFT_M4CT(2500, 25, 10, 10, 0),
      GBFFT_M4CT(3125, 25, 25, 5, 0),   GBFFT_M4CT(4000, 25, 16, 10, 0), GBFFT_M4CT(4096, 16, 16, 16, 0),
  };
  for (const Mixed4CtInfo& t : tab)
    if (t.L == L) return &t;
  return nullptr;
}

}  // namespace gbfft
