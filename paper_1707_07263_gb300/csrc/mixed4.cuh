// mixed4.cuh -- one strided pass of the mixed-radix recurrence: a tile of
// C = 2^CSH adjacent sub-transforms ("columns") of length L = a.m.N, element n
// of column c read from in + b*in_bs + (col0 + c)*in_cs + n*in_ns and written
// (transformed) to the same form of address in out.
//
// Every radix pass follows the Stockham recurrence of mixed.cu (natural order
// in and out, radices 16/8/4/2/3/5/7 in the order of the schedule):
//   butterfly j of a pass with radix R and Ns = product of the earlier radices:
//     v[r] = a[j + r L/R] * W_{Ns R}^{r (j mod Ns)},  V = R-point DFT of v,
//     b[(j div Ns) Ns R + (j mod Ns) + q Ns] = V[q].
// Threads take columns fastest (thread t: column t mod C, butterfly t div C),
// so a warp's global accesses are runs of C adjacent columns and, in shared
// memory, element (c, n) sits at sidx(n) * C + c: the C lanes of one
// butterfly index read and write adjacent words in every pass.  PAD inserts
// one row every 16 (sidx(n) = n + n/16), which spreads the stride-R writes of
// a leading radix-8/16 pass over the banks.
//
// On the last pass, the output k of column col can be multiplied by the
// four-step twiddle W_Nt^{col k} (Sec. 2.3.2: the partition's twiddle
// scaling), read as the product of two table entries (the exponent col*k is
// below Nt, split into low and high bits).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "gbfft_internal.h"
#include "mixed_common.cuh"

namespace gbfft {

template <int R, int CSH, bool PAD, typename T>
__device__ __forceinline__ void m4_pass(const Mixed4Args& a, int s, const T* gin, const T* src, T* dst, T* gout,
                                        bool first, bool last, long long col0, int valid) {
  using S = typename Cx<T>::S;
  constexpr int C = 1 << CSH;
  const MixedArgs& m = a.m;
  const T* tw = (const T*)m.tw;
  const unsigned NB = m.nb[s], Ns = m.ns[s], nsm = m.ns_m[s];
  const int total = (int)NB << CSH;
  const int stride = (int)m.tws[s];
  S sx, sy;
  if constexpr (std::is_same_v<T, double2>) {
    sx = m.sx;
    sy = m.sy;
  } else {
    sx = m.fsx;
    sy = m.fsy;
  }
  const T* ft_lo = (const T*)a.ft_lo;
  const T* ft_hi = (const T*)a.ft_hi;
  const unsigned long long ft_mask = (1ULL << a.ft_s) - 1ULL;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int c = b & (C - 1), j = b >> CSH;
    const bool ok = c < valid;
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int n = j + r * (int)NB;
      if (first)
        v[r] = ok ? __ldcs(gin + c * a.in_cs + (long long)n * a.in_ns) : Cx<T>::make(0, 0);
      else
        v[r] = src[msidx<PAD>(n) * C + c];
    }
    if (first && m.conj_in) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
    }
    const int jq = (int)fdiv((unsigned)j, nsm);
    const int k = j - jq * (int)Ns;
    if (Ns > 1) mixed_twiddles<R>(v, tw, k * stride);
    dft_any<R>(v);
    const int m0 = jq * (int)Ns * R + k;
    if (last) {
      if (!ok) continue;
      const unsigned long long col = (unsigned long long)(col0 + c);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int kk = m0 + q * (int)Ns;
        T y = v[q];
        if (ft_lo) {
          const unsigned long long e = col * (unsigned long long)kk;
          y = gmul(y, gmul(__ldg(ft_lo + (e & ft_mask)), __ldg(ft_hi + (e >> a.ft_s))));
        }
        if (m.scale_out) y = Cx<T>::make(y.x * sx, y.y * sy);
        __stcs(gout + c * a.out_cs + (long long)kk * a.out_ns, y);
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) dst[msidx<PAD>(m0 + q * (int)Ns) * C + c] = v[q];
    }
  }
}

// Tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...: batch t / tiles_per_batch,
// columns from (t mod tiles_per_batch) * C.  The first pass reads the whole
// tile from global memory before the last pass writes it, so in == out is
// safe when the passes of different tiles touch disjoint elements.
template <typename T, int CSH, bool PAD>
__device__ __forceinline__ void m4_tiles(const Mixed4Args& a, T* smem) {
  constexpr int C = 1 << CSH;
  const MixedArgs& m = a.m;
  T* const buf0 = smem;
  T* const buf1 = smem + (msidx<PAD>(m.N - 1) + 1) * C;
  for (long long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const long long bt = t / a.tiles_per_batch;
    const long long col0 = (t - bt * a.tiles_per_batch) * C;
    const int valid = (int)(a.ncols - col0 < C ? a.ncols - col0 : C);
    const T* gin = (const T*)m.in + bt * a.in_bs + col0 * a.in_cs;
    T* gout = (T*)m.out + bt * a.out_bs + col0 * a.out_cs;
    for (int s = 0; s < m.nrad; ++s) {
      const bool first = s == 0, last = s == m.nrad - 1;
      const T* src = (s & 1) ? buf0 : buf1;
      T* dst = (s & 1) ? buf1 : buf0;
      switch (m.rad[s]) {
        case 2: m4_pass<2, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
        case 3: m4_pass<3, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
        case 4: m4_pass<4, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
        case 5: m4_pass<5, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
        case 7: m4_pass<7, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
        case 8: m4_pass<8, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
        default: m4_pass<16, CSH, PAD>(a, s, gin, src, dst, gout, first, last, col0, valid); break;
      }
      __syncthreads();
    }
  }
}

}  // namespace gbfft
