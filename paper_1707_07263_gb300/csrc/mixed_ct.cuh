// mixed_ct.cuh -- compile-time radix building blocks of the mixed-radix
// kernels with fixed schedules (mixed_ct.cu: one on-chip pass per transform;
// mixed4_ct.cu: the strided passes of the two-pass plans): constant
// twiddle products, composite register radices of 10..25 points as
// Cooley-Tukey splits inside the register file, and the per-butterfly twiddles
// from one W_N table.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "ct_trig.h"
#include "mixed_common.cuh"

namespace gbfft {

// a * W_R^M (W_R = exp(-2 pi i / R)) for compile-time R, M: quarter turns are
// exact rotations, eighth turns two products, the rest a complex product with
// constant factors.
template <int R, int M>
__device__ __forceinline__ float2 mul_wc(float2 a) {
  constexpr int m = M % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr ((4 * m) % R == 0) {
    constexpr int qt = 4 * m / R;   // W^m = (-i)^qt
    if constexpr (qt == 1) return make_float2(a.y, -a.x);
    else if constexpr (qt == 2) return make_float2(-a.x, -a.y);
    else return make_float2(-a.y, a.x);
  } else if constexpr ((8 * m) % R == 0) {
    constexpr int et = 8 * m / R;   // odd eighth of a turn
    if constexpr (et == 1) return make_float2(GBFFT_R2 * (a.x + a.y), GBFFT_R2 * (a.y - a.x));
    else if constexpr (et == 3) return make_float2(GBFFT_R2 * (a.y - a.x), -GBFFT_R2 * (a.x + a.y));
    else if constexpr (et == 5) return make_float2(-GBFFT_R2 * (a.x + a.y), GBFFT_R2 * (a.x - a.y));
    else return make_float2(GBFFT_R2 * (a.x - a.y), GBFFT_R2 * (a.x + a.y));
  } else {
    constexpr float c = (float)ct_cos(m, R), s = (float)ct_sin(m, R);
    return cmul(a, make_float2(c, -s));
  }
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B..E-1
template <int B, int E, typename F>
__device__ __forceinline__ void ct_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    ct_for<B + 1, E>(f);
  }
}

template <int R>
__device__ __forceinline__ void ct_dft(float2* v);

// R = A * B, n = B n1 + n2, k = k1 + A k2:
//   X[k1 + A k2] = sum_{n2} W_B^{n2 k2} W_R^{n2 k1} sum_{n1} x[B n1 + n2] W_A^{n1 k1}
template <int A, int B>
__device__ __forceinline__ void ct_dft_split(float2* v) {
  constexpr int R = A * B;
  float2 x[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2)
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) x[n2][n1] = v[B * n1 + n2];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) ct_dft<A>(x[n2]);
  ct_for<1, B>([&](auto n2c) {
    constexpr int n2 = decltype(n2c)::value;
    ct_for<1, A>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      x[n2][k1] = mul_wc<R, n2 * k1>(x[n2][k1]);
    });
  });
  float2 y[A][B];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) y[k1][n2] = x[n2][k1];
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) ct_dft<B>(y[k1]);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = y[k1][k2];
}

template <int R>
__device__ __forceinline__ void ct_dft(float2* v) {
  if constexpr (R == 2 || R == 4 || R == 8 || R == 16) dft_fwd<R>(v);
  else if constexpr (R == 3 || R == 5 || R == 7) dft_odd<R>(v);
  else if constexpr (R == 10) ct_dft_split<2, 5>(v);
  else if constexpr (R == 12) ct_dft_split<4, 3>(v);
  else if constexpr (R == 15) ct_dft_split<3, 5>(v);
  else if constexpr (R == 20) ct_dft_split<4, 5>(v);
  else if constexpr (R == 24) ct_dft_split<8, 3>(v);
  else {
    static_assert(R == 25, "compiled radices: 2, 3, 4, 5, 7, 8, 10, 12, 15, 16, 20, 24, 25");
    ct_dft_split<5, 5>(v);
  }
}

// largest power of two <= r (r >= 1)
constexpr int ct_hp2(int r) { return r >= 16 ? 16 : r >= 8 ? 8 : r >= 4 ? 4 : r >= 2 ? 2 : 1; }

// v[r] *= w^r, r = 1..R-1, w = W_N^e: the powers w^{2^i} < R are loaded from
// the W_N table (r e < N for every r < R, so no reduction is needed), the
// others are products of one loaded power and an earlier power.
template <int R>
__device__ __forceinline__ void ct_twiddles(float2* v, const float2* tw, int e) {
  float2 w[R];
#pragma unroll
  for (int p = 1; p < R; p *= 2) w[p] = __ldg(tw + p * e);
  ct_for<3, R>([&](auto rc) {
    constexpr int r = decltype(rc)::value;
    constexpr int h = ct_hp2(r);
    if constexpr (h != r) w[r] = cmul(w[h], w[r - h]);
  });
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r]);
}

}  // namespace gbfft
