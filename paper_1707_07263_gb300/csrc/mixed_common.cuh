// mixed_common.cuh -- the butterflies shared by the mixed-radix kernels
// (mixed.cu, run-time radix schedule; mixed_ct.cu, compile-time schedules):
// complex arithmetic for FP32 and FP64 elements, radix-2/4/8/16 and odd-prime
// 3/5/7 DFTs, the per-butterfly twiddles, the padded shared-memory index and
// the reciprocal division.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "fft_common.cuh"

namespace gbfft {

// ---- complex arithmetic for both element types -----------------------------
template <typename T>
struct Cx;
template <>
struct Cx<float2> {
  using S = float;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
};
template <>
struct Cx<double2> {
  using S = double;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
};
template <typename T>
__device__ __forceinline__ T gadd(T a, T b) { return Cx<T>::make(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ T gsub(T a, T b) { return Cx<T>::make(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ T gmul(T a, T b) {
  return Cx<T>::make(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename T>
__device__ __forceinline__ T gmul_mi(T a) { return Cx<T>::make(a.y, -a.x); }   // -i * a

// FP64 radix-2/4/8/16 DFTs (the FP32 path uses dft_fwd of fft_common.cuh):
// radix 8 = 2 x 4 and radix 16 = 4 x 4 with the inner twiddles W_16^m.
template <typename T>
__device__ __forceinline__ void gdft4(T& x0, T& x1, T& x2, T& x3) {
  const T t0 = gadd(x0, x2), t1 = gsub(x0, x2);
  const T t2 = gadd(x1, x3), t3 = gmul_mi(gsub(x1, x3));
  x0 = gadd(t0, t2);
  x2 = gsub(t0, t2);
  x1 = gadd(t1, t3);
  x3 = gsub(t1, t3);
}
template <typename T>
__device__ __forceinline__ T gw16(T a, int m) {
  // a * W_16^m, m in {1, 2, 3, 4, 6, 9}
  using S = typename Cx<T>::S;
  const S c8 = (S)0.92387953251128675613, s8 = (S)0.38268343236508977173, r2 = (S)0.70710678118654752440;
  switch (m) {
    case 1: return gmul(a, Cx<T>::make(c8, -s8));
    case 2: return Cx<T>::make(r2 * (a.x + a.y), r2 * (a.y - a.x));
    case 3: return gmul(a, Cx<T>::make(s8, -c8));
    case 4: return gmul_mi(a);
    case 6: return Cx<T>::make(r2 * (a.y - a.x), -r2 * (a.x + a.y));
    default: return gmul(a, Cx<T>::make(-c8, s8));   // m = 9
  }
}
template <int R, typename T>
__device__ __forceinline__ void gdft_pow2(T* v) {
  if constexpr (R == 2) {
    const T t = v[0];
    v[0] = gadd(t, v[1]);
    v[1] = gsub(t, v[1]);
  } else if constexpr (R == 4) {
    gdft4(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 8) {
    T e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    gdft4(e0, e1, e2, e3);
    gdft4(o0, o1, o2, o3);
    o1 = gw16(o1, 2);
    o2 = gmul_mi(o2);
    o3 = gw16(o3, 6);
    v[0] = gadd(e0, o0);
    v[4] = gsub(e0, o0);
    v[1] = gadd(e1, o1);
    v[5] = gsub(e1, o1);
    v[2] = gadd(e2, o2);
    v[6] = gsub(e2, o2);
    v[3] = gadd(e3, o3);
    v[7] = gsub(e3, o3);
  } else {
    static_assert(R == 16, "radix");
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) gdft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    v[5] = gw16(v[5], 1);
    v[6] = gw16(v[6], 2);
    v[7] = gw16(v[7], 3);
    v[9] = gw16(v[9], 2);
    v[10] = gw16(v[10], 4);
    v[11] = gw16(v[11], 6);
    v[13] = gw16(v[13], 3);
    v[14] = gw16(v[14], 6);
    v[15] = gw16(v[15], 9);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) gdft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    T t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
  }
}

// cos(2 pi m / R), sin(2 pi m / R) for the odd prime radices, m = 0..R-1
__device__ __forceinline__ constexpr double mixed_cos(int R, int m) {
  return R == 3 ? (m == 0 ? 1.0 : -0.5)
       : R == 5 ? (m == 0 ? 1.0 : (m == 1 || m == 4) ? 0.30901699437494742410 : -0.80901699437494742410)
       : (m == 0 ? 1.0 : (m == 1 || m == 6) ? 0.62348980185873353053
                       : (m == 2 || m == 5) ? -0.22252093395631440429 : -0.90096886790241912624);
}
__device__ __forceinline__ constexpr double mixed_sin(int R, int m) {
  return R == 3 ? (m == 0 ? 0.0 : m == 1 ? 0.86602540378443864676 : -0.86602540378443864676)
       : R == 5 ? (m == 0 ? 0.0 : m == 1 ? 0.95105651629515357212 : m == 2 ? 0.58778525229247312917
                 : m == 3 ? -0.58778525229247312917 : -0.95105651629515357212)
       : (m == 0 ? 0.0 : m == 1 ? 0.78183148246802980871 : m == 2 ? 0.97492791218182360702
          : m == 3 ? 0.43388373911755812048 : m == 4 ? -0.43388373911755812048 : m == 5 ? -0.97492791218182360702
          : -0.78183148246802980871);
}

// R-point forward DFT for an odd prime R: with t_m = x_m + x_{R-m},
// u_m = x_m - x_{R-m} (m = 1..(R-1)/2),
//   X_k = x_0 + sum_m cos(2 pi mk/R) t_m - i sum_m sin(2 pi mk/R) u_m,
//   X_{R-k} the same with +i.
template <int R, typename T>
__device__ __forceinline__ void dft_odd(T* v) {
  using S = typename Cx<T>::S;
  constexpr int H = (R - 1) / 2;
  T t[H], u[H];
  T s = v[0];
#pragma unroll
  for (int m = 1; m <= H; ++m) {
    t[m - 1] = gadd(v[m], v[R - m]);
    u[m - 1] = gsub(v[m], v[R - m]);
    s = gadd(s, t[m - 1]);
  }
  T out[R];
  out[0] = s;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    T A = v[0], B = Cx<T>::make(0, 0);
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      const S c = (S)mixed_cos(R, (m * k) % R), sn = (S)mixed_sin(R, (m * k) % R);
      A.x = fma(c, t[m - 1].x, A.x);
      A.y = fma(c, t[m - 1].y, A.y);
      B.x = fma(sn, u[m - 1].x, B.x);
      B.y = fma(sn, u[m - 1].y, B.y);
    }
    out[k] = Cx<T>::make(A.x + B.y, A.y - B.x);
    out[R - k] = Cx<T>::make(A.x - B.y, A.y + B.x);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = out[q];
}

template <int R, typename T>
__device__ __forceinline__ void dft_any(T* v) {
  if constexpr (R == 3 || R == 5 || R == 7)
    dft_odd<R>(v);
  else if constexpr (std::is_same_v<T, float2>)
    dft_fwd<R>(v);
  else
    gdft_pow2<R>(v);
}

// Twiddles w^r, r = 1..R-1, of one butterfly (w = W_N^e, e = k * stride).
// FP32: the powers w, w^2, w^4, w^8 that the radix needs are loaded from the
// W_N^m table, the others are products of them (radix 16: 4 loads + 11
// products instead of 15 loads; radix 5: 2 + 2; radix 7: 3 + 3); measured
// 2-16 % faster.  FP64: every power is loaded (FP64 products are the scarce
// resource; the product form measured 5-10 % slower).
template <int R, typename T>
__device__ __forceinline__ void mixed_twiddles(T* v, const T* tw, int e) {
  if constexpr (std::is_same_v<T, double2>) {
    // FP64 products cost far more than loads on this GPU: load every power
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = gmul(v[r], __ldg(tw + r * e));
    return;
  }
  T w[R];
  w[1] = __ldg(tw + e);
  if constexpr (R >= 3) w[2] = __ldg(tw + 2 * e);
  if constexpr (R >= 5) w[4] = __ldg(tw + 4 * e);
  if constexpr (R >= 9) w[8] = __ldg(tw + 8 * e);
  if constexpr (R >= 4) w[3] = gmul(w[1], w[2]);
  if constexpr (R >= 6) w[5] = gmul(w[4], w[1]);
  if constexpr (R >= 7) w[6] = gmul(w[4], w[2]);
  if constexpr (R >= 8) w[7] = gmul(w[4], w[3]);
  if constexpr (R >= 16) {
#pragma unroll
    for (int r = 1; r < 8; ++r) w[8 + r] = gmul(w[8], w[r]);
  }
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = gmul(v[r], w[r]);
}

// Shared-memory index of tile element n: padded by one entry every 16 when
// PAD (conflict-free strided writes of a leading radix-8/16 pass, chosen per
// plan from a bank model of every pass), identity otherwise.
template <bool PAD>
__device__ __forceinline__ int msidx(int n) { return PAD ? n + (n >> 4) : n; }

// n / d from the reciprocal m = ceil(2^32 / d) (m = 0 stands for d = 1)
__device__ __forceinline__ unsigned fdiv(unsigned n, unsigned m) { return m ? __umulhi(n, m) : n; }

}  // namespace gbfft
