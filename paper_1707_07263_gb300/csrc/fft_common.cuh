// fft_common.cuh -- complex helpers and the register-resident forward
// radix-2/4/8/16 DFTs used by every pass (the butterfly of paper Sec. 2.1).
//
// dft_fwd<R>(v) replaces v[0..R) by V[q] = sum_r v[r] W_R^{rq}, W_R = e^{-2*pi*i/R},
// in natural order.  Radix 8 is split 2 x 4 and radix 16 is split 4 x 4
// (Cooley-Tukey inside the register file); the inner twiddles are the
// constants W_16^m = cos(2*pi*m/16) - i sin(2*pi*m/16).
#pragma once
#include <cuda_runtime.h>

namespace gbfft {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// -i * a
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// cos(pi/8), sin(pi/8), sqrt(2)/2
#define GBFFT_C8 0.92387953251128674f
#define GBFFT_S8 0.38268343236508977f
#define GBFFT_R2 0.70710678118654752f

// a * W_16^m for the exponents that occur in the 4 x 4 split (m = n2*k1).
template <int M>
__device__ __forceinline__ float2 mul_w16(float2 a) {
  if constexpr (M == 0) {
    return a;
  } else if constexpr (M == 4) {
    return mul_mi(a);
  } else if constexpr (M == 2) {  // (1 - i)/sqrt2
    return make_float2(GBFFT_R2 * (a.x + a.y), GBFFT_R2 * (a.y - a.x));
  } else if constexpr (M == 6) {  // (-1 - i)/sqrt2
    return make_float2(GBFFT_R2 * (a.y - a.x), -GBFFT_R2 * (a.x + a.y));
  } else if constexpr (M == 1) {
    return cmul(a, make_float2(GBFFT_C8, -GBFFT_S8));
  } else if constexpr (M == 3) {
    return cmul(a, make_float2(GBFFT_S8, -GBFFT_C8));
  } else if constexpr (M == 9) {
    return cmul(a, make_float2(-GBFFT_C8, GBFFT_S8));
  } else {
    static_assert(M == 0, "unsupported W16 exponent");
    return a;
  }
}

__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// in-place 4-point forward DFT on (a, b, c, d) = x0..x3
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
  const float2 t2 = cadd(x1, x3), t3 = mul_mi(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

template <int R>
__device__ __forceinline__ void dft_fwd(float2* v);

template <>
__device__ __forceinline__ void dft_fwd<1>(float2*) {}

template <>
__device__ __forceinline__ void dft_fwd<2>(float2* v) { dft2(v[0], v[1]); }

template <>
__device__ __forceinline__ void dft_fwd<4>(float2* v) { dft4(v[0], v[1], v[2], v[3]); }

template <>
__device__ __forceinline__ void dft_fwd<8>(float2* v) {
  // E = DFT4 of even samples, O = DFT4 of odd samples;
  // X[k] = E[k] + W8^k O[k], X[k+4] = E[k] - W8^k O[k]
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  o1 = mul_w16<2>(o1);  // W8^1 = W16^2
  o2 = mul_mi(o2);      // W8^2
  o3 = mul_w16<6>(o3);  // W8^3 = W16^6
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

template <>
__device__ __forceinline__ void dft_fwd<16>(float2* v) {
  // n = 4*n1 + n2, k = k1 + 4*k2:
  //  (1) 4-point DFTs over n1 for each n2 -> slot n2 + 4*k1
  //  (2) multiply slot n2 + 4*k1 by W16^{n2*k1}
  //  (3) 4-point DFTs over n2 for each k1 -> slot 4*k1 + k2 holds X[k1 + 4*k2]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  v[5] = mul_w16<1>(v[5]);
  v[6] = mul_w16<2>(v[6]);
  v[7] = mul_w16<3>(v[7]);
  v[9] = mul_w16<2>(v[9]);
  v[10] = mul_w16<4>(v[10]);
  v[11] = mul_w16<6>(v[11]);
  v[13] = mul_w16<3>(v[13]);
  v[14] = mul_w16<6>(v[14]);
  v[15] = mul_w16<9>(v[15]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

}  // namespace gbfft
