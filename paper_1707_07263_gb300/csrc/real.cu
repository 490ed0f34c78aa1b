// real.cu -- the even/odd split of real-data transforms longer than one
// on-chip pass (N = 2M reals, M > 2^14; every FP64 real transform): the
// complex length-M plan runs on the row read as z[m] = x[2m] + i x[2m+1], and
// these kernels turn Z into the
// N/2 + 1 outputs of Eq. 1 (real-to-complex) or X into Z (complex-to-real).
// Each thread handles the pair (k, M - k), so every value is read once.
#include <cuda_runtime.h>

#include "gbfft_internal.h"
#include "mixed_common.cuh"

namespace gbfft {

__device__ __forceinline__ float2 w_two_level(const float2* lo, const float2* hi, int s, long long k) {
  return cmul(__ldg(lo + (k & ((1LL << s) - 1))), __ldg(hi + (k >> s)));
}

// X[k] = E + W_N^k O, E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / (2i),
// for the pair k = q, M - q (q = 0..M/2; Z[M] = Z[0], W_N^M = -1).
// Outputs X[1..M-1] are multiplied by s_int, X[0] and X[M] by s_end (1 and 1
// for the transform; 2/N and 1/N for the adjoint of the complex-to-real one).
__global__ void r2c_split_kernel(const float2* __restrict__ z, float2* __restrict__ x, long long M, long long batch,
                                 const float2* lo, const float2* hi, int s, float s_int, float s_end) {
  const long long half = M / 2 + 1;
  const long long total = half * batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / half, q = i - b * half;
    const float2* zr = z + b * M;
    float2* xr = x + b * (M + 1);
    const float2 zk = __ldcs(zr + q);
    const float2 zm = __ldcs(zr + ((M - q) & (M - 1)));
    const float2 w = w_two_level(lo, hi, s, q);
    {
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      const float sc = q == 0 ? s_end : s_int;
      const float2 xq = cadd(e, cmul(w, o));
      __stcs(xr + q, make_float2(xq.x * sc, xq.y * sc));
    }
    if (M - q != q) {
      // the partner output M - q: roles of zk and zm swap, W_N^{M-q} = -conj(W_N^q)
      const float2 e = make_float2(0.5f * (zm.x + zk.x), 0.5f * (zm.y - zk.y));
      const float2 o = make_float2(0.5f * (zm.y + zk.y), -0.5f * (zm.x - zk.x));
      const float sc = q == 0 ? s_end : s_int;   // q == 0: the partner is X[M]
      const float2 xm = cadd(e, cmul(make_float2(-w.x, w.y), o));
      __stcs(xr + (M - q), make_float2(xm.x * sc, xm.y * sc));
    }
  }
}

// Z[k] = E + i O, E = (X[k] + conj X[M-k]) / 2, O = (X[k] - conj X[M-k]) W_N^{-k} / 2,
// for the pair k = q, M - q (q = 0..M/2; M - q < M only); Im X[0], Im X[M] do not enter.
// end_mul multiplies the real parts of X[0] and X[M] (1 for the transform, 2
// for the adjoint of the real-to-complex transform).
__global__ void c2r_split_kernel(const float2* __restrict__ x, float2* __restrict__ z, long long M, long long batch,
                                 const float2* lo, const float2* hi, int s, float end_mul) {
  const long long half = M / 2 + 1;
  const long long total = half * batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / half, q = i - b * half;
    const float2* xr = x + b * (M + 1);
    float2* zr = z + b * M;
    float2 xk = __ldcs(xr + q);
    float2 xm = __ldcs(xr + (M - q));
    if (q == 0) {
      xk = make_float2(xk.x * end_mul, 0.f);
      xm = make_float2(xm.x * end_mul, 0.f);
    }
    const float2 w = w_two_level(lo, hi, s, q);
    {
      const float2 e = make_float2(0.5f * (xk.x + xm.x), 0.5f * (xk.y - xm.y));
      const float2 d = make_float2(0.5f * (xk.x - xm.x), 0.5f * (xk.y + xm.y));
      const float2 o = cmul(d, make_float2(w.x, -w.y));
      __stcs(zr + q, make_float2(e.x - o.y, e.y + o.x));
    }
    if (q != 0 && M - q != q) {
      // Z[M - q]: W_N^{-(M-q)} = conj(-conj(W_N^q)) = -W_N^q
      const float2 e = make_float2(0.5f * (xm.x + xk.x), 0.5f * (xm.y - xk.y));
      const float2 d = make_float2(0.5f * (xm.x - xk.x), 0.5f * (xm.y + xk.y));
      const float2 o = cmul(d, make_float2(-w.x, -w.y));
      __stcs(zr + (M - q), make_float2(e.x - o.y, e.y + o.x));
    }
  }
}

// FP64 (complex128) forms of the two kernels above for any even N = 2M (M a
// 7-smooth FP64 length): the same steps in double, partner index M - q taken
// mod M, W_N^q = lo[q & (2^s - 1)] * hi[q >> s] from FP64 tables.
__device__ __forceinline__ double2 w_two_level64(const double2* lo, const double2* hi, int s, long long q) {
  return gmul(__ldg(lo + (q & ((1LL << s) - 1))), __ldg(hi + (q >> s)));
}

__global__ void r2c_split64_kernel(const double2* __restrict__ z, double2* __restrict__ x, long long M,
                                   long long batch, const double2* lo, const double2* hi, int s, double s_int,
                                   double s_end) {
  const long long half = M / 2 + 1;
  const long long total = half * batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / half, q = i - b * half;
    const double2* zr = z + b * M;
    double2* xr = x + b * (M + 1);
    const double2 zk = __ldcs(zr + q);
    const double2 zm = __ldcs(zr + (q == 0 ? 0 : M - q));
    const double2 w = w_two_level64(lo, hi, s, q);
    {
      const double2 e = make_double2(0.5 * (zk.x + zm.x), 0.5 * (zk.y - zm.y));
      const double2 o = make_double2(0.5 * (zk.y + zm.y), -0.5 * (zk.x - zm.x));
      const double sc = q == 0 ? s_end : s_int;
      const double2 xq = gadd(e, gmul(w, o));
      __stcs(xr + q, make_double2(xq.x * sc, xq.y * sc));
    }
    if (M - q != q) {
      const double2 e = make_double2(0.5 * (zm.x + zk.x), 0.5 * (zm.y - zk.y));
      const double2 o = make_double2(0.5 * (zm.y + zk.y), -0.5 * (zm.x - zk.x));
      const double sc = q == 0 ? s_end : s_int;
      const double2 xm = gadd(e, gmul(make_double2(-w.x, w.y), o));
      __stcs(xr + (M - q), make_double2(xm.x * sc, xm.y * sc));
    }
  }
}

__global__ void c2r_split64_kernel(const double2* __restrict__ x, double2* __restrict__ z, long long M,
                                   long long batch, const double2* lo, const double2* hi, int s, double end_mul) {
  const long long half = M / 2 + 1;
  const long long total = half * batch;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / half, q = i - b * half;
    const double2* xr = x + b * (M + 1);
    double2* zr = z + b * M;
    double2 xk = __ldcs(xr + q);
    double2 xm = __ldcs(xr + (M - q));
    if (q == 0) {
      xk = make_double2(xk.x * end_mul, 0.0);
      xm = make_double2(xm.x * end_mul, 0.0);
    }
    const double2 w = w_two_level64(lo, hi, s, q);
    {
      const double2 e = make_double2(0.5 * (xk.x + xm.x), 0.5 * (xk.y - xm.y));
      const double2 d = make_double2(0.5 * (xk.x - xm.x), 0.5 * (xk.y + xm.y));
      const double2 o = gmul(d, make_double2(w.x, -w.y));
      __stcs(zr + q, make_double2(e.x - o.y, e.y + o.x));
    }
    if (q != 0 && M - q != q) {
      const double2 e = make_double2(0.5 * (xm.x + xk.x), 0.5 * (xm.y - xk.y));
      const double2 d = make_double2(0.5 * (xm.x - xk.x), 0.5 * (xm.y + xk.y));
      const double2 o = gmul(d, make_double2(-w.x, -w.y));
      __stcs(zr + (M - q), make_double2(e.x - o.y, e.y + o.x));
    }
  }
}

static unsigned split_grid(long long total) {
  long long g = (total + 255) / 256;
  return (unsigned)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

cudaError_t launch_r2c_split(const float2* z, float2* x, long long M, long long batch, const float2* lo,
                             const float2* hi, int s, float s_int, float s_end, cudaStream_t st) {
  r2c_split_kernel<<<split_grid((M / 2 + 1) * batch), 256, 0, st>>>(z, x, M, batch, lo, hi, s, s_int, s_end);
  return cudaGetLastError();
}

cudaError_t launch_c2r_split(const float2* x, float2* z, long long M, long long batch, const float2* lo,
                             const float2* hi, int s, float end_mul, cudaStream_t st) {
  c2r_split_kernel<<<split_grid((M / 2 + 1) * batch), 256, 0, st>>>(x, z, M, batch, lo, hi, s, end_mul);
  return cudaGetLastError();
}

cudaError_t launch_r2c_split64(const double2* z, double2* x, long long M, long long batch, const double2* lo,
                               const double2* hi, int s, double s_int, double s_end, cudaStream_t st) {
  r2c_split64_kernel<<<split_grid((M / 2 + 1) * batch), 256, 0, st>>>(z, x, M, batch, lo, hi, s, s_int, s_end);
  return cudaGetLastError();
}

cudaError_t launch_c2r_split64(const double2* x, double2* z, long long M, long long batch, const double2* lo,
                               const double2* hi, int s, double end_mul, cudaStream_t st) {
  c2r_split64_kernel<<<split_grid((M / 2 + 1) * batch), 256, 0, st>>>(x, z, M, batch, lo, hi, s, end_mul);
  return cudaGetLastError();
}

}  // namespace gbfft
