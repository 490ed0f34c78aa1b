// mixed.cu -- transforms whose length is not a power of two but a product
// N = 2^a 3^b 5^c 7^d (N <= 14336), one on-chip pass per transform; the same
// kernel in FP64 (complex128) for every such N <= 7168, powers of two
// included.
//
// Eq. 1 holds for any N; the paper's Cooley-Tukey split (Sec. 2.1) works for
// any factorisation N = R_1 R_2 ... R_s.  These kernels run the same Stockham
// autosort recurrence as the power-of-two tiles (natural order in and out),
// with the radix of every pass chosen at run time from {16, 8, 4, 2, 3, 5, 7}:
//   pass with radix R, Ns = product of the earlier radices, butterfly j:
//     v[r] = a[j + r N/R] * W_{Ns R}^{r (j mod Ns)},   r = 0..R-1
//     V    = R-point DFT of v
//     b[(j div Ns) Ns R + (j mod Ns) + q Ns] = V[q].
// The first pass reads global memory, the last writes it; the passes in
// between go through two shared-memory buffers in turn.  Twiddles come from
// one table W_N^m, m < N (FP64 sincospi rounded once to FP32), since
// W_{Ns R}^{r k} = W_N^{r k N / (Ns R)}.
#include <cuda_runtime.h>

#include <cstdlib>

#include <type_traits>

#include "gbfft_internal.h"

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

// One pass s over the tile: C transforms of length N at src (global when
// FIRST, else shared memory), written to dst (global when LAST).
template <int R, bool PAD, typename T>
__device__ __forceinline__ void mixed_pass(const MixedArgs& a, int s, const T* src, T* dst, bool first, bool last,
                                           long long col0) {
  using S = typename Cx<T>::S;
  const T* tw = (const T*)a.tw;
  const int N = a.N;
  const unsigned NB = a.nb[s], nbm = a.nb_m[s], Ns = a.ns[s], nsm = a.ns_m[s];
  const int total = a.C * (int)NB;
  const int stride = (int)a.tws[s];
  S sx, sy;   // the FP32 kernel reads FP32 copies: no FP64 conversion on its path
  if constexpr (std::is_same_v<T, double2>) {
    sx = a.sx;
    sy = a.sy;
  } else {
    sx = a.fsx;
    sy = a.fsy;
  }
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int c = (int)fdiv((unsigned)b, nbm), j = b - c * (int)NB;
    const bool ok = col0 + c < a.batch;
    T v[R];
    const int n0 = c * N + j;   // tile index of input r = 0
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (first)
        v[r] = ok ? __ldcs(src + n0 + r * NB) : Cx<T>::make(0, 0);
      else
        v[r] = src[msidx<PAD>(n0 + r * (int)NB)];
    }
    if (first && a.conj_in) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
    }
    const int jq = (int)fdiv((unsigned)j, nsm);
    const int k = j - jq * (int)Ns;
    if (Ns > 1) mixed_twiddles<R>(v, tw, k * stride);
    dft_any<R>(v);
    const int m0 = c * N + jq * (int)Ns * R + k;   // tile index of output q = 0
    if (last) {
      if (!ok) continue;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        T y = v[q];
        if (a.scale_out) y = Cx<T>::make(y.x * sx, y.y * sy);
        __stcs(dst + m0 + q * (int)Ns, y);
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) dst[msidx<PAD>(m0 + q * (int)Ns)] = v[q];
    }
  }
}

template <typename T, bool PAD>
__device__ __forceinline__ void mixed_tile(const MixedArgs& a, T* smem) {
  const long long tile = blockIdx.x;
  const long long col0 = tile * a.C;
  const long long off = col0 * a.N;
  const T* in = (const T*)a.in + off;
  T* out = (T*)a.out + off;
  T* const buf1 = smem + msidx<PAD>(a.C * a.N - 1) + 1;
  for (int s = 0; s < a.nrad; ++s) {
    const bool first = s == 0, last = s == a.nrad - 1;
    const T* src = first ? in : ((s & 1) ? smem : buf1);
    T* dst = last ? out : ((s & 1) ? buf1 : smem);
    switch (a.rad[s]) {
      case 2: mixed_pass<2, PAD>(a, s, src, dst, first, last, col0); break;
      case 3: mixed_pass<3, PAD>(a, s, src, dst, first, last, col0); break;
      case 4: mixed_pass<4, PAD>(a, s, src, dst, first, last, col0); break;
      case 5: mixed_pass<5, PAD>(a, s, src, dst, first, last, col0); break;
      case 7: mixed_pass<7, PAD>(a, s, src, dst, first, last, col0); break;
      case 8: mixed_pass<8, PAD>(a, s, src, dst, first, last, col0); break;
      default: mixed_pass<16, PAD>(a, s, src, dst, first, last, col0); break;
    }
    __syncthreads();
  }
}

// FP32: two resident CTAs of up to 512 threads (64 registers); FP64: one.
template <bool PAD>
__global__ void __launch_bounds__(512, 2) mixed_kernel(const MixedArgs a) {
  extern __shared__ __align__(16) unsigned char mixed_smem[];
  mixed_tile<float2, PAD>(a, (float2*)mixed_smem);
}
template <bool PAD>
__global__ void __launch_bounds__(512, 1) mixed_kernel64(const MixedArgs a) {
  extern __shared__ __align__(16) unsigned char mixed_smem[];
  mixed_tile<double2, PAD>(a, (double2*)mixed_smem);
}

static const void* mixed_fn(bool fp64, bool pad) {
  return fp64 ? (pad ? (const void*)mixed_kernel64<true> : (const void*)mixed_kernel64<false>)
              : (pad ? (const void*)mixed_kernel<true> : (const void*)mixed_kernel<false>);
}

// Radix schedule: radix-16 passes for 2^a and one 8/4/2 pass for the rest of
// 2^a first, then the 3s, 5s and 7s.  The first pass (Ns = 1) needs no
// twiddles, so it gets the largest radix.  (A bank model prefers the
// power-of-two radices last -- their first-pass writes at stride 8 or 16
// conflict -- but measured on GB300 that order is 10-25 % slower: the
// twiddle loads and products of a radix-16 pass cost more than the
// conflicts.)  Returns the number of passes, 0 if N has another prime factor
// or needs more than kMixedMaxPasses passes.
int mixed_radices(long long N, int* rad) {
  int n = 0;
  long long m = N;
  int a = 0;
  while (m % 2 == 0) {
    m /= 2;
    ++a;
  }
  while (a >= 4 && n < kMixedMaxPasses) {
    rad[n++] = 16;
    a -= 4;
  }
  if (a > 0 && n < kMixedMaxPasses) rad[n++] = 1 << a;
  const int odd[3] = {3, 5, 7};
  for (int i = 0; i < 3; ++i)
    while (m % odd[i] == 0 && n < kMixedMaxPasses) {
      m /= odd[i];
      rad[n++] = odd[i];
    }
  return (m == 1) ? n : 0;
}

int mixed_plan_init(fft_plan* p) {
  MixedArgs& a = p->mixed;
  const long long N = p->n;
  const bool fp64 = p->prec == FFT_PREC_FP64;
  const size_t esz = fp64 ? 16 : 8;
  // points per CTA when several transforms share one, and the CTA size for
  // such tiles (in the test build of the library, GBFFT_MIXED_TILE /
  // GBFFT_MIXED_THREADS override the FP32 values for measurement)
  long long tile = fp64 ? 2048 : 4096;
  int small_threads = 256;
#ifdef GBFFT_TEST_HOOKS
  if (!fp64) {
    const char* et = getenv("GBFFT_MIXED_TILE");
    const char* eh = getenv("GBFFT_MIXED_THREADS");
    const long long t = (et && *et) ? atoll(et) : 0;
    const int h = (eh && *eh) ? atoi(eh) : 0;
    if (t >= 256 && t <= 8192) tile = t;
    if (h == 128 || h == 256 || h == 512) small_threads = h;
  }
#endif
  a.nrad = mixed_radices(N, a.rad);
  if (a.nrad == 0 || N > (fp64 ? kMixedMaxN64 : kMixedMaxN)) return FFT_ERR_UNSUPPORTED;
  a.N = (int)N;
  a.C = N <= tile ? (int)(tile / N) : 1;
  if (a.C > p->batch) a.C = (int)p->batch;
  a.batch = p->batch;
  {
    unsigned ns = 1;
    for (int s = 0; s < a.nrad; ++s) {
      const unsigned nb = (unsigned)(N / a.rad[s]);
      a.nb[s] = nb;
      a.nb_m[s] = nb == 1 ? 0u : (unsigned)((0x100000000ULL + nb - 1) / nb);
      a.ns[s] = ns;
      a.ns_m[s] = ns == 1 ? 0u : (unsigned)((0x100000000ULL + ns - 1) / ns);
      ns *= (unsigned)a.rad[s];
      a.tws[s] = (unsigned)(N / ns);
    }
  }
  p->mixed_threads = a.C * N <= tile ? small_threads : 512;
  // padding pays when a radix-8 or -16 pass leads (its writes are strided by
  // the radix); pure odd-radix lengths keep the unpadded layout
  // (when the padded buffers fit in shared memory)
  const size_t pts = (size_t)a.C * (size_t)N;
  const size_t padded = pts + ((pts - 1) >> 4) + 1;
  p->mixed_pad = (a.rad[0] >= 8 && 2 * padded * esz <= 227 * 1024) ? 1 : 0;
  const size_t buf = p->mixed_pad ? padded : pts;
  p->mixed_smem = (int)(2 * buf * esz);
  if (p->mixed_smem > 227 * 1024) return FFT_ERR_UNSUPPORTED;
  const void* fn = mixed_fn(fp64, p->mixed_pad);
  if (p->mixed_smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->mixed_smem) != cudaSuccess)
    return FFT_ERR_UNSUPPORTED;
  const size_t tw_bytes = ((size_t)N * esz + 255) & ~(size_t)255;
  if (cudaMalloc(&p->d_tables, tw_bytes + 256) != cudaSuccess) return FFT_ERR_ALLOC;
  a.tw = p->d_tables;
  p->d_status = (int*)((char*)p->d_tables + tw_bytes);
  const cudaError_t e = fp64 ? launch_gen_twiddles_n64((double2*)p->d_tables, N, N, 0)
                             : launch_gen_twiddles_n((float2*)p->d_tables, N, N, 0);
  if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess || e != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess)
    return FFT_ERR_CUDA;
  p->launches = 1;
  return FFT_OK;
}

int mixed_exec(fft_plan* p, const void* in, void* out, int conj, double sx, double sy, int scale_out,
               cudaStream_t s) {
  // in == out is safe: a tile's first pass reads all of it (into shared
  // memory, or into one thread's registers when N is a single radix) before
  // its last pass writes
  MixedArgs a = p->mixed;
  a.in = in;
  a.out = out;
  a.conj_in = conj;
  a.scale_out = scale_out;
  a.sx = sx;
  a.sy = sy;
  a.fsx = (float)sx;
  a.fsy = (float)sy;
  const long long tiles = (p->batch + a.C - 1) / a.C;
  if (tiles > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
  void* args[] = {(void*)&a};
  const void* fn = mixed_fn(p->prec == FFT_PREC_FP64, p->mixed_pad);
  return cudaLaunchKernel(fn, dim3((unsigned)tiles), dim3(p->mixed_threads), args, (size_t)p->mixed_smem, s) ==
                 cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace gbfft
