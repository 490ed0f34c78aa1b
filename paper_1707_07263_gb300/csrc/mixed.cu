// mixed.cu -- transforms whose length is not a power of two but a product
// N = 2^a 3^b 5^c 7^d (N <= 14336), one on-chip pass per transform.
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

#include "gbfft_internal.h"

namespace gbfft {

// cos(2 pi m / R), sin(2 pi m / R) for the odd prime radices, m = 0..R-1
__device__ __forceinline__ constexpr float mixed_cos(int R, int m) {
  return R == 3 ? (m == 0 ? 1.0f : -0.5f)
       : R == 5 ? (m == 0 ? 1.0f : (m == 1 || m == 4) ? 0.30901699437494742f : -0.80901699437494742f)
       : (m == 0 ? 1.0f : (m == 1 || m == 6) ? 0.62348980185873353f
                        : (m == 2 || m == 5) ? -0.22252093395631440f : -0.90096886790241913f);
}
__device__ __forceinline__ constexpr float mixed_sin(int R, int m) {
  return R == 3 ? (m == 0 ? 0.0f : m == 1 ? 0.86602540378443865f : -0.86602540378443865f)
       : R == 5 ? (m == 0 ? 0.0f : m == 1 ? 0.95105651629515357f : m == 2 ? 0.58778525229247313f
                 : m == 3 ? -0.58778525229247313f : -0.95105651629515357f)
       : (m == 0 ? 0.0f : m == 1 ? 0.78183148246802981f : m == 2 ? 0.97492791218182361f
          : m == 3 ? 0.43388373911755812f : m == 4 ? -0.43388373911755812f : m == 5 ? -0.97492791218182361f
          : -0.78183148246802981f);
}

// R-point forward DFT for an odd prime R: with t_m = x_m + x_{R-m},
// u_m = x_m - x_{R-m} (m = 1..(R-1)/2),
//   X_k = x_0 + sum_m cos(2 pi mk/R) t_m - i sum_m sin(2 pi mk/R) u_m,
//   X_{R-k} the same with +i.
template <int R>
__device__ __forceinline__ void dft_odd(float2* v) {
  constexpr int H = (R - 1) / 2;
  float2 t[H], u[H];
  float2 s = v[0];
#pragma unroll
  for (int m = 1; m <= H; ++m) {
    t[m - 1] = cadd(v[m], v[R - m]);
    u[m - 1] = csub(v[m], v[R - m]);
    s = cadd(s, t[m - 1]);
  }
  float2 out[R];
  out[0] = s;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    float2 A = v[0], B = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      const float c = mixed_cos(R, (m * k) % R), sn = mixed_sin(R, (m * k) % R);
      A.x = fmaf(c, t[m - 1].x, A.x);
      A.y = fmaf(c, t[m - 1].y, A.y);
      B.x = fmaf(sn, u[m - 1].x, B.x);
      B.y = fmaf(sn, u[m - 1].y, B.y);
    }
    out[k] = make_float2(A.x + B.y, A.y - B.x);
    out[R - k] = make_float2(A.x - B.y, A.y + B.x);
  }
#pragma unroll
  for (int q = 0; q < R; ++q) v[q] = out[q];
}

template <int R>
__device__ __forceinline__ void dft_any(float2* v) {
  if constexpr (R == 3 || R == 5 || R == 7)
    dft_odd<R>(v);
  else
    dft_fwd<R>(v);
}

// n / d from the reciprocal m = ceil(2^32 / d) (m = 0 stands for d = 1)
__device__ __forceinline__ unsigned fdiv(unsigned n, unsigned m) { return m ? __umulhi(n, m) : n; }

// One pass s over the tile: C transforms of length N at src (global when
// FIRST, else shared memory), written to dst (global when LAST).
template <int R>
__device__ __forceinline__ void mixed_pass(const MixedArgs& a, int s, const float2* src, float2* dst, bool first,
                                           bool last, long long col0) {
  const int N = a.N;
  const unsigned NB = a.nb[s], nbm = a.nb_m[s], Ns = a.ns[s], nsm = a.ns_m[s];
  const int total = a.C * (int)NB;
  const int stride = N / ((int)Ns * R);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int c = (int)fdiv((unsigned)b, nbm), j = b - c * (int)NB;
    const bool ok = col0 + c < a.batch;
    float2 v[R];
    const float2* s = src + (long long)c * N + j;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (first)
        v[r] = ok ? __ldcs(s + r * NB) : make_float2(0.f, 0.f);
      else
        v[r] = s[r * NB];
    }
    if (first && a.conj_in) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r].y = -v[r].y;
    }
    const int jq = (int)fdiv((unsigned)j, nsm);
    const int k = j - jq * (int)Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(a.tw + r * k * stride));
    }
    dft_any<R>(v);
    const int base = jq * (int)Ns * R + k;
    float2* d = dst + (long long)c * N + base;
    if (last) {
      if (!ok) continue;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        float2 y = v[q];
        if (a.scale_out) y = make_float2(y.x * a.sx, y.y * a.sy);
        __stcs(d + q * Ns, y);
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) d[q * Ns] = v[q];
    }
  }
}

__global__ void __launch_bounds__(512, 2) mixed_kernel(const MixedArgs a) {
  extern __shared__ float2 smem[];
  const long long tile = blockIdx.x;
  const long long col0 = tile * a.C;
  const long long off = col0 * a.N;
  float2* const buf1 = smem + (size_t)a.C * a.N;
  for (int s = 0; s < a.nrad; ++s) {
    const bool first = s == 0, last = s == a.nrad - 1;
    const float2* src = first ? a.in + off : ((s & 1) ? smem : buf1);
    float2* dst = last ? a.out + off : ((s & 1) ? buf1 : smem);
    switch (a.rad[s]) {
      case 2: mixed_pass<2>(a, s, src, dst, first, last, col0); break;
      case 3: mixed_pass<3>(a, s, src, dst, first, last, col0); break;
      case 4: mixed_pass<4>(a, s, src, dst, first, last, col0); break;
      case 5: mixed_pass<5>(a, s, src, dst, first, last, col0); break;
      case 7: mixed_pass<7>(a, s, src, dst, first, last, col0); break;
      case 8: mixed_pass<8>(a, s, src, dst, first, last, col0); break;
      default: mixed_pass<16>(a, s, src, dst, first, last, col0); break;
    }
    __syncthreads();
  }
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
  a.nrad = mixed_radices(N, a.rad);
  if (a.nrad == 0 || N > kMixedMaxN) return FFT_ERR_UNSUPPORTED;
  a.N = (int)N;
  a.C = N <= 4096 ? (int)(4096 / N) : 1;
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
    }
  }
  p->mixed_threads = a.C * N <= 4096 ? 256 : 512;
  p->mixed_smem = (int)(2 * (size_t)a.C * (size_t)N * 8);
  if (p->mixed_smem > 48 * 1024 &&
      cudaFuncSetAttribute(mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, p->mixed_smem) != cudaSuccess)
    return FFT_ERR_UNSUPPORTED;
  const size_t tw_bytes = ((size_t)N * 8 + 255) & ~(size_t)255;
  if (cudaMalloc(&p->d_tables, tw_bytes + 256) != cudaSuccess) return FFT_ERR_ALLOC;
  a.tw = (const float2*)p->d_tables;
  p->d_status = (int*)((char*)p->d_tables + tw_bytes);
  if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess ||
      launch_gen_twiddles_n((float2*)a.tw, N, N, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess)
    return FFT_ERR_CUDA;
  p->launches = 1;
  return FFT_OK;
}

int mixed_exec(fft_plan* p, const float2* in, float2* out, int conj, float sx, float sy, int scale_out,
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
  const long long tiles = (p->batch + a.C - 1) / a.C;
  if (tiles > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
  void* args[] = {(void*)&a};
  return cudaLaunchKernel((const void*)mixed_kernel, dim3((unsigned)tiles), dim3(p->mixed_threads), args,
                          (size_t)p->mixed_smem, s) == cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace gbfft
