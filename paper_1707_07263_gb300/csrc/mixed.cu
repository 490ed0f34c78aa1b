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

#include <algorithm>
#include <cstdlib>

#include <type_traits>

#include "gbfft_internal.h"
#include "mixed_common.cuh"

namespace gbfft {

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

// The pass schedule of length N into a: radices, N/R and Ns per pass with
// their reciprocals, and the twiddle strides into the W_N table.  Returns
// false when N is not 7-smooth or needs too many passes.
bool mixed_schedule(MixedArgs& a, long long N) {
  a.nrad = mixed_radices(N, a.rad);
  if (a.nrad == 0 || N > kMixedMaxN) return false;
  a.N = (int)N;
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
  return true;
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
  if (!mixed_schedule(a, N) || N > (fp64 ? kMixedMaxN64 : kMixedMaxN)) return FFT_ERR_UNSUPPORTED;
  a.C = N <= tile ? (int)(tile / N) : 1;
  if (a.C > p->batch) a.C = (int)p->batch;
  a.batch = p->batch;
  p->mixed_threads = a.C * N <= tile ? small_threads : 512;
  // lengths with a compiled three-pass schedule of composite radices
  // (mixed_ct.cu): their own tile size, CTA size and padding choice
  p->mixed_ct = fp64 ? nullptr : mixed_ct_lookup(N);
  const int generic_C = a.C;
  if (p->mixed_ct) {
    a.C = (int)std::min<long long>(p->mixed_ct->C, p->batch);
    const size_t pts = (size_t)a.C * (size_t)N;
    const size_t buf = p->mixed_ct->pad ? pts + ((pts - 1) >> 4) + 1 : pts;
    p->mixed_threads = p->mixed_ct->threads;
    p->mixed_smem = (int)(2 * buf * esz);
    if (p->mixed_smem > 227 * 1024) {
      p->mixed_ct = nullptr;   // does not fit: the run-time schedule below
      a.C = generic_C;
      p->mixed_threads = a.C * N <= tile ? small_threads : 512;
    } else if (p->mixed_smem > 48 * 1024 &&
               cudaFuncSetAttribute(p->mixed_ct->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->mixed_smem) !=
                   cudaSuccess) {
      return FFT_ERR_UNSUPPORTED;
    }
  }
  // padding pays when a radix-8 or -16 pass leads (its writes are strided by
  // the radix); pure odd-radix lengths keep the unpadded layout
  // (when the padded buffers fit in shared memory)
  const size_t pts = (size_t)a.C * (size_t)N;
  const size_t padded = pts + ((pts - 1) >> 4) + 1;
  p->mixed_pad = (a.rad[0] >= 8 && 2 * padded * esz <= 227 * 1024) ? 1 : 0;
  if (!p->mixed_ct) {
    const size_t buf = p->mixed_pad ? padded : pts;
    p->mixed_smem = (int)(2 * buf * esz);
    if (p->mixed_smem > 227 * 1024) return FFT_ERR_UNSUPPORTED;
    const void* fn = mixed_fn(fp64, p->mixed_pad);
    if (p->mixed_smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->mixed_smem) != cudaSuccess)
      return FFT_ERR_UNSUPPORTED;
  }
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
  const void* fn = p->mixed_ct ? p->mixed_ct->fn : mixed_fn(p->prec == FFT_PREC_FP64, p->mixed_pad);
  return cudaLaunchKernel(fn, dim3((unsigned)tiles), dim3(p->mixed_threads), args, (size_t)p->mixed_smem, s) ==
                 cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace gbfft
