// tc.cu -- plans whose radix-16 passes run on the tensor cores
// (FFT_PREC_TC_BF16 / _FP16 / _BF16_SPLIT / _FP16_SPLIT).
//
// Compiled for the shapes of the precision workload: single-pass lengths 2^8,
// 2^10 and 2^12, and four-step lengths 2^16 (2^8 x 2^8), 2^20 (2^10 x 2^10) and
// 2^24 (2^12 x 2^12).  Other lengths return FFT_ERR_UNSUPPORTED for these
// precisions.  The split of work between passes and the kernels' I/O are the
// FP32 plan's; only the radix-16 DFTs change arithmetic.
#include <cuda_runtime.h>

#include <cstring>

#include "gbfft_internal.h"
#include "tc_fft.cuh"
#include "tile_registry.h"

namespace gbfft {

const TileKernelInfo* tc_kernel_bf16(int map, int lg, int C);
const TileKernelInfo* tc_kernel_fp16(int map, int lg, int C);
const TileKernelInfo* tc_kernel_bf16s(int map, int lg, int C);
const TileKernelInfo* tc_kernel_fp16s(int map, int lg, int C);

static const TileKernelInfo* tc_kernel(int prec, int map, int lg, int C) {
  switch (prec) {
    case FFT_PREC_TC_BF16: return tc_kernel_bf16(map, lg, C);
    case FFT_PREC_TC_FP16: return tc_kernel_fp16(map, lg, C);
    case FFT_PREC_TC_BF16_SPLIT: return tc_kernel_bf16s(map, lg, C);
    case FFT_PREC_TC_FP16_SPLIT: return tc_kernel_fp16s(map, lg, C);
  }
  return nullptr;
}

__global__ void gen_tc_twiddles(float2* tab, int lg) {
  const int total = tc_tw_size(lg);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int s = 1;
    while (s + 1 < radix_nst(lg) && idx >= tc_tw_off(lg, s + 1)) ++s;
    const int local = idx - tc_tw_off(lg, s);
    const int NS = 1 << radix_lgns(lg, s);
    const int r = local / NS + 1, k = local % NS;
    const long long M = 16LL * NS;
    double sn, cs;
    sincospi(-2.0 * (double)(((long long)r * k) % M) / (double)M, &sn, &cs);
    tab[idx] = make_float2((float)cs, (float)sn);
  }
}

static int prep(const TileKernelInfo* k) {
  if (!k) return FFT_ERR_UNSUPPORTED;
  if (k->smem_bytes > 48 * 1024 &&
      cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k->smem_bytes) != cudaSuccess)
    return FFT_ERR_CUDA;
  return FFT_OK;
}

int tc_plan_init(fft_plan* p) {
  const TileKernelInfo *k1 = nullptr, *k2 = nullptr;
  int lgA = 0, lgB = 0;
  if (p->kind == KIND_SINGLE) {
    k1 = tc_kernel(p->prec, MAP_JJ, p->lg, jj_cols(p->lg));
    lgA = p->lg;
  } else if (p->kind == KIND_FOURSTEP) {
    k1 = tc_kernel(p->prec, MAP_CC, p->lg1, p->c1);
    k2 = tc_kernel(p->prec, MAP_JC, p->lg2, p->c2);
    if (!k2) return FFT_ERR_UNSUPPORTED;
    lgA = p->lg1;
    lgB = p->lg2;
  }
  if (!k1) return FFT_ERR_UNSUPPORTED;
  int rc = prep(k1);
  if (!rc && k2) rc = prep(k2);
  if (rc) return rc;
  const size_t szA = (size_t)tc_tw_size(lgA), szB = lgB ? (size_t)tc_tw_size(lgB) : 0;
  const size_t offB = ((szA * 8 + 8) + 255) & ~(size_t)255;
  if (cudaMalloc(&p->d_tc, offB + szB * 8 + 256) != cudaSuccess) return FFT_ERR_ALLOC;
  float2* ta = (float2*)p->d_tc;
  float2* tb = (float2*)((char*)p->d_tc + offB);
  if (szA) gen_tc_twiddles<<<(unsigned)((szA + 255) / 256), 256>>>(ta, lgA);
  if (szB) gen_tc_twiddles<<<(unsigned)((szB + 255) / 256), 256>>>(tb, lgB);
  if (cudaDeviceSynchronize() != cudaSuccess) return FFT_ERR_CUDA;
  p->ktc1 = k1;
  p->ktc2 = k2;
  p->tctw1 = ta;
  p->tctw2 = tb;
  return FFT_OK;
}

static int launch(const TileKernelInfo* k, const TileArgs& a, long long ntiles, cudaStream_t s) {
  void* args[] = {(void*)&a};
  return cudaLaunchKernel(k->fn, dim3((unsigned)ntiles), dim3(k->threads), args, (size_t)k->smem_bytes, s) ==
                 cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

int tc_exec(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s) {
  if ((uintptr_t)out & 15) return FFT_ERR_ALIGN;  // the last pass stores 16-byte pairs
  const int inv = dir & FFT_INVERSE, adj = (dir & FFT_ADJOINT) ? 1 : 0;
  const int conj = inv ^ adj;
  const float scale = inv ? (float)(1.0 / (double)p->n) : 1.0f;
  TileArgs a;
  memset(&a, 0, sizeof(a));
  a.stream_in = a.stream_out = 1;
  a.conj_in = conj;
  if (p->kind == KIND_SINGLE) {
    const int C = p->ktc1->C;
    const long long L = p->n;
    a.in = in;
    a.out = out;
    a.tw = p->tctw1;
    a.tiles_per_batch = (p->batch + C - 1) / C;
    a.in_gstride = a.out_gstride = (long long)C * L;
    a.in_sc = a.out_sc = L;
    a.in_sn = a.out_sn = 1;
    a.ncols = p->batch;
    a.scale_out = (conj || inv) ? 1 : 0;
    a.sx = scale;
    a.sy = conj ? -scale : scale;
    return launch(p->ktc1, a, a.tiles_per_batch, s);
  }
  if (!p->ws) return FFT_ERR_NO_WORKSPACE;
  const long long N = p->n, N1 = 1LL << p->lg1, N2 = 1LL << p->lg2;
  float2* ws = (float2*)p->ws;
  a.in = in;
  a.out = ws;
  a.tw = p->tctw1;
  a.tiles_per_batch = N2 / p->c1;
  a.in_bstride = a.out_bstride = N;
  a.in_gstride = a.out_gstride = p->c1;
  a.in_sc = a.out_sc = 1;
  a.in_sn = a.out_sn = N2;
  a.ncols = N2;
  a.ft_lo = p->ft_lo;
  a.ft_hi = p->ft_hi;
  a.ft_lgN = p->lg1 + p->lg2;
  a.ft_s = p->ft_s;
  a.stream_out = 0;
  int rc = launch(p->ktc1, a, a.tiles_per_batch * p->batch, s);
  if (rc) return rc;
  TileArgs b;
  memset(&b, 0, sizeof(b));
  b.in = ws;
  b.out = out;
  b.tw = p->tctw2;
  b.tiles_per_batch = N1 / p->c2;
  b.in_bstride = b.out_bstride = N;
  b.in_gstride = (long long)p->c2 * N2;
  b.in_sc = N2;
  b.in_sn = 1;
  b.out_gstride = p->c2;
  b.out_sc = 1;
  b.out_sn = N1;
  b.ncols = N1;
  b.stream_in = 0;
  b.stream_out = 1;
  b.scale_out = (conj || inv) ? 1 : 0;
  b.sx = scale;
  b.sy = conj ? -scale : scale;
  return launch(p->ktc2, b, b.tiles_per_batch * p->batch, s);
}

}  // namespace gbfft
