// mixed4.cu -- plans of strided mixed-radix passes (kernels in mixed4.cuh,
// mixed4_f32.cu, mixed4_f64.cu):
//  * 1-D lengths beyond one on-chip pass: FP64 (complex128) N > 7168 and FP32
//    7-smooth N > 14336 that are not powers of two.  Sec. 2.3.2's partition:
//    N = N1 N2, n = n1 N2 + n2, k = k1 + N1 k2,
//      column pass  Y[k1][n2] = W_N^{n2 k1} sum_{n1} x[n1 N2 + n2] W_N1^{n1 k1}
//      row pass     X[k1 + N1 k2] = sum_{n2} Y[k1][n2] W_N2^{n2 k2},
//    through a workspace of N complex values per transform (Y stored as
//    ws[k1 N2 + n2]).  Both lengths are one on-chip mixed-radix sub-transform.
//  * 2-D transforms in FP64, and in FP32 when a side is not a power of two:
//    the transforms of every row, then of every column (Sec. 2.3.2), in place
//    in the output.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "gbfft_internal.h"

namespace gbfft {

const void* mixed4_kernel_fn32(int csh, bool pad);
const void* mixed4_kernel_fn64(int csh, bool pad);

const void* mixed4_kernel_fn(bool fp64, int csh, bool pad) {
  return fp64 ? mixed4_kernel_fn64(csh, pad) : mixed4_kernel_fn32(csh, pad);
}

constexpr int kMixed4Threads = 256;
constexpr size_t kMixed4SmemLimit = 227 * 1024;

static size_t m4_smem(long long L, int csh, bool pad, size_t esz) {
  const size_t rows = pad ? (size_t)(L + ((L - 1) >> 4)) : (size_t)L;
  return 2 * rows * ((size_t)1 << csh) * esz;
}

// One pass: sub-length L, ncols columns in each of `batches` batches, element
// n of column col of batch b at b*bs + col*cs + n*ns on either side.  Columns
// per CTA: as many as make a tile of about 4096 (FP32) or 2048 (FP64) points,
// at most 16 (8) and at most ncols, fewer when the buffers do not fit.
static int m4_pass_init(fft_plan* p, Mixed4Pass& P, long long L, long long ncols, long long batches,
                        long long in_bs, long long in_cs, long long in_ns, long long out_bs, long long out_cs,
                        long long out_ns, const void* tw, int in_role, int out_role) {
  const bool fp64 = p->prec == FFT_PREC_FP64;
  const size_t esz = fp64 ? 16 : 8;
  memset(&P, 0, sizeof(P));
  Mixed4Args& a = P.a;
  if (!mixed_schedule(a.m, L)) return FFT_ERR_UNSUPPORTED;
  a.m.tw = tw;
  // FP32 sub-lengths with a compiled schedule take it when the batch has
  // at least its columns per CTA
  const Mixed4CtInfo* ct = fp64 ? nullptr : mixed4_ct_lookup(L);
  if (ct && (1LL << ct->csh) > ncols) ct = nullptr;
  const long long target = fp64 ? 2048 : 4096;
  const int csh_max = fp64 ? 3 : 4;
  int csh = 0;
  while (csh < csh_max && (L << (csh + 1)) <= target && (2LL << csh) <= ncols) ++csh;
  while (csh > 0 && m4_smem(L, csh, true, esz) > kMixed4SmemLimit) --csh;
  if (ct) csh = ct->csh;
  const bool pad = m4_smem(L, csh, true, esz) <= kMixed4SmemLimit;
  const size_t smem = m4_smem(L, csh, pad, esz);
  if (smem > kMixed4SmemLimit || (ct && !pad)) return FFT_ERR_UNSUPPORTED;
  P.fn = ct ? ct->fn : mixed4_kernel_fn(fp64, csh, pad);
  if (!P.fn) return FFT_ERR_UNSUPPORTED;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(P.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FFT_ERR_CUDA;
  const int C = 1 << csh;
  a.m.C = C;
  a.m.batch = batches;
  a.in_bs = in_bs;
  a.in_cs = in_cs;
  a.in_ns = in_ns;
  a.out_bs = out_bs;
  a.out_cs = out_cs;
  a.out_ns = out_ns;
  a.ncols = ncols;
  a.tiles_per_batch = (ncols + C - 1) / C;
  a.ntiles = a.tiles_per_batch * batches;
  int per_sm = 0, sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.fn, kMixed4Threads, smem) != cudaSuccess ||
      per_sm < 1)
    return FFT_ERR_CUDA;
  const long long resident = (long long)per_sm * sms;
  P.grid = a.ntiles < resident ? a.ntiles : resident;
  P.threads = kMixed4Threads;
  P.smem = (int)smem;
  P.in_role = in_role;
  P.out_role = out_role;
  return FFT_OK;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// The twiddle tables of a plan in one allocation: W_La^m (m < La), W_Lb^m
// (m < Lb; shared when La == Lb), and for a four-step plan the two levels
// of W_N^e, e < N: lo[i] = W_N^i (i < 2^s), hi[j] = W_N^{j 2^s}; then the
// status word.  Entries are FP64 sincospi values (rounded once for FP32).
struct M4Tables {
  const void *wa, *wb, *lo, *hi;
  int s;
};
static int m4_tables(fft_plan* p, long long La, long long Lb, long long Nft, M4Tables* t) {
  const bool fp64 = p->prec == FFT_PREC_FP64;
  const size_t esz = fp64 ? 16 : 8;
  int s = 0;
  long long nlo = 0, nhi = 0;
  if (Nft > 0) {
    int bits = 0;
    while ((1LL << bits) < Nft) ++bits;
    s = (bits + 1) / 2;
    nlo = 1LL << s;
    nhi = ((Nft - 1) >> s) + 1;
  }
  const size_t oa = 0, ob = al256(La * esz);
  const size_t olo = ob + (Lb == La ? 0 : al256(Lb * esz));
  const size_t ohi = olo + al256(nlo * esz);
  const size_t ost = ohi + al256(nhi * esz);
  if (cudaMalloc(&p->d_tables, ost + 256) != cudaSuccess) return FFT_ERR_ALLOC;
  char* base = (char*)p->d_tables;
  t->wa = base + oa;
  t->wb = Lb == La ? t->wa : (const void*)(base + ob);
  t->lo = Nft > 0 ? base + olo : nullptr;
  t->hi = Nft > 0 ? base + ohi : nullptr;
  t->s = s;
  p->d_status = (int*)(base + ost);
  cudaError_t e = launch_gen_twiddles_step(base + oa, fp64, La, La, 1, 0);
  if (e == cudaSuccess && Lb != La) e = launch_gen_twiddles_step(base + ob, fp64, Lb, Lb, 1, 0);
  if (e == cudaSuccess && Nft > 0) e = launch_gen_twiddles_step(base + olo, fp64, Nft, nlo, 1, 0);
  if (e == cudaSuccess && Nft > 0) e = launch_gen_twiddles_step(base + ohi, fp64, Nft, nhi, nlo, 0);
  if (e != cudaSuccess || cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess)
    return FFT_ERR_CUDA;
  return FFT_OK;
}

// N = N1 N2 with N1 the largest divisor of N at most sqrt(N) whose cofactor
// is one on-chip sub-transform; in FP32 the largest such N1 for which both
// lengths have a compiled schedule, when there is one.
int mixed4_plan_1d(fft_plan* p) {
  const bool fp64 = p->prec == FFT_PREC_FP64;
  const long long N = p->n, Lmax = fp64 ? kMixedMaxN64 : kMixedMaxN;
  long long n1 = 0, n1_ct = 0;
  long long d = (long long)std::sqrt((double)N) + 1;
  while (d * d > N) --d;
  for (; d >= 2; --d) {
    if (N % d != 0 || N / d > Lmax) continue;
    if (n1 == 0) n1 = d;
    if (!fp64 && mixed4_ct_lookup(d) && mixed4_ct_lookup(N / d)) {
      n1_ct = d;
      break;
    }
    if (fp64) break;
  }
  if (n1_ct) n1 = n1_ct;
  if (n1 == 0) return FFT_ERR_UNSUPPORTED;
  const long long n2 = N / n1;
  M4Tables t;
  int rc = m4_tables(p, n1, n2, N, &t);
  if (rc) return rc;
  p->kind = KIND_MIXED_PASSES;
  p->m4_n1 = n1;
  p->m4_n2 = n2;
  p->m4n = 2;
  // column pass: C adjacent n2, the length-N1 transform over n1, times W_N^{n2 k1}
  rc = m4_pass_init(p, p->m4[0], n1, n2, p->batch, N, 1, n2, N, 1, n2, t.wa, 0, 2);
  if (rc) return rc;
  p->m4[0].a.ft_lo = t.lo;
  p->m4[0].a.ft_hi = t.hi;
  p->m4[0].a.ft_s = t.s;
  // row pass: C adjacent k1, the length-N2 transform over n2, to X[k1 + N1 k2]
  rc = m4_pass_init(p, p->m4[1], n2, n1, p->batch, N, n2, 1, N, 1, n1, t.wb, 2, 1);
  if (rc) return rc;
  p->ws_bytes = (size_t)N * (size_t)p->batch * (fp64 ? 16 : 8);
  p->launches = 2;
  return FFT_OK;
}

// ny-by-nx images: row transforms (input -> output), then column transforms in
// place in the output.
int mixed4_plan_2d(fft_plan* p) {
  const long long ny = p->ny, nx = p->nx, img = ny * nx;
  M4Tables t;
  int rc = m4_tables(p, nx, ny, 0, &t);
  if (rc) return rc;
  p->kind = KIND_MIXED_PASSES;
  p->m4_n1 = ny;
  p->m4_n2 = nx;
  p->m4n = 2;
  rc = m4_pass_init(p, p->m4[0], nx, ny, p->batch, img, nx, 1, img, nx, 1, t.wa, 0, 1);
  if (rc) return rc;
  rc = m4_pass_init(p, p->m4[1], ny, nx, p->batch, img, 1, nx, img, 1, nx, t.wb, 1, 1);
  if (rc) return rc;
  p->ws_bytes = 0;
  p->launches = 2;
  return FFT_OK;
}

int mixed4_exec(fft_plan* p, const void* in, void* out, int conj, double sx, double sy, int scale_out,
                cudaStream_t s) {
  void* bufs[3] = {(void*)in, out, p->ws};
  for (int i = 0; i < p->m4n; ++i)
    if ((p->m4[i].in_role == 2 || p->m4[i].out_role == 2) && !p->ws) return FFT_ERR_NO_WORKSPACE;
  for (int i = 0; i < p->m4n; ++i) {
    const Mixed4Pass& P = p->m4[i];
    Mixed4Args a = P.a;
    a.m.in = bufs[P.in_role];
    a.m.out = bufs[P.out_role];
    a.m.conj_in = i == 0 ? conj : 0;
    a.m.scale_out = i == p->m4n - 1 ? scale_out : 0;
    a.m.sx = sx;
    a.m.sy = sy;
    a.m.fsx = (float)sx;
    a.m.fsy = (float)sy;
    if (P.grid < 1 || P.grid > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
    void* args[] = {(void*)&a};
    if (cudaLaunchKernel(P.fn, dim3((unsigned)P.grid), dim3(P.threads), args, (size_t)P.smem, s) != cudaSuccess)
      return FFT_ERR_CUDA;
  }
  return FFT_OK;
}

}  // namespace gbfft
