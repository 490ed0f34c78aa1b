// plan.cu -- host-side planner and the C ABI (include/gbfft.h).
//
// The planner maps a request onto the tile kernels:
//   * n <= 2^14: one on-chip pass per transform (paper Sec. 2.3.2: small data
//     need no division; here the bound is GB300's shared memory and register
//     file rather than the C2070's).
//   * n  > 2^14: four-step split N = N1*N2 (Sec. 2.3.2, two exchanges through global memory):
//       pass 1  column FFTs of length N1 over stride N2, each output scaled by
//               W_N^{n2*k1}, written to the workspace as Y[k1][n2];
//       pass 2  row FFTs of length N2 of Y[k1][.], written transposed to
//               X[k1 + N1*k2].
//     From 2^22 the row length N2 is itself split once more (three passes,
//     N = N1*N2*N3), so that every pass's sub-FFT stays at most 2^12 points.
//   * 2-D ny x nx: row FFTs, then column FFTs in place (Sec. 2.3.2: rows,
//     then columns).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_set>

#include "gbfft_internal.h"
#include "tile_registry.h"

using namespace gbfft;

namespace gbfft {

// defined in many.cu / tc.cu
int many_plan_init(fft_plan* p, const int64_t* lengths, int64_t count, const fft_many_config* cfg);
int many_get_config(const fft_plan* p, fft_many_config* out);
int many_resolve_config(const fft_many_config* in, fft_many_config* out);
void many_plan_free(fft_plan* p);
int many_exec(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s);
int tc_plan_init(fft_plan* p);
int tc_exec(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s);
int fused_plan_init(fft_plan* p, int lgN, long long slab_bytes);
void fused_plan_free(fft_plan* p);
bool fused_supported(int lgN);
int fused_exec(fft_plan* p, const float2* in, float2* out, int conj, float sx, float sy, int scale,
               cudaStream_t s);

thread_local int g_last_error = FFT_OK;

int set_err(int code) {
  if (code != FFT_OK) g_last_error = code;
  return code;
}

const TileKernelInfo* tile_kernel(int map, int lg, int C) {
  switch (map) {
    case MAP_JJ:
      return (C == jj_cols(lg)) ? tile_kernel_jj(lg) : nullptr;
    case MAP_CC:
      if (lg <= 7) return tile_kernel_cc_a(lg, C);
      if (lg <= 10) return tile_kernel_cc_b(lg, C);
      return tile_kernel_cc_c(lg, C);
    case MAP_JC:
      if (lg <= 8) return tile_kernel_jc_a(lg, C);
      return tile_kernel_jc_b(lg, C);
  }
  return nullptr;
}

static int ilog2_exact(int64_t v) {
  if (v < 1 || (v & (v - 1)) != 0) return -1;
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

// Planner overrides for tests and measurements (which split, which staging
// kernel, how many passes), read from the environment at plan creation.  Only
// the test build of the library (libgbfft_testhooks.so, -DGBFFT_TEST_HOOKS)
// reads them; in libgbfft.so every override is its default, so no variable of
// the environment changes a production plan (fft_plan_config is the API for
// choosing a configuration).
#ifdef GBFFT_TEST_HOOKS
static int env_int(const char* name, int dflt) {
  const char* s = getenv(name);
  return (s && *s) ? atoi(s) : dflt;
}
#else
static int env_int(const char*, int dflt) { return dflt; }
#endif

static int prepare_kernel(const TileKernelInfo* k) {
  if (!k) return FFT_ERR_UNSUPPORTED;
  if (k->smem_bytes > 48 * 1024) {
    if (cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k->smem_bytes) != cudaSuccess)
      return FFT_ERR_CUDA;
  }
  return FFT_OK;
}

// Columns per CTA for a column (c-fast) pass of length 2^lg: as many adjacent
// columns as fit a 2^13-point tile (64 KB), at most 16.
static int default_cols(int lg) {
  int c = (1 << 13) >> lg;
  if (c < 1) c = 1;
  if (c > 16) c = 16;
  return c;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Allocates and fills the plan's twiddle tables in one device buffer: stage
// tables for up to three lengths (lgs[i] > 0) and two-level W_N tables for up
// to two four-step levels (lgNs[i] > 0).  Also the device status word.
static int build_tables_multi(fft_plan* p, const int lgs[3], const int lgNs[2]) {
  size_t off = 0, stage_off[3], lo_off[2], hi_off[2];
  size_t lo_n[2] = {0, 0}, hi_n[2] = {0, 0};
  int ss[2] = {0, 0};
  for (int i = 0; i < 3; ++i) {
    stage_off[i] = off;
    off += align256((lgs[i] > 0 ? (size_t)stage_tw_size(lgs[i]) : 0) * 8 + 8);
  }
  for (int i = 0; i < 2; ++i) {
    if (lgNs[i] > 0) {
      ss[i] = (lgNs[i] + 1) / 2;
      lo_n[i] = (size_t)1 << ss[i];
      hi_n[i] = (size_t)1 << (lgNs[i] - ss[i]);
    }
    lo_off[i] = off;
    off += align256(lo_n[i] * 8 + 8);
    hi_off[i] = off;
    off += align256(hi_n[i] * 8 + 8);
  }
  const size_t st_off = off;
  off += 256;
  char* base = nullptr;
  if (cudaMalloc(&base, off) != cudaSuccess) return FFT_ERR_ALLOC;
  p->d_tables = base;
  p->tw1 = (const float2*)(base + stage_off[0]);
  p->tw2 = (const float2*)(base + stage_off[1]);
  p->tw3 = (const float2*)(base + stage_off[2]);
  p->ft_lo = (const float2*)(base + lo_off[0]);
  p->ft_hi = (const float2*)(base + hi_off[0]);
  p->ft_s = ss[0];
  p->ft2_lo = (const float2*)(base + lo_off[1]);
  p->ft2_hi = (const float2*)(base + hi_off[1]);
  p->ft2_s = ss[1];
  p->d_status = (int*)(base + st_off);
  cudaStream_t s = 0;
  if (cudaMemsetAsync(p->d_status, 0, sizeof(int), s) != cudaSuccess) return FFT_ERR_CUDA;
  const float2* st[3] = {p->tw1, p->tw2, p->tw3};
  for (int i = 0; i < 3; ++i)
    if (lgs[i] > 0 && launch_gen_stage_twiddles((float2*)st[i], lgs[i], s) != cudaSuccess) return FFT_ERR_CUDA;
  const float2* los[2] = {p->ft_lo, p->ft2_lo};
  const float2* his[2] = {p->ft_hi, p->ft2_hi};
  for (int i = 0; i < 2; ++i) {
    if (lgNs[i] <= 0) continue;
    if (launch_gen_power_twiddles((float2*)los[i], lgNs[i], (long long)lo_n[i], 1, s) != cudaSuccess ||
        launch_gen_power_twiddles((float2*)his[i], lgNs[i], (long long)hi_n[i], (long long)lo_n[i], s) !=
            cudaSuccess)
      return FFT_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return FFT_ERR_CUDA;
  return FFT_OK;
}

static int build_tables(fft_plan* p, int lgA, int lgB, int lgN) {
  const int lgs[3] = {lgA, lgB, 0};
  const int lgNs[2] = {lgN, 0};
  return build_tables_multi(p, lgs, lgNs);
}

static fft_plan* new_plan() {
  fft_plan* p = new (std::nothrow) fft_plan;
  if (!p) return nullptr;
  memset(p, 0, sizeof(*p));
  cudaGetDevice(&p->device);
  return p;
}

static void free_plan(fft_plan* p) {
  if (!p) return;
  if (p->inner) free_plan(p->inner);
  if (p->d_rtw) cudaFree(p->d_rtw);
  if (p->many) many_plan_free(p);
  if (p->fused) fused_plan_free(p);
  if (p->ws_owned && p->ws) cudaFree(p->ws);
  if (p->d_tc) cudaFree(p->d_tc);
  if (p->d_rctw) cudaFree(p->d_rctw);
  if (p->d_radtw) cudaFree(p->d_radtw);
  if (p->d_tables) cudaFree(p->d_tables);
  delete p;
}

static bool valid_dir(int dir) { return dir >= 0 && dir <= 3; }
static bool valid_prec(int prec) { return prec >= FFT_PREC_FP32 && prec <= FFT_PREC_FP64; }
static bool tc_prec(int prec) { return prec >= FFT_PREC_TC_BF16 && prec <= FFT_PREC_TC_FP16_SPLIT; }

// Direction -> load/store transform: conjugate direction via conj in/out,
// 1/N of Eq. 2 folded into the store.
struct DirXf {
  int conj;
  float scale;
};
static DirXf dir_xf(int dir, int64_t n) {
  const int inv = dir & FFT_INVERSE;
  const int adj = (dir & FFT_ADJOINT) ? 1 : 0;
  DirXf x;
  x.conj = inv ^ adj;
  x.scale = inv ? (float)(1.0 / (double)n) : 1.0f;
  return x;
}

static void base_args(TileArgs& a) {
  memset(&a, 0, sizeof(a));
  a.stream_in = 1;
  a.stream_out = 1;
}

static int launch_tile(const TileKernelInfo* k, const TileArgs& a, long long ntiles, cudaStream_t s) {
  if (ntiles <= 0) return FFT_OK;
  if (ntiles > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
  void* args[] = {(void*)&a};
  cudaError_t e = cudaLaunchKernel(k->fn, dim3((unsigned)ntiles), dim3(k->threads), args, (size_t)k->smem_bytes, s);
  return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

static void set_out_xf(TileArgs& a, const DirXf& x) {
  a.scale_out = (x.conj || x.scale != 1.0f) ? 1 : 0;
  a.sx = x.scale;
  a.sy = x.conj ? -x.scale : x.scale;
}

// ---- single on-chip pass -------------------------------------------------
static int exec_single(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s) {
  const DirXf x = dir_xf(dir, p->n);
  if (p->kdif2) {
    // two CTAs per transform: (b, k1) computes outputs k1, k1 + 2, ...
    TileArgs a;
    base_args(a);
    a.in = in;
    a.out = out;
    a.tw = p->tw2;  // stage table of the half length
    a.in_bstride = a.out_bstride = p->n;
    a.in_sn = 1;
    a.out_sn = 2;
    a.ncols = 1;
    a.pre_half = p->n / 2;
    a.pre_tw = p->pre_tw;
    a.conj_in = x.conj;
    set_out_xf(a, x);
    return launch_tile(p->kdif2, a, 2 * p->batch, s);
  }
  if (p->ktma && ((uintptr_t)in & 15) == 0) {
    // persistent TMA-staged kernel: grid = resident CTAs, tiles looped
    TileArgs a;
    base_args(a);
    const int C = p->ktma->C;
    a.in = in;
    a.out = out;
    a.tw = p->tw1;
    a.ncols = p->batch;
    a.conj_in = x.conj;
    set_out_xf(a, x);
    long long ntiles = (p->batch + C - 1) / C;
    long long grid = p->tma_grid < ntiles ? p->tma_grid : ntiles;
    int* st = p->d_status;
    void* args[] = {(void*)&a, (void*)&ntiles, (void*)&st};
    cudaError_t e = cudaLaunchKernel(p->ktma->fn, dim3((unsigned)grid), dim3(p->ktma->threads), args,
                                     (size_t)p->ktma->smem_bytes, s);
    return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
  }
  TileArgs a;
  base_args(a);
  const TileKernelInfo* k = p->kradix ? p->kradix : p->k1;
  const int C = k->C;
  const long long L = p->n;
  a.in = in;
  a.out = out;
  a.tw = p->kradix ? (const float2*)p->d_radtw : p->tw1;
  a.tiles_per_batch = (p->batch + C - 1) / C;
  a.in_gstride = a.out_gstride = (long long)C * L;
  a.in_sc = a.out_sc = L;
  a.in_sn = a.out_sn = 1;
  a.ncols = p->batch;
  a.conj_in = x.conj;
  set_out_xf(a, x);
  if (p->kpfs && ((uintptr_t)in & 15) == 0) {
    // bulk copies need a 16-byte aligned source (rows are L * 8 bytes apart)
    long long ntiles = a.tiles_per_batch;
    const long long grid = p->pf_grid < ntiles ? p->pf_grid : ntiles;
    int* st = p->d_status;
    void* args[] = {(void*)&a, (void*)&ntiles, (void*)&st};
    return cudaLaunchKernel(p->kpfs->fn, dim3((unsigned)grid), dim3(p->kpfs->threads), args,
                            (size_t)p->kpfs->smem_bytes, s) == cudaSuccess
               ? FFT_OK
               : FFT_ERR_CUDA;
  }
  if (p->kpf) {
    long long ntiles = a.tiles_per_batch;
    const long long grid = p->pf_grid < ntiles ? p->pf_grid : ntiles;
    void* args[] = {(void*)&a, (void*)&ntiles};
    return cudaLaunchKernel(p->kpf->fn, dim3((unsigned)grid), dim3(p->kpf->threads), args,
                            (size_t)p->kpf->smem_bytes, s) == cudaSuccess
               ? FFT_OK
               : FFT_ERR_CUDA;
  }
  return launch_tile(k, a, a.tiles_per_batch, s);
}

// Attach the tensor-TMA variant to every column pass that has one, when
// asked for (config tma = 1, the default of FP32 1-D multi-pass plans;
// GBFFT_COLTMA=1 / 0 forces it on / off).  Measured on GB300 once the column
// tiles' step table stopped conflicting in shared memory, it is the faster
// column pass at every multi-pass length (autotuner: 2^16 395 -> 328 us,
// 2^20 499 -> 427, 2^24 639 -> 514, 2^26 690 -> 580 per 2^26 points).
// Whether a given exec can use it (alignment, strides) is decided per call.
// The last pass of a multi-pass 1-D plan, when it is a row pass with a
// TMA-store variant (row_tmas.cu).
static int attach_rowtmas(fft_plan* p) {
  if (env_int("GBFFT_ROWTMAS", 1) == 0) return FFT_OK;
  PassDesc& d = p->pass[p->npass - 1];
  if (!d.k || d.k->map != MAP_JC || d.k->lg > 11) return FFT_OK;
  const TileKernelInfo* k = tile_kernel_rowtmas(d.k->lg, d.k->C);
  if (!k) return FFT_OK;
  const int rc = prepare_kernel(k);
  if (rc) return rc;
  d.kst = k;
  return FFT_OK;
}

static int attach_coltma(fft_plan* p, bool want) {
  const int env = env_int("GBFFT_COLTMA", -1);
  if (env >= 0) want = env > 0;
  if (!want) return FFT_OK;
  for (int i = 0; i < p->npass; ++i) {
    PassDesc& d = p->pass[i];
    if (d.k->map != MAP_CC) continue;
    const TileKernelInfo* kc = tile_kernel_coltma(d.k->lg, d.k->C);
    if (!kc) continue;
    int rc = prepare_kernel(kc);
    if (rc) return rc;
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc->fn, kc->threads, (size_t)kc->smem_bytes) !=
            cudaSuccess ||
        per_sm < 1)
      return FFT_ERR_CUDA;
    d.kcol = kc;
    d.col_grid = per_sm * sms;
  }
  return FFT_OK;
}

// ---- multi-pass plans: run the pass list ------------------------------------
static int exec_passes(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s) {
  const DirXf x = dir_xf(dir, p->n);
  float2* roles[3] = {(float2*)in, out, (float2*)p->ws};
  for (int i = 0; i < p->npass; ++i) {
    const PassDesc& d = p->pass[i];
    if ((d.in_role == 2 || d.out_role == 2) && !p->ws) return FFT_ERR_NO_WORKSPACE;
    TileArgs a = d.a;
    a.in = roles[d.in_role];
    a.out = roles[d.out_role];
    if (i == 0) a.conj_in = x.conj;
    if (i == p->npass - 1) set_out_xf(a, x);
    int rc;
    if (d.kpfs && ((uintptr_t)a.in & 15) == 0) {
      // contiguous rows, one per CTA in turn; the bulk copies need a 16-byte aligned source
      long long ntiles = d.ntiles;
      const long long grid = d.pf_grid < ntiles ? d.pf_grid : ntiles;
      int* st = p->d_status;
      void* args[] = {(void*)&a, (void*)&ntiles, (void*)&st};
      rc = cudaLaunchKernel(d.kpfs->fn, dim3((unsigned)grid), dim3(d.kpfs->threads), args,
                            (size_t)d.kpfs->smem_bytes, s) == cudaSuccess
               ? FFT_OK
               : FFT_ERR_CUDA;
    } else if (d.kcol && coltma_usable(d.kcol, a, a.in))
      rc = coltma_launch(d.kcol, a, d.ntiles, d.col_grid, p->d_status, s);
    else if (d.kst && rowtmas_usable(d.kst, a, a.out, d.ntiles))
      rc = rowtmas_launch(d.kst, a, d.ntiles, s);
    else
      rc = launch_tile(d.k, a, d.ntiles, s);
    if (rc) return rc;
  }
  return FFT_OK;
}

// ---- range compression (fast convolution with a frequency-domain filter) --
// One-pass lengths: the fused kernel, one read and one write per value.
// Multi-pass plans: the passes run twice.  The first run is the forward
// transform whose last (row) pass stores conj(H X); the second is a forward
// transform of that, conjugated and scaled by 1/N on its last store, which is
// Eq. 2 applied to H X.  `out` holds the intermediate.
static int exec_filter_plan(fft_plan* p, const float2* in, float2* out, const float2* filt, int conj_filt,
                            cudaStream_t s) {
  if (p->prec != FFT_PREC_FP32) return FFT_ERR_UNSUPPORTED;
  const float inv_n = (float)(1.0 / (double)p->n);
  if (p->kind == KIND_SINGLE) {
    if (!p->krc) return FFT_ERR_UNSUPPORTED;
    TileArgs a;
    base_args(a);
    const int C = p->krc->C;
    const long long L = p->n;
    a.in = in;
    a.out = out;
    a.tw = p->tw1;
    a.tiles_per_batch = (p->batch + C - 1) / C;
    a.in_gstride = a.out_gstride = (long long)C * L;
    a.in_sc = a.out_sc = L;
    a.in_sn = a.out_sn = 1;
    a.ncols = p->batch;
    a.tw_rev = p->d_rctw ? (const float2*)p->d_rctw : p->tw1;
    a.filt = filt;
    a.filt_mask = L - 1;
    a.filt_conj = conj_filt;
    a.scale_out = 1;
    a.sx = inv_n;
    a.sy = -inv_n;
    long long ntiles = a.tiles_per_batch;
    const long long grid = (p->rc_grid > 0 && p->rc_grid < ntiles) ? p->rc_grid : ntiles;
    if (grid > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
    void* args[] = {(void*)&a, (void*)&ntiles};
    return cudaLaunchKernel(p->krc->fn, dim3((unsigned)grid), dim3(p->krc->threads), args,
                            (size_t)p->krc->smem_bytes, s) == cudaSuccess
               ? FFT_OK
               : FFT_ERR_CUDA;
  }
  if (p->kind != KIND_FOURSTEP || p->fused || p->npass < 2) return FFT_ERR_UNSUPPORTED;
  if (p->pass[p->npass - 1].k->map != MAP_JC) return FFT_ERR_UNSUPPORTED;
  float2* roles[3] = {(float2*)in, out, (float2*)p->ws};
  for (int run = 0; run < 2; ++run) {
    if (run == 1) roles[0] = out;
    for (int i = 0; i < p->npass; ++i) {
      const PassDesc& d = p->pass[i];
      if ((d.in_role == 2 || d.out_role == 2) && !p->ws) return FFT_ERR_NO_WORKSPACE;
      TileArgs a = d.a;
      a.in = roles[d.in_role];
      a.out = roles[d.out_role];
      if (i == 0) a.conj_in = 0;
      if (i == p->npass - 1) {
        a.scale_out = 1;
        if (run == 0) {
          a.filt = filt;
          a.filt_mask = p->n - 1;
          a.filt_conj = conj_filt;
          a.sx = 1.0f;
          a.sy = -1.0f;
        } else {
          a.sx = inv_n;
          a.sy = -inv_n;
        }
      }
      const int rc = (d.kcol && coltma_usable(d.kcol, a, a.in))
                         ? coltma_launch(d.kcol, a, d.ntiles, d.col_grid, p->d_status, s)
                         : launch_tile(d.k, a, d.ntiles, s);
      if (rc) return rc;
    }
  }
  return FFT_OK;
}

int exec_plan(fft_plan* p, const void* in, void* out, int dir, cudaStream_t s);

// ---- real-data transforms (KIND_REAL): N = 2M reals per row ----------------
// FP64 real-data plans: the complex128 plan and the FP64 split kernels.
static int exec_real64(fft_plan* p, const void* in, void* out, bool to_complex, bool adj, cudaStream_t s) {
  const long long M = p->n / 2;
  if (!p->inner || !p->zbuf) return FFT_ERR_NO_WORKSPACE;
  const double2* lo = (const double2*)p->r_lo;
  const double2* hi = (const double2*)p->r_hi;
  double2* z = (double2*)p->zbuf;
  if (to_complex) {
    const int rc = exec_plan(p->inner, in, z, FFT_FORWARD, s);
    if (rc) return rc;
    const double s_int = adj ? 1.0 / (double)M : 1.0, s_end = adj ? 0.5 / (double)M : 1.0;
    return launch_r2c_split64(z, (double2*)out, M, p->batch, lo, hi, p->r_s, s_int, s_end, s) == cudaSuccess
               ? FFT_OK
               : FFT_ERR_CUDA;
  }
  if (launch_c2r_split64((const double2*)in, z, M, p->batch, lo, hi, p->r_s, adj ? 2.0 : 1.0, s) != cudaSuccess)
    return FFT_ERR_CUDA;
  return exec_plan(p->inner, z, out, adj ? FFT_ADJOINT : FFT_INVERSE, s);
}

static int exec_real(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s) {
  if (dir < 0 || dir > (FFT_INVERSE | FFT_ADJOINT)) return FFT_ERR_INVALID_ARG;
  if ((const void*)in == (const void*)out) return FFT_ERR_INVALID_ARG;
  if (p->prec == FFT_PREC_FP64)
    return exec_real64(p, in, out, dir == FFT_FORWARD || dir == (FFT_INVERSE | FFT_ADJOINT),
                       (dir & FFT_ADJOINT) != 0, s);
  const long long M = p->n / 2;
  // Real rows in, complex rows out: the transform (FFT_FORWARD) and the adjoint
  // of the complex-to-real transform (FFT_INVERSE | FFT_ADJOINT), which is the
  // same split with the interior outputs times 2/N and X[0], X[M] times 1/N.
  // Complex rows in, real rows out: the inverse (FFT_INVERSE, 1/N) and the
  // adjoint of the real-to-complex transform (FFT_ADJOINT), which doubles the
  // real parts of X[0] and X[M] and drops the 1/N.
  const bool to_complex = dir == FFT_FORWARD || dir == (FFT_INVERSE | FFT_ADJOINT);
  const bool adj = (dir & FFT_ADJOINT) != 0;
  const float s_int = adj ? (float)(1.0 / (double)M) : 1.0f;   // 2/N
  const float s_end = adj ? (float)(0.5 / (double)M) : 1.0f;   // 1/N
  if (p->kr2c) {
    const TileKernelInfo* k = to_complex ? p->kr2c : p->kc2r;
    const int C = k->C;
    TileArgs a;
    base_args(a);
    a.in = in;
    a.out = out;
    a.tw = p->tw1;
    a.tiles_per_batch = (p->batch + C - 1) / C;
    a.ncols = p->batch;
    a.r_w = p->r_lo;   // one-level table W_N^k, k < M
    a.in_sn = a.out_sn = 1;
    if (to_complex) {
      // rows of M complex (2M reals) in, rows of M + 1 complex out
      a.in_gstride = (long long)C * M;
      a.in_sc = M;
      a.out_gstride = (long long)C * (M + 1);
      a.out_sc = M + 1;
      if (adj) {
        a.scale_out = 1;
        a.sx = s_int;
        a.sy = s_end;
      }
    } else {
      a.in_gstride = (long long)C * (M + 1);
      a.in_sc = M + 1;
      a.out_gstride = (long long)C * M;
      a.out_sc = M;
      a.conj_in = 1;
      a.scale_out = 1;
      a.sx = adj ? 1.0f : (float)(1.0 / (double)M);
      a.sy = -a.sx;
      a.r_end2 = adj ? 1 : 0;
    }
    return launch_tile(k, a, a.tiles_per_batch, s);
  }
  if (!p->inner || !p->zbuf) return FFT_ERR_NO_WORKSPACE;
  if (to_complex && p->krfold) {
    // column pass of the inner plan into its workspace, then the row pass with
    // the split folded in (rows k1 and N1 - k1 in one tile)
    const fft_plan* q = p->inner;
    if (!q->ws) return FFT_ERR_NO_WORKSPACE;
    const PassDesc& A = q->pass[0];
    TileArgs a = A.a;
    a.in = in;
    a.out = (float2*)q->ws;
    const int rc = (A.kcol && coltma_usable(A.kcol, a, a.in))
                       ? coltma_launch(A.kcol, a, A.ntiles, A.col_grid, q->d_status, s)
                       : launch_tile(A.k, a, A.ntiles, s);
    if (rc) return rc;
    TileArgs b = q->pass[1].a;
    b.in = (const float2*)q->ws;
    b.out = out;
    return r2c_fold_launch(p->krfold, b, M, 1 << q->lg1, p->batch, p->r_lo, p->r_hi, p->r_s, adj ? 1 : 0, s_int,
                           s_end, s);
  }
  if (!to_complex && p->kcfold) {
    // the inner plan's column pass with the split folded in, reading the rows
    // of M + 1 values, then its row pass
    const fft_plan* q = p->inner;
    if (!q->ws) return FFT_ERR_NO_WORKSPACE;
    const PassDesc& A = q->pass[0];
    TileArgs a = A.a;
    a.in = in;
    a.out = (float2*)q->ws;
    a.in_bstride = M + 1;
    a.r_w = p->r_lo;
    a.r_hi = p->r_hi;
    a.r_s = p->r_s;
    a.r_end2 = adj ? 1 : 0;
    a.conj_in = 1;   // the inverse as conj(F(conj Z))
    int rc = launch_tile(p->kcfold, a, A.ntiles, s);
    if (rc) return rc;
    const PassDesc& B = q->pass[1];
    TileArgs b = B.a;
    b.in = (const float2*)q->ws;
    b.out = out;
    b.scale_out = 1;
    b.sx = adj ? 1.0f : (float)(1.0 / (double)M);
    b.sy = -b.sx;
    if (B.kst && rowtmas_usable(B.kst, b, b.out, B.ntiles)) return rowtmas_launch(B.kst, b, B.ntiles, s);
    return launch_tile(B.k, b, B.ntiles, s);
  }
  if (to_complex) {
    const int rc = exec_plan(p->inner, in, p->zbuf, FFT_FORWARD, s);
    if (rc) return rc;
    return launch_r2c_split(p->zbuf, out, M, p->batch, p->r_lo, p->r_hi, p->r_s, s_int, s_end, s) == cudaSuccess
               ? FFT_OK
               : FFT_ERR_CUDA;
  }
  if (launch_c2r_split(in, p->zbuf, M, p->batch, p->r_lo, p->r_hi, p->r_s, adj ? 2.0f : 1.0f, s) != cudaSuccess)
    return FFT_ERR_CUDA;
  return exec_plan(p->inner, p->zbuf, out, adj ? FFT_ADJOINT : FFT_INVERSE, s);
}

int exec_plan(fft_plan* p, const void* in, void* out, int dir, cudaStream_t s) {
  if (!p || !in || !out || !valid_dir(dir)) return FFT_ERR_INVALID_ARG;
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7)) return FFT_ERR_ALIGN;
  const float2* fin = (const float2*)in;
  float2* fout = (float2*)out;
  int rc;
  if (p->prec == FFT_PREC_FP64 && (((uintptr_t)in & 15) || ((uintptr_t)out & 15))) return FFT_ERR_ALIGN;
  if (tc_prec(p->prec) && p->kind != KIND_MANY) {
    rc = tc_exec(p, fin, fout, dir, s);
  } else {
    switch (p->kind) {
      case KIND_SINGLE: rc = exec_single(p, fin, fout, dir, s); break;
      case KIND_FOURSTEP:
        if (p->fused) {
          const DirXf x = dir_xf(dir, p->n);
          rc = fused_exec(p, fin, fout, x.conj, x.scale, x.conj ? -x.scale : x.scale,
                          (x.conj || x.scale != 1.0f) ? 1 : 0, s);
          break;
        }
        rc = exec_passes(p, fin, fout, dir, s);
        break;
      case KIND_2D: rc = exec_passes(p, fin, fout, dir, s); break;
      case KIND_MANY: rc = many_exec(p, fin, fout, dir, s); break;
      case KIND_REAL: rc = exec_real(p, fin, fout, dir, s); break;
      case KIND_MIXED:
      case KIND_MIXED_PASSES: {
        const DirXf x = dir_xf(dir, p->n);
        const double sc = (dir & FFT_INVERSE) ? 1.0 / (double)p->n : 1.0;
        const int so = (x.conj || sc != 1.0) ? 1 : 0;
        rc = p->kind == KIND_MIXED ? mixed_exec(p, in, out, x.conj, sc, x.conj ? -sc : sc, so, s)
                                   : mixed4_exec(p, in, out, x.conj, sc, x.conj ? -sc : sc, so, s);
        break;
      }
      default: rc = FFT_ERR_INVALID_ARG;
    }
  }
  if (rc == FFT_OK && cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    rc = FFT_ERR_CUDA;
  }
  return rc;
}

// Planner for 1-D lengths: kind, split and kernel variants.  cfg fields <= 0
// (or tma < 0) take the defaults: one on-chip pass up to 2^14 (radix-8 passes
// at 2^5 and 2^6, TMA-staged for 2^9..2^11, persistent with the next transform
// staged into the exchange buffer at 2^13 and 2^14), two passes
// below 2^22 (2^8-point column tiles from 2^16 to 2^20, else the even split),
// three passes 2^8 * 2^8 * rest from 2^22; as many adjacent columns per CTA
// as fit 2^13 points (at most 16).
static int plan_1d(fft_plan* p, int lgN, const fft_plan_config* cfg) {
  fft_plan_config dflt;
  memset(&dflt, 0, sizeof(dflt));
  dflt.tma = -1;
  dflt.fused = -1;
  dflt.halves = 0;
  if (!cfg) cfg = &dflt;
  // radix 4 / 8: one on-chip FP32 pass on the register path only, where a
  // kernel is compiled (checked before any CUDA call).  Left open by the
  // configuration, the planner takes radix-8 passes at 2^5 and 2^6, where
  // they measured faster on GB300 than radix 16 (per 2^26 points: 2^5 224 ->
  // 176 us, 2^6 162 -> 158 us; bench.py --workload radix).
  const bool open_kernel = cfg->radix <= 0 && cfg->npass <= 1 && cfg->tma < 0 && cfg->fused <= 0 &&
                           cfg->halves != 2 && p->prec == FFT_PREC_FP32;
  const int radix = cfg->radix > 0 ? cfg->radix : ((open_kernel && (lgN == 5 || lgN == 6)) ? 8 : 16);
  const bool small_radix = radix != 16;
  if (small_radix && ((radix != 4 && radix != 8) || cfg->npass > 1 || cfg->tma > 0 || cfg->fused > 0 ||
                      cfg->halves == 2 || p->prec != FFT_PREC_FP32 || !tile_kernel_radix(lgN, radix == 8 ? 3 : 2)))
    return FFT_ERR_UNSUPPORTED;
  // fused two-pass launch (fused.cu): only on request (config or
  // GBFFT_FUSED=1) or when the autotuner measures it faster.  Measured on
  // GB300 it keeps the intermediate in L2 (DRAM reads = input only) but loses
  // to the single pass and to separate launches, because its 4096-point tiles
  // are bound by per-tile latency and issue, not by DRAM traffic.
  const int env_fused = env_int("GBFFT_FUSED", -1);
  const bool default_fused = false;
  const bool want_fused = fused_supported(lgN) && p->prec == FFT_PREC_FP32 &&
                          (cfg->fused > 0 || (cfg->fused < 0 && (env_fused >= 0 ? env_fused > 0 : default_fused)));
  if (want_fused) {
    p->kind = KIND_FOURSTEP;
    p->npass = 2;
    const int lg1 = lgN / 2, lg2 = lgN - lgN / 2;
    int rc = build_tables(p, lg1, lg2, lgN);
    if (rc) return rc;
    return fused_plan_init(p, lgN, (long long)env_int("GBFFT_SLAB_MB", 16) << 20);
  }
  if (lgN <= 14 && cfg->npass <= 1) {
    p->kind = KIND_SINGLE;
    p->lg = p->lg1 = lgN;
    p->k1 = tile_kernel(MAP_JJ, lgN, jj_cols(lgN));
    p->c1 = p->k1 ? p->k1->C : 0;
    p->launches = 1;
    int rc = prepare_kernel(p->k1);
    if (rc) return rc;
    if (p->prec == FFT_PREC_FP32) {
      p->krc = tile_kernel_rc(lgN);
      rc = prepare_kernel(p->krc);
      if (rc) return rc;
      if (rc_persistent(lgN)) {
        int per_sm = 0, sms = 0, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->krc->fn, p->krc->threads,
                                                          (size_t)p->krc->smem_bytes) != cudaSuccess ||
            per_sm < 1)
          return FFT_ERR_CUDA;
        p->rc_grid = (long long)per_sm * sms;
      }
      if (lgN % 4 != 0 && lgN > 4) {
        // the fused kernel's second transform runs the remainder pass last
        if (cudaMalloc(&p->d_rctw, (size_t)stage_tw_size(lgN, true) * 8) != cudaSuccess) return FFT_ERR_ALLOC;
        if (launch_gen_stage_twiddles((float2*)p->d_rctw, lgN, 0, true) != cudaSuccess ||
            cudaStreamSynchronize(0) != cudaSuccess)
          return FFT_ERR_CUDA;
      }
    }
    // Radix-8 / radix-4 passes with 8 / 4 points per thread (autotuner
    // option): more, lighter threads and more passes over shared memory.
    if (small_radix) {
      const int lgm = radix == 8 ? 3 : 2;
      p->kradix = tile_kernel_radix(lgN, lgm);
      rc = prepare_kernel(p->kradix);
      if (rc) return rc;
      p->radix_lgm = lgm;
      const size_t nt = (size_t)stage_tw_size(lgN, false, lgm);
      if (cudaMalloc(&p->d_radtw, nt * 8 + 8) != cudaSuccess) return FFT_ERR_ALLOC;
      if (launch_gen_stage_twiddles((float2*)p->d_radtw, lgN, 0, false, lgm) != cudaSuccess ||
          cudaStreamSynchronize(0) != cudaSuccess)
        return FFT_ERR_CUDA;
      return build_tables(p, lgN, 0, 0);
    }
    // Two CTAs per transform (radix-2 split) is an autotuner option: with the
    // linear shared-memory addressing the one-CTA pass measures faster at
    // 2^12..2^14 on GB300.  Persistent TMA staging pays where several CTAs
    // share an SM and the tile amortises the copy (measured: 2^9..2^11; at
    // 2^12 the register path is as fast).
    const int env_halves = env_int("GBFFT_HALVES", 0);
    const bool dflt_halves = env_halves == 2;
    const bool want_dif2 = (cfg->halves == 2 || (cfg->halves == 0 && cfg->tma < 0 && dflt_halves)) &&
                           p->prec == FFT_PREC_FP32 && tile_kernel_dif2(lgN - 1);
    if (want_dif2) {
      p->kdif2 = tile_kernel_dif2(lgN - 1);
      rc = prepare_kernel(p->kdif2);
      if (rc) return rc;
      const int lgs[3] = {lgN, lgN - 1, 0};
      const int lgNs[2] = {0, 0};
      rc = build_tables_multi(p, lgs, lgNs);
      if (rc) return rc;
      // W_N^n, n < N/2, in the first stage-table slot's place is not enough:
      // allocate it beside the plan tables
      void* t = nullptr;
      if (cudaMalloc(&t, (size_t)(1LL << (lgN - 1)) * 8) != cudaSuccess) return FFT_ERR_ALLOC;
      p->d_tc = t;  // freed with the plan
      p->pre_tw = (const float2*)t;
      if (launch_gen_power_twiddles((float2*)t, lgN, 1LL << (lgN - 1), 1, 0) != cudaSuccess ||
          cudaStreamSynchronize(0) != cudaSuccess)
        return FFT_ERR_CUDA;
      return FFT_OK;
    }
    // Persistent register path with an L2 prefetch of the next transform:
    // measured on GB300 it pays where one CTA fills an SM (2^14: 279 -> 248
    // us per 2^26 points), not at 2^13 (two CTAs per SM already overlap)
    // nor at 2^12 (its loop costs a resident CTA).
    // tma = 3 (the default at 2^13 and 2^14): the same loop, with the next
    // transform brought into the exchange buffer by a bulk copy issued once
    // the last pass has read it (measured on GB300 per 2^26 points: 2^14 248
    // -> 242 us, 2^13 241 -> 228 us; no change at 2^12).
    const int env_pf = env_int("GBFFT_PF", -1);
    const bool dflt_pf = env_pf >= 0 ? env_pf > 0 : (lgN == 13 || lgN == 14);
    const bool want_pf = tile_kernel_pf(lgN) && p->prec == FFT_PREC_FP32 && cfg->halves != 2 &&
                         (cfg->tma == 2 || cfg->tma == 3 || (cfg->tma < 0 && dflt_pf));
    if (want_pf) {
      p->kpf = tile_kernel_pf(lgN);
      rc = prepare_kernel(p->kpf);
      if (rc) return rc;
      if (cfg->tma == 3 || (cfg->tma < 0 && (env_pf < 0 || env_pf == 3))) {
        p->kpfs = tile_kernel_pfs(lgN);
        rc = prepare_kernel(p->kpfs);
        if (rc) return rc;
      }
      int per_sm = 0, sms = 0, dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->kpfs ? p->kpfs->fn : p->kpf->fn, p->kpf->threads,
                                                        (size_t)(p->kpfs ? p->kpfs->smem_bytes : p->kpf->smem_bytes)) !=
              cudaSuccess ||
          per_sm < 1)
        return FFT_ERR_CUDA;
      p->pf_grid = (long long)per_sm * sms;
      return build_tables(p, lgN, 0, 0);
    }
    const bool want_tma =
        cfg->tma < 0 ? (lgN >= 9 && lgN <= 11 && !env_int("GBFFT_NO_TMA", 0)) : (cfg->tma > 0 && lgN >= 1);
    if (want_tma) {
      p->ktma = tile_kernel_tma(lgN);
      rc = prepare_kernel(p->ktma);
      if (rc) return rc;
      int per_sm = 0, sms = 0, dev = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->ktma->fn, p->ktma->threads,
                                                        (size_t)p->ktma->smem_bytes) != cudaSuccess ||
          per_sm < 1)
        return FFT_ERR_CUDA;
      p->tma_grid = (long long)per_sm * sms;
    }
    return build_tables(p, lgN, 0, 0);
  }
  p->kind = KIND_FOURSTEP;
  // measured on GB300 (autotuner): three passes 2^8 * 2^8 * rest from 2^22 up
  int npass = cfg->npass >= 2 ? cfg->npass : ((lgN >= 22) ? 3 : 2);
  const int force_np = env_int("GBFFT_PASSES", 0);
  if (cfg->npass < 2 && (force_np == 2 || force_np == 3)) npass = force_np;
  if (npass == 3 && lgN < 3) return FFT_ERR_UNSUPPORTED;
  if (p->prec != FFT_PREC_FP32) npass = 2;  // tensor-core kernels are compiled for two-pass splits
  if (npass == 2 && lgN > 28) return FFT_ERR_UNSUPPORTED;
  if (npass == 2) {
    // measured on GB300 (autotuner, per 2^26 points): rows of 2^10 or 2^11
    // points, whose row pass stores by tensor TMA, from 2^17 (2^7 x 2^10:
    // 336 us against 375 for 2^8 x 2^9; 2^20 = 2^10 x 2^10: 419 against 436
    // for 2^8 x 2^12); 2^8 x 2^8 at 2^16; beyond 2^20, the even split
    // (tensor-core plans keep the even split their kernels are compiled for)
    const bool fp32 = p->prec == FFT_PREC_FP32;
    static const int kLg2Default[5] = {8, 10, 10, 11, 10};   // lgN = 16..20
    int lg2 = (fp32 && lgN >= 16 && lgN <= 20) ? kLg2Default[lgN - 16] : (lgN + 1) / 2;
    const int force_lg1 = cfg->lg1 > 0 ? cfg->lg1 : env_int("GBFFT_FORCE_SPLIT", 0);
    if (force_lg1 > 0 && force_lg1 < lgN && lgN - force_lg1 <= 14 && force_lg1 <= 14) lg2 = lgN - force_lg1;
    const int lg1 = lgN - lg2;
    if (lg1 > 14 || lg2 > 14 || lg1 < 1 || lg2 < 1) return FFT_ERR_UNSUPPORTED;
    p->lg1 = lg1;
    p->lg2 = lg2;
    p->c1 = cfg->c1 > 0 ? cfg->c1 : env_int("GBFFT_FORCE_C1", default_cols(lg1));
    p->c2 = cfg->c2 > 0 ? cfg->c2 : env_int("GBFFT_FORCE_C2", fp32 && lg2 >= 10 && lg2 <= 12 ? 4 : default_cols(lg2));
    if (p->c1 > (1 << lg2)) p->c1 = 1 << lg2;
    if (p->c2 > (1 << lg1)) p->c2 = 1 << lg1;
    p->k1 = tile_kernel(MAP_CC, lg1, p->c1);
    p->k2 = tile_kernel(MAP_JC, lg2, p->c2);
    if (!p->k1 || !p->k2) return FFT_ERR_UNSUPPORTED;
    int rc = prepare_kernel(p->k1);
    if (!rc) rc = prepare_kernel(p->k2);
    if (!rc) rc = build_tables(p, lg1, lg2, lgN);
    if (rc) return rc;
    const long long N = p->n, N1 = 1LL << lg1, N2 = 1LL << lg2;
    // pass 1: tile g = columns [g*C1, g*C1+C1) of the N1 x N2 view x[N2*n1 + n2],
    // scaled by W_N^{n2*k1}, written to the workspace as Y[k1][n2]
    PassDesc& A = p->pass[0];
    A.k = p->k1;
    base_args(A.a);
    A.a.tw = p->tw1;
    A.a.tiles_per_batch = N2 / p->c1;
    A.a.in_bstride = A.a.out_bstride = N;
    A.a.in_gstride = A.a.out_gstride = p->c1;
    A.a.in_sc = A.a.out_sc = 1;
    A.a.in_sn = A.a.out_sn = N2;
    A.a.ncols = N2;
    A.a.ft_lo = p->ft_lo;
    A.a.ft_hi = p->ft_hi;
    A.a.ft_lgN = lgN;
    A.a.ft_s = p->ft_s;
    A.a.stream_out = 0;  // read back by pass 2: keep it in L2
    A.in_role = 0;
    A.out_role = 2;
    A.ntiles = A.a.tiles_per_batch * p->batch;
    // pass 2: tile g = rows k1 in [g*C2, g*C2+C2) of Y, written to X[k1 + N1*k2]
    PassDesc& B = p->pass[1];
    B.k = p->k2;
    base_args(B.a);
    B.a.tw = p->tw2;
    B.a.tiles_per_batch = N1 / p->c2;
    B.a.in_bstride = B.a.out_bstride = N;
    B.a.in_gstride = (long long)p->c2 * N2;
    B.a.in_sc = N2;
    B.a.in_sn = 1;
    B.a.out_gstride = p->c2;
    B.a.out_sc = 1;
    B.a.out_sn = N1;
    B.a.ncols = N1;
    B.a.stream_in = 0;
    B.in_role = 2;
    B.out_role = 1;
    B.ntiles = B.a.tiles_per_batch * p->batch;
    p->npass = 2;
    p->launches = 2;
    p->ws_bytes = (size_t)p->n * (size_t)p->batch * 8;
    int rc2 = attach_coltma(p, cfg->tma > 0 || (cfg->tma < 0 && p->prec == FFT_PREC_FP32));
    if (!rc2 && p->prec == FFT_PREC_FP32) rc2 = attach_rowtmas(p);
    return rc2;
  }
  // three passes, N = N1 * N2 * N3 (M = N2 * N3):
  //   A  columns of length N1 over stride M, scaled by W_N^{m*k1}     in -> ws
  //   B  per k1, columns of length N2 over stride N3 of the M-point
  //      row, scaled by W_M^{n3*k2}                                   ws -> ws (in place)
  //   C  rows of length N3, written to X[k1 + N1*k2 + N1*N2*k3]      ws -> out
  // measured on GB300: 2^8 x 2^8 x rest from 2^22 to 2^28 (rest <= 2^12)
  int l1 = (lgN >= 22 && lgN <= 28) ? 8 : (lgN + 2) / 3;
  int l2 = (lgN >= 22 && lgN <= 28) ? 8 : (lgN - l1 + 1) / 2;
  if (cfg->lg1 > 0) {
    l1 = cfg->lg1;
    l2 = cfg->lg2 > 0 ? cfg->lg2 : (lgN - l1 + 1) / 2;
  }
  const int l3 = lgN - l1 - l2;
  if (l1 < 1 || l2 < 1 || l1 > 14 || l2 > 14 || l3 > 14 || l3 < 1) return FFT_ERR_UNSUPPORTED;
  p->lg1 = l1;
  p->lg2 = l2;
  p->lg3 = l3;
  const long long N = p->n, N1 = 1LL << l1, N2 = 1LL << l2, N3 = 1LL << l3, M = N2 * N3;
  const int cA = (int)std::min<long long>(cfg->c1 > 0 ? cfg->c1 : default_cols(l1), M);
  const int cB = (int)std::min<long long>(cfg->c2 > 0 ? cfg->c2 : default_cols(l2), N3);
  const int cC = (int)std::min<long long>(cfg->c3 > 0 ? cfg->c3 : default_cols(l3), N1);
  const TileKernelInfo* kA = tile_kernel(MAP_CC, l1, cA);
  const TileKernelInfo* kB = tile_kernel(MAP_CC, l2, cB);
  const TileKernelInfo* kC = tile_kernel(MAP_JC, l3, cC);
  if (!kA || !kB || !kC) return FFT_ERR_UNSUPPORTED;
  int rc = prepare_kernel(kA);
  if (!rc) rc = prepare_kernel(kB);
  if (!rc) rc = prepare_kernel(kC);
  const int lgs[3] = {l1, l2, l3};
  const int lgNs[2] = {lgN, l2 + l3};
  if (!rc) rc = build_tables_multi(p, lgs, lgNs);
  if (rc) return rc;
  p->k1 = kA;
  p->k2 = kC;
  p->c1 = cA;
  p->c2 = cC;
  PassDesc& A = p->pass[0];
  A.k = kA;
  base_args(A.a);
  A.a.tw = p->tw1;
  A.a.tiles_per_batch = M / cA;
  A.a.in_bstride = A.a.out_bstride = N;
  A.a.in_gstride = A.a.out_gstride = cA;
  A.a.in_sc = A.a.out_sc = 1;
  A.a.in_sn = A.a.out_sn = M;
  A.a.ncols = M;
  A.a.ft_lo = p->ft_lo;
  A.a.ft_hi = p->ft_hi;
  A.a.ft_lgN = lgN;
  A.a.ft_s = p->ft_s;
  A.a.stream_out = 0;
  A.in_role = 0;
  A.out_role = 2;
  A.ntiles = A.a.tiles_per_batch * p->batch;
  PassDesc& B = p->pass[1];
  B.k = kB;
  base_args(B.a);
  B.a.tw = p->tw2;
  B.a.tiles_per_batch = N3 / cB;
  B.a.in_bstride = B.a.out_bstride = M;  // batch index = (b, k1): row (b*N1 + k1) of length M
  B.a.in_gstride = B.a.out_gstride = cB;
  B.a.in_sc = B.a.out_sc = 1;
  B.a.in_sn = B.a.out_sn = N3;
  B.a.ncols = N3;
  B.a.ft_lo = p->ft2_lo;
  B.a.ft_hi = p->ft2_hi;
  B.a.ft_lgN = l2 + l3;
  B.a.ft_s = p->ft2_s;
  B.a.stream_in = 0;
  B.a.stream_out = 0;
  B.in_role = 2;
  B.out_role = 2;
  B.ntiles = B.a.tiles_per_batch * p->batch * N1;
  PassDesc& Cp = p->pass[2];
  Cp.k = kC;
  base_args(Cp.a);
  Cp.a.tw = p->tw3;
  Cp.a.tiles_per_batch = N1 / cC;  // tile = ((b, k2), k1 group)
  Cp.a.nb1 = N2;
  Cp.a.in_b2stride = Cp.a.out_b2stride = N;
  Cp.a.in_bstride = N3;
  Cp.a.out_bstride = N1;
  Cp.a.in_gstride = cC * M;
  Cp.a.out_gstride = cC;
  Cp.a.in_sc = M;
  Cp.a.in_sn = 1;
  Cp.a.out_sc = 1;
  Cp.a.out_sn = N1 * N2;
  Cp.a.ncols = N1;
  Cp.a.stream_in = 0;
  Cp.in_role = 2;
  Cp.out_role = 1;
  Cp.ntiles = Cp.a.tiles_per_batch * N2 * p->batch;
  p->npass = 3;
  p->launches = 3;
  p->ws_bytes = (size_t)p->n * (size_t)p->batch * 8;
  return attach_coltma(p, cfg->tma > 0 || (cfg->tma < 0 && p->prec == FFT_PREC_FP32));
}

// 2-D plan (Sec. 2.3.2: rows, then columns).  Rows: one on-chip pass over all
// ny*batch rows.  Columns: for ny <= 2^10 one column pass of C >= 8 adjacent
// columns (>= 64 contiguous bytes per row); taller images split the column
// length ny = Y1*Y2 into two column passes (the four-step split applied along
// y), so every column tile stays 16 columns wide.
// 2-D in two passes over memory, each a row transform whose output is stored
// transposed (rows of the image in, columns of the result out): pass 1 takes
// the rows of x (length nx) to ws[b][kx][y], pass 2 the rows of ws (length
// ny) to out[b][ky][kx].  The column transforms thus read contiguous rows;
// the transposition is in the stores (runs of C adjacent outputs, C rows per
// CTA).
static int build_2d_transposed(fft_plan* p, int ly, int lx) {
  const long long ny = p->ny, nx = p->nx, img = ny * nx;
  // rows per CTA: as many as a 2^14-point tile holds, at most 8 (longer output runs)
  auto pick = [](int lg, long long rows) {
    int c = (int)std::min<long long>(std::min(16384 >> lg, 8), rows);
    while (c > 1 && !tile_kernel(MAP_JC, lg, c)) c >>= 1;
    return c;
  };
  const int c1 = pick(lx, ny), c2 = pick(ly, nx);
  const TileKernelInfo* k1 = tile_kernel(MAP_JC, lx, c1);
  const TileKernelInfo* k2 = tile_kernel(MAP_JC, ly, c2);
  if (!k1 || !k2 || ny % c1 || nx % c2) return FFT_ERR_UNSUPPORTED;
  int rc = prepare_kernel(k1);
  if (!rc) rc = prepare_kernel(k2);
  const int lgs[3] = {lx, ly, 0};
  const int lgNs[2] = {0, 0};
  if (!rc) rc = build_tables_multi(p, lgs, lgNs);
  if (rc) return rc;
  PassDesc& A = p->pass[0];
  A.k = k1;
  base_args(A.a);
  A.a.tw = p->tw1;
  A.a.tiles_per_batch = ny / c1;
  A.a.in_bstride = A.a.out_bstride = img;
  A.a.in_gstride = (long long)c1 * nx;
  A.a.in_sc = nx;
  A.a.in_sn = 1;
  A.a.out_gstride = c1;
  A.a.out_sc = 1;
  A.a.out_sn = ny;
  A.a.ncols = ny;
  A.a.stream_out = 0;  // read back by pass 2
  A.in_role = 0;
  A.out_role = 2;
  A.ntiles = A.a.tiles_per_batch * p->batch;
  PassDesc& B = p->pass[1];
  B.k = k2;
  base_args(B.a);
  B.a.tw = p->tw2;
  B.a.tiles_per_batch = nx / c2;
  B.a.in_bstride = B.a.out_bstride = img;
  B.a.in_gstride = (long long)c2 * ny;
  B.a.in_sc = ny;
  B.a.in_sn = 1;
  B.a.out_gstride = c2;
  B.a.out_sc = 1;
  B.a.out_sn = nx;
  B.a.ncols = nx;
  B.a.stream_in = 0;
  B.in_role = 2;
  B.out_role = 1;
  B.ntiles = B.a.tiles_per_batch * p->batch;
  p->k1 = k1;
  p->c1 = c1;
  p->k2 = k2;
  p->c2 = c2;
  p->npass = 2;
  p->launches = 2;
  p->ws_bytes = (size_t)img * (size_t)p->batch * 8;
  for (int i = 0; i < 2 && env_int("GBFFT_ROWTMAS", 1); ++i) {
    const TileKernelInfo* kt = tile_kernel_rowtmas(p->pass[i].k->lg, p->pass[i].k->C);
    if (kt) {
      rc = prepare_kernel(kt);
      if (rc) return rc;
      p->pass[i].kst = kt;
    }
  }
  return FFT_OK;
}

static int build_2d(fft_plan* p, int ly, int lx) {
  // measured on GB300 per 2^26 points against rows + column passes: 1024^2
  // 427 -> 388 us, 2048^2 577 -> 507, 4096^2 579 -> 545, 2048 x 1024 578 ->
  // 443, 4096 x 1024 579 -> 460 (ny x nx); but 1024 x 4096 418 -> 466 (its
  // rows + one column pass is already two passes) and 8192^2 623 -> 1066 (two
  // rows per CTA, 16-byte runs), so sides of 2^10..2^12 with ny >= 2^11 or
  // nx == ny == 2^10
  const int tr = env_int("GBFFT_2D_TRANSPOSE", -1);
  const bool transposed = tr >= 0 ? (tr > 0 && lx >= 8 && ly >= 8)
                                  : (lx >= 10 && lx <= 12 && ly >= 10 && ly <= 12 && (ly >= 11 || lx == 10));
  if (transposed) return build_2d_transposed(p, ly, lx);
  const long long ny = p->ny, nx = p->nx, img = ny * nx;
  const TileKernelInfo* kr = tile_kernel(MAP_JJ, lx, jj_cols(lx));
  if (!kr) return FFT_ERR_UNSUPPORTED;
  int rc = prepare_kernel(kr);
  if (rc) return rc;
  const int two = (ly >= 11 && !env_int("GBFFT_2D_ONE_COLUMN_PASS", 0)) ? 1 : 0;
  PassDesc& R = p->pass[0];
  R.k = kr;
  base_args(R.a);
  const int Cr = kr->C;
  R.a.tiles_per_batch = (ny * p->batch + Cr - 1) / Cr;
  R.a.in_gstride = R.a.out_gstride = (long long)Cr * nx;
  R.a.in_sc = R.a.out_sc = nx;
  R.a.in_sn = R.a.out_sn = 1;
  R.a.ncols = ny * p->batch;
  R.a.stream_out = 0;  // read back by the column pass
  R.in_role = 0;
  R.out_role = two ? 2 : 1;
  R.ntiles = R.a.tiles_per_batch;
  p->k1 = kr;
  p->c1 = Cr;
  if (Cr == 1 && lx >= 13 && env_int("GBFFT_2D_ROWS_PFS", 1)) {
    // rows of 2^13 and 2^14 points: the persistent kernel that stages the
    // next row by a bulk copy, as the 1-D single pass (8192^2: 623 -> 611 us,
    // 512 x 8192: 464 -> 449; rows of 2^12 measured slower, 416 -> 427)
    const TileKernelInfo* kp = tile_kernel_pfs(lx);
    int per_sm = 0, sms = 0, dev = 0;
    if (kp && !prepare_kernel(kp) && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kp->fn, kp->threads, (size_t)kp->smem_bytes) ==
            cudaSuccess &&
        per_sm >= 1) {
      R.kpfs = kp;
      R.pf_grid = (long long)per_sm * sms;
    }
  }
  if (!two) {
    const int C = (int)std::min<long long>(env_int("GBFFT_FORCE_C2", default_cols(ly)), nx);
    const TileKernelInfo* kc = tile_kernel(MAP_CC, ly, C);
    if (!kc) return FFT_ERR_UNSUPPORTED;
    rc = prepare_kernel(kc);
    const int lgs[3] = {ly, lx, 0};
    const int lgNs[2] = {0, 0};
    if (!rc) rc = build_tables_multi(p, lgs, lgNs);
    if (rc) return rc;
    R.a.tw = p->tw2;
    PassDesc& Cp = p->pass[1];
    Cp.k = kc;
    base_args(Cp.a);
    Cp.a.tw = p->tw1;
    Cp.a.tiles_per_batch = nx / C;
    Cp.a.in_bstride = Cp.a.out_bstride = img;
    Cp.a.in_gstride = Cp.a.out_gstride = C;
    Cp.a.in_sc = Cp.a.out_sc = 1;
    Cp.a.in_sn = Cp.a.out_sn = nx;
    Cp.a.ncols = nx;
    Cp.a.stream_in = 0;
    Cp.in_role = 1;
    Cp.out_role = 1;
    Cp.ntiles = Cp.a.tiles_per_batch * p->batch;
    p->k2 = kc;
    p->c2 = C;
    p->npass = 2;
    p->launches = 2;
    p->ws_bytes = 0;
    return attach_coltma(p, false);
  }
  int ly1 = ly / 2;
  const int env_ly1 = env_int("GBFFT_2D_LY1", 0);
  if (env_ly1 >= 1 && env_ly1 < ly && ly - env_ly1 <= 14) ly1 = env_ly1;
  const int ly2 = ly - ly1;
  const long long Y1 = 1LL << ly1, Y2 = 1LL << ly2;
  // first column pass: 32 columns per tile where compiled (8192^2, 2^6 x 2^7:
  // 611 -> 586 us against 16; 64 columns 599, other splits 590..660)
  const int ca_default = tile_kernel(MAP_CC, ly1, 32) ? 32 : default_cols(ly1);
  const int ca = (int)std::min<long long>(env_int("GBFFT_2D_CA", ca_default), nx);
  const int cb = (int)std::min<long long>(env_int("GBFFT_2D_CB", default_cols(ly2)), nx);
  const TileKernelInfo* ka = tile_kernel(MAP_CC, ly1, ca);
  const TileKernelInfo* kb = tile_kernel(MAP_CC, ly2, cb);
  if (!ka || !kb) return FFT_ERR_UNSUPPORTED;
  rc = prepare_kernel(ka);
  if (!rc) rc = prepare_kernel(kb);
  const int lgs[3] = {ly1, lx, ly2};
  const int lgNs[2] = {ly, 0};
  if (!rc) rc = build_tables_multi(p, lgs, lgNs);
  if (rc) return rc;
  R.a.tw = p->tw2;
  // column pass A: y = y1*Y2 + y2; per (image, y2) the FFT over y1 of C
  // adjacent columns, scaled by W_ny^{y2*ky1}; in place in the workspace
  PassDesc& A = p->pass[1];
  A.k = ka;
  base_args(A.a);
  A.a.tw = p->tw1;
  A.a.tiles_per_batch = nx / ca;
  A.a.nb1 = Y2;
  A.a.in_b2stride = A.a.out_b2stride = img;
  A.a.in_bstride = A.a.out_bstride = nx;
  A.a.in_gstride = A.a.out_gstride = ca;
  A.a.in_sc = A.a.out_sc = 1;
  A.a.in_sn = A.a.out_sn = Y2 * nx;
  A.a.ncols = nx;
  A.a.ft_lo = p->ft_lo;
  A.a.ft_hi = p->ft_hi;
  A.a.ft_lgN = ly;
  A.a.ft_s = p->ft_s;
  A.a.ft_by_batch = 1;
  A.a.stream_in = 0;
  A.a.stream_out = 0;
  A.in_role = 2;
  A.out_role = 2;
  A.ntiles = A.a.tiles_per_batch * Y2 * p->batch;
  // column pass B: per (image, ky1) the FFT over y2, written to row ky1 + Y1*ky2
  PassDesc& B = p->pass[2];
  B.k = kb;
  base_args(B.a);
  B.a.tw = p->tw3;
  B.a.tiles_per_batch = nx / cb;
  B.a.nb1 = Y1;
  B.a.in_b2stride = B.a.out_b2stride = img;
  B.a.in_bstride = Y2 * nx;
  B.a.out_bstride = nx;
  B.a.in_gstride = B.a.out_gstride = cb;
  B.a.in_sc = B.a.out_sc = 1;
  B.a.in_sn = nx;
  B.a.out_sn = Y1 * nx;
  B.a.ncols = nx;
  B.a.stream_in = 0;
  B.in_role = 2;
  B.out_role = 1;
  B.ntiles = B.a.tiles_per_batch * Y1 * p->batch;
  p->k2 = kb;
  p->c2 = cb;
  p->npass = 3;
  p->launches = 3;
  p->ws_bytes = (size_t)img * (size_t)p->batch * 8;
  return attach_coltma(p, false);
}

}  // namespace gbfft

// ============================================================================
// C ABI
// ============================================================================
// ---- live plan handles -------------------------------------------------------
// Every plan handed to a caller is recorded until fft_destroy; the entry
// points reject any other pointer (never created, or already destroyed) with
// FFT_ERR_INVALID_ARG instead of reading freed memory.  The set and its lock
// are never destroyed, so calls made while the process exits stay valid.
static std::mutex& live_mutex() {
  static std::mutex* m = new std::mutex;
  return *m;
}
static std::unordered_set<const fft_plan*>& live_plans() {
  static auto* s = new std::unordered_set<const fft_plan*>;
  return *s;
}
static fft_plan* publish(fft_plan* p) {
  if (!p) return nullptr;
  try {
    std::lock_guard<std::mutex> g(live_mutex());
    live_plans().insert(p);
  } catch (...) {
    free_plan(p);
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  return p;
}
static bool is_live(const fft_plan* p) {
  if (!p) return false;
  std::lock_guard<std::mutex> g(live_mutex());
  return live_plans().count(p) != 0;
}
static bool retire(const fft_plan* p) {
  if (!p) return false;
  std::lock_guard<std::mutex> g(live_mutex());
  return live_plans().erase(p) != 0;
}

extern "C" {

static bool smooth7(int64_t n) {
  if (n < 1) return false;
  for (const int f : {2, 3, 5, 7})
    while (n % f == 0) n /= f;
  return n == 1;
}

// Lengths that are not powers of two (7-smooth, FP32) and every FP64 plan:
// one pass of the mixed-radix kernel up to kMixedMaxN (FP32) or kMixedMaxN64
// (FP64) points, the strided four-step passes of mixed4.cu beyond that (both
// factors one on-chip pass).
static fft_plan* create_mixed(int64_t n, int64_t batch, int dir, int prec) {
  const bool fp64 = prec == FFT_PREC_FP64;
  const bool pow2 = n > 0 && (n & (n - 1)) == 0;
  if (n < 2 || batch < 1 || !valid_dir(dir) || !valid_prec(prec) || (double)n * (double)batch > 9.0e15) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  if (!smooth7(n) || (pow2 && n > (1LL << FFT_MAX_LOG2N))) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  const long long one_pass = fp64 ? kMixedMaxN64 : kMixedMaxN;
  const long long max_n = one_pass * one_pass;
  if (tc_prec(prec) || n > max_n) {
    // valid lengths this build does not run at that precision or size
    set_err(FFT_ERR_UNSUPPORTED);
    return nullptr;
  }
  fft_plan* p = new_plan();
  if (!p) {
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  p->kind = KIND_MIXED;
  p->n = n;
  p->batch = batch;
  p->dir = dir;
  p->prec = prec;
  const int rc = n <= one_pass ? mixed_plan_init(p) : mixed4_plan_1d(p);
  if (rc != FFT_OK) {
    free_plan(p);
    set_err(rc);
    return nullptr;
  }
  return p;
}

static fft_plan* create_1d(int64_t n, int64_t batch, int dir, int prec, const fft_plan_config* cfg) {
  const int lgN = ilog2_exact(n);
  if (prec == FFT_PREC_FP64) {
    if (cfg) {
      set_err(FFT_ERR_UNSUPPORTED);
      return nullptr;
    }
    return create_mixed(n, batch, dir, prec);
  }
  if (lgN < 0 && n > 2 && !cfg) return create_mixed(n, batch, dir, prec);
  if (lgN < 1 || lgN > FFT_MAX_LOG2N || batch < 1 || !valid_dir(dir) || !valid_prec(prec)) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  if ((double)n * (double)batch > 9.0e15) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  fft_plan* p = new_plan();
  if (!p) {
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  p->n = n;
  p->batch = batch;
  p->dir = dir;
  p->prec = prec;
  int rc = plan_1d(p, lgN, cfg);
  if (rc == FFT_OK && prec != FFT_PREC_FP32) rc = tc_plan_init(p);
  if (rc != FFT_OK) {
    free_plan(p);
    set_err(rc);
    return nullptr;
  }
  return p;
}

fft_plan* fft_plan_create(int64_t n, int64_t batch, int dir, int prec) {
  return publish(create_1d(n, batch, dir, prec, nullptr));
}

static int plan_real(fft_plan* p, int lgN) {
  const int lgM = lgN - 1;
  const long long M = 1LL << lgM;
  // W_N^k for k < M: one level (M entries) for the fused kernels, two levels
  // (r_lo[k & (2^r_s - 1)] * r_hi[k >> r_s]) for the split kernels
  p->r_s = lgM <= 14 ? lgM : (lgM + 1) / 2;
  const long long nlo = 1LL << p->r_s, nhi = 1LL << (lgM - p->r_s);
  const size_t hi_off = align256((size_t)nlo * 8);
  if (cudaMalloc(&p->d_rtw, hi_off + (size_t)nhi * 8) != cudaSuccess) return FFT_ERR_ALLOC;
  p->r_lo = (const float2*)p->d_rtw;
  p->r_hi = (const float2*)((char*)p->d_rtw + hi_off);
  if (launch_gen_power_twiddles((float2*)p->r_lo, lgN, nlo, 1, 0) != cudaSuccess ||
      launch_gen_power_twiddles((float2*)p->r_hi, lgN, nhi, nlo, 0) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess)
    return FFT_ERR_CUDA;
  p->lg = p->lg1 = lgM;
  if (lgM <= 14) {
    p->kr2c = tile_kernel_r2c(lgM);
    p->kc2r = tile_kernel_c2r(lgM);
    if (!p->kr2c || !p->kc2r) return FFT_ERR_UNSUPPORTED;
    int rc = prepare_kernel(p->kr2c);
    if (!rc) rc = prepare_kernel(p->kc2r);
    if (rc) return rc;
    p->k1 = p->kr2c;
    p->c1 = p->kr2c->C;
    p->launches = 1;
    return build_tables(p, lgM, 0, 0);
  }
  p->inner = create_1d(M, p->batch, FFT_FORWARD, FFT_PREC_FP32, nullptr);
  if (!p->inner) return fft_last_error();
  p->launches = p->inner->launches + 1;
  // Two-pass inner plans with rows of 2^6..2^12 points and at least 16 rows:
  // the real-to-complex split runs inside the row pass (real_fold.cu), two
  // passes over memory instead of three.
  const fft_plan* q = p->inner;
  if (q->kind == KIND_FOURSTEP && q->npass == 2 && !q->fused && q->pass[1].k && q->pass[1].k->map == MAP_JC &&
      q->lg1 >= 4 && r2c_fold_kernel_info(q->lg2)) {
    p->krfold = r2c_fold_kernel_info(q->lg2);
    const int rc = prepare_kernel(p->krfold);
    if (rc) return rc;
  }
  // ... and the complex-to-real split inside the column pass
  if (q->kind == KIND_FOURSTEP && q->npass == 2 && !q->fused && q->pass[0].k && q->pass[0].k->map == MAP_CC &&
      c2r_fold_kernel_info(q->lg1, q->pass[0].k->C)) {
    p->kcfold = c2r_fold_kernel_info(q->lg1, q->pass[0].k->C);
    const int rc = prepare_kernel(p->kcfold);
    if (rc) return rc;
  }
  if (p->krfold && p->kcfold) p->launches = p->inner->launches;   // both directions folded
  p->lg2 = p->inner->lg2;
  p->d_status = p->inner->d_status;
  p->ws_bytes = align256(p->inner->ws_bytes) + (size_t)M * (size_t)p->batch * 8;
  return FFT_OK;
}

// FP64 real-data plans: N = 2M reals, the complex128 plan of length M (one
// mixed-radix pass or the strided four-step passes) plus the FP64 split
// kernels, with a two-level FP64 table W_N^k, k < M.
static int plan_real64(fft_plan* p) {
  const long long M = p->n / 2;
  p->inner = create_1d(M, p->batch, FFT_FORWARD, FFT_PREC_FP64, nullptr);
  if (!p->inner) return fft_last_error();
  int bits = 0;
  while ((1LL << bits) < M) ++bits;
  p->r_s = (bits + 1) / 2;
  const long long nlo = 1LL << p->r_s, nhi = ((M - 1) >> p->r_s) + 1;
  const size_t hi_off = align256((size_t)nlo * 16);
  if (cudaMalloc(&p->d_rtw, hi_off + (size_t)nhi * 16) != cudaSuccess) return FFT_ERR_ALLOC;
  p->r_lo = (const float2*)p->d_rtw;   // complex128 entries
  p->r_hi = (const float2*)((char*)p->d_rtw + hi_off);
  if (launch_gen_twiddles_step((void*)p->r_lo, true, p->n, nlo, 1, 0) != cudaSuccess ||
      launch_gen_twiddles_step((void*)p->r_hi, true, p->n, nhi, nlo, 0) != cudaSuccess ||
      cudaStreamSynchronize(0) != cudaSuccess)
    return FFT_ERR_CUDA;
  p->launches = p->inner->launches + 1;
  p->d_status = p->inner->d_status;
  p->ws_bytes = align256(p->inner->ws_bytes) + (size_t)M * (size_t)p->batch * 16;
  return FFT_OK;
}

fft_plan* fft_plan_create_r2c(int64_t n, int64_t batch, int prec) {
  const int lgN = ilog2_exact(n);
  if (prec == FFT_PREC_FP64) {
    // any even n >= 4 whose half is a 7-smooth FP64 length
    if (n < 4 || (n & 1) || !smooth7(n / 2) || batch < 1 || (double)n * (double)batch > 9.0e15) {
      set_err(FFT_ERR_INVALID_ARG);
      return nullptr;
    }
    fft_plan* p = new_plan();
    if (!p) {
      set_err(FFT_ERR_ALLOC);
      return nullptr;
    }
    p->kind = KIND_REAL;
    p->n = n;
    p->batch = batch;
    p->dir = FFT_FORWARD;
    p->prec = prec;
    const int rc = plan_real64(p);
    if (rc != FFT_OK) {
      free_plan(p);
      set_err(rc);
      return nullptr;
    }
    return publish(p);
  }
  if (lgN < 2 || lgN > FFT_MAX_LOG2N || batch < 1 || !valid_prec(prec) || (double)n * (double)batch > 9.0e15) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  if (prec != FFT_PREC_FP32) {
    set_err(FFT_ERR_UNSUPPORTED);
    return nullptr;
  }
  fft_plan* p = new_plan();
  if (!p) {
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  p->kind = KIND_REAL;
  p->n = n;
  p->batch = batch;
  p->dir = FFT_FORWARD;
  p->prec = prec;
  const int rc = plan_real(p, lgN);
  if (rc != FFT_OK) {
    free_plan(p);
    set_err(rc);
    return nullptr;
  }
  return publish(p);
}

fft_plan* fft_plan_create_config(int64_t n, int64_t batch, int dir, int prec, const fft_plan_config* cfg) {
  return publish(create_1d(n, batch, dir, prec, cfg));
}

int fft_plan_get_config(const fft_plan* p, fft_plan_config* out) {
  if (!is_live(p) || !out) return set_err(FFT_ERR_INVALID_ARG);
  memset(out, 0, sizeof(*out));
  out->tma = -1;
  out->fused = 0;
  out->halves = 1;
  out->radix = 16;
  if (p->kind == KIND_SINGLE) {
    out->npass = 1;
    out->lg1 = p->lg;
    out->c1 = p->c1;
    out->tma = p->ktma ? 1 : (p->kpfs ? 3 : (p->kpf ? 2 : 0));
    out->halves = p->kdif2 ? 2 : 1;
    out->radix = p->kradix ? (1 << p->radix_lgm) : 16;
  } else if (p->kind == KIND_FOURSTEP) {
    out->npass = p->npass ? p->npass : 2;
    out->fused = p->fused ? 1 : 0;
    out->tma = (!p->fused && p->pass[0].kcol) ? 1 : 0;
    out->lg1 = p->lg1;
    out->lg2 = p->lg2;
    if (out->npass == 3) {
      out->c1 = p->pass[0].k->C;
      out->c2 = p->pass[1].k->C;
      out->c3 = p->pass[2].k->C;
    } else {
      out->c1 = p->c1;
      out->c2 = p->c2;
    }
  } else {
    return set_err(FFT_ERR_INVALID_ARG);
  }
  return FFT_OK;
}

// 2-D plans of 7-smooth sides that are not both powers of two, and every FP64
// 2-D plan: row then column passes of the strided mixed-radix kernel.
static fft_plan* create_2d_mixed(int64_t ny, int64_t nx, int64_t batch, int dir, int prec) {
  const long long side_max = prec == FFT_PREC_FP64 ? kMixedMaxN64 : kMixedMaxN;
  if (tc_prec(prec) || ny > side_max || nx > side_max) {
    set_err(FFT_ERR_UNSUPPORTED);
    return nullptr;
  }
  fft_plan* p = new_plan();
  if (!p) {
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  p->kind = KIND_MIXED_PASSES;
  p->n = ny * nx;
  p->ny = ny;
  p->nx = nx;
  p->batch = batch;
  p->dir = dir;
  p->prec = prec;
  const int rc = mixed4_plan_2d(p);
  if (rc != FFT_OK) {
    free_plan(p);
    set_err(rc);
    return nullptr;
  }
  return publish(p);
}

fft_plan* fft_plan_create_2d(int64_t ny, int64_t nx, int64_t batch, int dir, int prec) {
  const int ly = ilog2_exact(ny), lx = ilog2_exact(nx);
  if (ny < 2 || nx < 2 || !smooth7(ny) || !smooth7(nx) || batch < 1 || !valid_dir(dir) || !valid_prec(prec) ||
      (double)ny * (double)nx * (double)batch > 9.0e15) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  const bool pow2 = ly >= 1 && lx >= 1;
  if (prec == FFT_PREC_FP64 || !pow2) return create_2d_mixed(ny, nx, batch, dir, prec);
  if (ly > FFT_MAX_LOG2_SIDE || lx > FFT_MAX_LOG2_SIDE) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  if (prec != FFT_PREC_FP32) {
    set_err(FFT_ERR_UNSUPPORTED);
    return nullptr;
  }
  fft_plan* p = new_plan();
  if (!p) {
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  p->kind = KIND_2D;
  p->n = ny * nx;
  p->ny = ny;
  p->nx = nx;
  p->batch = batch;
  p->dir = dir;
  p->prec = prec;
  p->lg1 = ly;
  p->lg2 = lx;
  int rc = build_2d(p, ly, lx);
  if (rc != FFT_OK) {
    free_plan(p);
    set_err(rc);
    return nullptr;
  }
  return publish(p);
}

fft_plan* fft_plan_create_many(const int64_t* lengths, int64_t count, int dir, int prec) {
  return fft_plan_create_many_config(lengths, count, dir, prec, nullptr);
}

int fft_plan_get_many_config(const fft_plan* plan, fft_many_config* out) {
  if (!is_live(plan) || !out || plan->kind != KIND_MANY) return set_err(FFT_ERR_INVALID_ARG);
  return set_err(many_get_config(plan, out));
}

fft_plan* fft_plan_create_many_config(const int64_t* lengths, int64_t count, int dir, int prec,
                                      const fft_many_config* cfg) {
  fft_many_config resolved;
  if (!lengths || count < 1 || !valid_dir(dir) || !valid_prec(prec) || many_resolve_config(cfg, &resolved) != FFT_OK) {
    set_err(FFT_ERR_INVALID_ARG);
    return nullptr;
  }
  if (prec == FFT_PREC_FP64) {
    set_err(FFT_ERR_UNSUPPORTED);
    return nullptr;
  }

  if (prec != FFT_PREC_FP32) {
    set_err(FFT_ERR_UNSUPPORTED);
    return nullptr;
  }
  fft_plan* p = new_plan();
  if (!p) {
    set_err(FFT_ERR_ALLOC);
    return nullptr;
  }
  p->kind = KIND_MANY;
  p->dir = dir;
  p->prec = prec;
  p->batch = count;
  int rc = many_plan_init(p, lengths, count, cfg);
  if (rc != FFT_OK) {
    free_plan(p);
    set_err(rc);
    return nullptr;
  }
  return publish(p);
}

int fft_exec(fft_plan* plan, const void* in, void* out, void* stream) {
  if (!is_live(plan)) return set_err(FFT_ERR_INVALID_ARG);
  return set_err(exec_plan(plan, in, out, plan->dir, (cudaStream_t)stream));
}

int fft_exec_dir(fft_plan* plan, const void* in, void* out, int dir, void* stream) {
  if (!is_live(plan)) return set_err(FFT_ERR_INVALID_ARG);
  return set_err(exec_plan(plan, in, out, dir, (cudaStream_t)stream));
}

int fft_exec_filter_dir(fft_plan* plan, const void* in, void* out, const void* filt, int dir, void* stream) {
  if (!is_live(plan) || !in || !out || !filt || (dir != FFT_FORWARD && dir != FFT_ADJOINT))
    return set_err(FFT_ERR_INVALID_ARG);
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7) || ((uintptr_t)filt & 7)) return set_err(FFT_ERR_ALIGN);
  // every launch below reports its own error; one left pending by an earlier,
  // unrelated call must not be taken for this call's
  cudaGetLastError();
  return set_err(exec_filter_plan(plan, (const float2*)in, (float2*)out, (const float2*)filt,
                                  dir == FFT_ADJOINT ? 1 : 0, (cudaStream_t)stream));
}

int fft_exec_filter(fft_plan* plan, const void* in, void* out, const void* filt, void* stream) {
  return fft_exec_filter_dir(plan, in, out, filt, FFT_FORWARD, stream);
}

void fft_destroy(fft_plan* plan) {
  if (retire(plan))
    free_plan(plan);
  else if (plan)
    set_err(FFT_ERR_INVALID_ARG);   // not a live plan (e.g. destroyed twice): nothing is freed
}

size_t fft_plan_workspace_bytes(const fft_plan* plan) { return is_live(plan) ? plan->ws_bytes : 0; }

// A real-data plan hands the front of its workspace to its complex plan and
// keeps the rest for Z.
static void distribute_real_ws(fft_plan* plan) {
  if (plan->kind != KIND_REAL || !plan->inner) return;
  char* base = (char*)plan->ws;
  plan->inner->ws = (base && plan->inner->ws_bytes) ? base : nullptr;
  plan->inner->ws_owned = 0;
  plan->zbuf = base ? (float2*)(base + align256(plan->inner->ws_bytes)) : nullptr;
}

int fft_plan_set_workspace(fft_plan* plan, void* dev_ptr) {
  if (!is_live(plan)) return set_err(FFT_ERR_INVALID_ARG);
  if (dev_ptr && ((uintptr_t)dev_ptr & 255)) return set_err(FFT_ERR_ALIGN);
  if (plan->ws_owned && plan->ws) cudaFree(plan->ws);
  plan->ws = nullptr;
  plan->ws_owned = 0;
  if (dev_ptr) {
    plan->ws = dev_ptr;
    distribute_real_ws(plan);
    return FFT_OK;
  }
  if (plan->ws_bytes == 0) return FFT_OK;
  if (cudaMalloc(&plan->ws, plan->ws_bytes) != cudaSuccess) {
    plan->ws = nullptr;
    distribute_real_ws(plan);
    return set_err(FFT_ERR_ALLOC);
  }
  plan->ws_owned = 1;
  distribute_real_ws(plan);
  return FFT_OK;
}

int64_t fft_plan_length(const fft_plan* plan) { return is_live(plan) ? plan->n : 0; }
int64_t fft_plan_batch(const fft_plan* plan) { return is_live(plan) ? plan->batch : 0; }
int fft_plan_launches(const fft_plan* plan) { return is_live(plan) ? plan->launches : 0; }
int fft_plan_kind(const fft_plan* plan) { return is_live(plan) ? plan->kind : -1; }

int fft_plan_describe(const fft_plan* p, char* buf, size_t len) {
  if (!is_live(p) || !buf || len == 0) return set_err(FFT_ERR_INVALID_ARG);
  static const char* kinds[] = {"single", "fourstep", "2d", "many", "real", "mixed", "mixed_passes", "?"};
  const TileKernelInfo* k1 = p->kradix ? p->kradix : p->k1;   // the first kernel that runs
  snprintf(buf, len,
           "kind=%s n=%lld batch=%lld lg1=%d lg2=%d c1=%d c2=%d threads1=%d smem1=%d threads2=%d smem2=%d "
           "prec=%d launches=%d ws=%zu tma_grid=%lld radix=%d",
           kinds[p->kind & 7], (long long)p->n, (long long)p->batch, p->lg1, p->lg2, p->c1, p->c2,
           k1 ? k1->threads : 0, k1 ? k1->smem_bytes : 0, p->k2 ? p->k2->threads : 0,
           p->k2 ? p->k2->smem_bytes : 0, p->prec, p->launches, p->ws_bytes, p->ktma ? p->tma_grid : 0LL,
           p->kradix ? 1 << p->radix_lgm : 16);
  return FFT_OK;
}

int fft_status(fft_plan* plan, void* stream) {
  if (!is_live(plan) || !plan->d_status) return set_err(FFT_ERR_INVALID_ARG);
  int h = 0;
  if (cudaMemcpyAsync(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return set_err(FFT_ERR_CUDA);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return set_err(FFT_ERR_CUDA);
  return h;
}

int fft_last_error(void) { return g_last_error; }

const char* fft_error_string(int code) {
  switch (code) {
    case FFT_OK: return "ok";
    case FFT_ERR_INVALID_ARG: return "invalid argument";
    case FFT_ERR_ALIGN: return "data pointer not aligned";
    case FFT_ERR_NO_WORKSPACE: return "plan needs a workspace (fft_plan_set_workspace)";
    case FFT_ERR_CUDA: return "CUDA runtime error";
    case FFT_ERR_TIMEOUT: return "bounded device wait timed out";
    case FFT_ERR_UNSUPPORTED: return "unsupported configuration";
    case FFT_ERR_ALLOC: return "allocation failed";
  }
  return "unknown error";
}

}  // extern "C"
