// noalloc.cu -- a large-transform entry point that allocates no memory.
//
// Who needs it: code that must not call cudaMalloc at the moment it wants a
// transform.  Typical cases are a custom allocator or memory-pool callback
// (calling back into the allocator would re-enter it), a plug-in living inside
// a host application that owns every byte of device memory and forbids private
// allocations, and real-time or certified code paths where every allocation
// must happen once at start-up.  The normal API cannot serve them: a plan
// allocates its twiddle tables, and a four-step plan also needs a workspace.
//
// What it does: the same two-pass four-step FFT as fft_exec on a four-step
// plan (column pass with twiddle, row pass written transposed), with its
// scratch -- the pass-1 workspace and the twiddle tables -- carved out of one
// file-scope static device array, g_noalloc_scratch, of fixed size.  The CUDA
// runtime loads this module (kernels and array) onto a device lazily, at the
// library's first use there, and that load allocates; the array then stays
// reserved on the device until the process exits.  The first call on a device
// should therefore come at start-up, from a context that may allocate.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; nothing in it needs to start at zero (each call regenerates its
// twiddles and overwrites the workspace before reading it).  Calls whose
// kernels overlap on the GPU (different streams, or different host threads)
// race on the array and produce garbage: serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "gbfft_internal.h"
#include "tile_registry.h"

namespace gbfft {

// Limits of this entry point: transform lengths 2^15..2^22 and at most 2^22
// points per call (n * batch), i.e. a 32 MiB workspace.
constexpr int kNoallocMinLog2 = 15;
constexpr int kNoallocMaxLog2 = 22;
constexpr long long kNoallocMaxPoints = 1LL << 22;
// twiddle area: four slots of 4096 complex entries for the two stage tables
// (lengths <= 2^11) and the two levels of the W_N table (<= 2^11 entries each)
constexpr long long kNoallocTwPoints = 4 * 4096;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocMaxPoints + kNoallocTwPoints];

// Host-side view: the symbol above is a host stand-in, not a device address.
// The device address is looked up once per device (cudaGetSymbolAddress) and
// cached here.  The same one-time set-up raises the dynamic shared-memory
// limit of every tile kernel this entry point can launch, so later calls make
// no attribute calls.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static float2* g_noalloc_ptr[kMaxDevices];

// Columns per tile of a pass of length 2^lg: 8192 points per tile, 1..16 columns.
static int noalloc_cols(int lg) {
  int c = (1 << 13) >> lg;
  return c < 1 ? 1 : (c > 16 ? 16 : c);
}

// Split of n = 2^lgN into N1 = 2^lg1 (column pass) and N2 = 2^lg2 (row pass).
static void noalloc_split(int lgN, int* lg1, int* lg2) {
  *lg2 = (lgN + 1) / 2;
  *lg1 = lgN - *lg2;
}

// The tile kernels of both passes.  Each pass is at least 2^7 long, so the
// other pass always has more columns than one tile takes (noalloc_cols <= 16).
static void noalloc_kernels(int lgN, const TileKernelInfo** k1, const TileKernelInfo** k2) {
  int lg1, lg2;
  noalloc_split(lgN, &lg1, &lg2);
  *k1 = tile_kernel(MAP_CC, lg1, noalloc_cols(lg1));
  *k2 = tile_kernel(MAP_JC, lg2, noalloc_cols(lg2));
}

static int noalloc_device_setup(int dev, float2** scratch) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    for (int lgN = kNoallocMinLog2; lgN <= kNoallocMaxLog2; ++lgN) {
      const TileKernelInfo *k1, *k2;
      noalloc_kernels(lgN, &k1, &k2);
      if (!k1 || !k2) return FFT_ERR_UNSUPPORTED;
      for (const TileKernelInfo* k : {k1, k2})
        if (k->smem_bytes > 48 * 1024 &&
            cudaFuncSetAttribute(k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k->smem_bytes) != cudaSuccess) {
          cudaGetLastError();
          return FFT_ERR_CUDA;
        }
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FFT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (float2*)p;
  }
  *scratch = g_noalloc_ptr[dev];
  return FFT_OK;
}

static int noalloc_launch(const TileKernelInfo* k, const TileArgs& a, long long ntiles, cudaStream_t s) {
  void* args[] = {(void*)&a};
  return cudaLaunchKernel(k->fn, dim3((unsigned)ntiles), dim3(k->threads), args, (size_t)k->smem_bytes, s) ==
                 cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

static int noalloc_run(int64_t n, int64_t batch, int dir, const float2* in, float2* out, cudaStream_t s) {
  int lgN = 0;
  while ((1LL << lgN) < n) ++lgN;
  int lg1, lg2;
  noalloc_split(lgN, &lg1, &lg2);
  const long long N1 = 1LL << lg1, N2 = 1LL << lg2;
  const int c1 = noalloc_cols(lg1), c2 = noalloc_cols(lg2);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FFT_ERR_CUDA;
  float2* scratch = nullptr;
  int rc = noalloc_device_setup(dev, &scratch);
  if (rc) return rc;
  const TileKernelInfo *k1, *k2;
  noalloc_kernels(lgN, &k1, &k2);

  // scratch layout: [workspace: n*batch points][tw1 4096][tw2 4096][lo 4096][hi 4096]
  float2* ws = scratch;
  float2* tw1 = scratch + kNoallocMaxPoints;
  float2* tw2 = tw1 + 4096;
  float2* lo = tw2 + 4096;
  float2* hi = lo + 4096;
  const int s_lo = (lgN + 1) / 2;
  if (launch_gen_stage_twiddles(tw1, lg1, s) != cudaSuccess) return FFT_ERR_CUDA;
  if (launch_gen_stage_twiddles(tw2, lg2, s) != cudaSuccess) return FFT_ERR_CUDA;
  if (launch_gen_power_twiddles(lo, lgN, 1LL << s_lo, 1, s) != cudaSuccess) return FFT_ERR_CUDA;
  if (launch_gen_power_twiddles(hi, lgN, 1LL << (lgN - s_lo), 1LL << s_lo, s) != cudaSuccess) return FFT_ERR_CUDA;

  const int inv = dir & FFT_INVERSE, adj = (dir & FFT_ADJOINT) ? 1 : 0;
  const int conj = inv ^ adj;
  const float scale = inv ? (float)(1.0 / (double)n) : 1.0f;

  TileArgs a;
  memset(&a, 0, sizeof(a));
  a.in = in;
  a.out = ws;
  a.tw = tw1;
  a.tiles_per_batch = N2 / c1;
  a.in_bstride = a.out_bstride = n;
  a.in_gstride = a.out_gstride = c1;
  a.in_sc = a.out_sc = 1;
  a.in_sn = a.out_sn = N2;
  a.ncols = N2;
  a.ft_lo = lo;
  a.ft_hi = hi;
  a.ft_lgN = lgN;
  a.ft_s = s_lo;
  a.conj_in = conj;
  a.stream_in = 1;
  rc = noalloc_launch(k1, a, a.tiles_per_batch * batch, s);
  if (rc) return rc;

  TileArgs b;
  memset(&b, 0, sizeof(b));
  b.in = ws;
  b.out = out;
  b.tw = tw2;
  b.tiles_per_batch = N1 / c2;
  b.in_bstride = b.out_bstride = n;
  b.in_gstride = (long long)c2 * N2;
  b.in_sc = N2;
  b.in_sn = 1;
  b.out_gstride = c2;
  b.out_sc = 1;
  b.out_sn = N1;
  b.ncols = N1;
  b.stream_out = 1;
  b.scale_out = (conj || scale != 1.0f) ? 1 : 0;
  b.sx = scale;
  b.sy = conj ? -scale : scale;
  return noalloc_launch(k2, b, b.tiles_per_batch * batch, s);
}

int set_err(int code);

}  // namespace gbfft

extern "C" GBFFT_API int fft_exec_noalloc(int64_t n, int64_t batch, int dir, const void* in, void* out,
                                          void* stream) {
  using namespace gbfft;
  int lgN = -1;
  if (n > 0 && (n & (n - 1)) == 0) {
    lgN = 0;
    while ((1LL << lgN) < n) ++lgN;
  }
  if (lgN < kNoallocMinLog2 || lgN > kNoallocMaxLog2 || batch < 1 || batch > kNoallocMaxPoints / n || dir < 0 ||
      dir > 3 || !in || !out)
    return set_err(FFT_ERR_INVALID_ARG);
  if (((uintptr_t)in & 7) || ((uintptr_t)out & 7)) return set_err(FFT_ERR_ALIGN);
  // The twiddle launchers report through cudaGetLastError, which would also
  // return an error left pending by an earlier, unrelated call on this thread:
  // clear it first, so that every check below sees only this call's launches.
  cudaGetLastError();
  return set_err(noalloc_run(n, batch, dir, (const float2*)in, (float2*)out, (cudaStream_t)stream));
}
