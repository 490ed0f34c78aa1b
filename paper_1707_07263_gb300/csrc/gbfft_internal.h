// gbfft_internal.h -- plan representation shared by the host-side planner and
// the kernel launchers.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gbfft.h"
#include "tile_fft.cuh"

namespace gbfft {

struct TileKernelInfo;
struct ManyPlan;
struct FusedPlan;

// One launch of a multi-pass plan.  Buffers are named by role so a plan can
// run on any (in, out) pair: 0 = the caller's input, 1 = the caller's output,
// 2 = the workspace.  conj-in is applied by the first pass, the output
// scale / conj by the last.
struct PassDesc {
  const TileKernelInfo* k;
  TileArgs a;
  int in_role, out_role;
  long long ntiles;
  const TileKernelInfo* kcol;  // tensor-TMA variant of a column pass (or NULL)
  int col_grid;                // its resident-CTA grid
  const TileKernelInfo* kst;   // row pass with a tensor-TMA output store (or NULL)
  const TileKernelInfo* kpfs;  // contiguous one-pass rows: the persistent staged kernel (or NULL)
  long long pf_grid;           // its resident-CTA grid
};
constexpr int kMaxPasses = 4;

enum PlanKind {
  KIND_SINGLE = 0,
  KIND_FOURSTEP = 1,
  KIND_2D = 2,
  KIND_MANY = 3,
  KIND_REAL = 4,
  KIND_MIXED = 5,
  KIND_MIXED_PASSES = 6   // strided mixed-radix passes: four-step 1-D or 2-D (mixed4.cu)
};

// Lengths N = 2^a 3^b 5^c 7^d that are not powers of two (mixed.cu).
constexpr int kMixedMaxPasses = 16;
constexpr long long kMixedMaxN = 14336;   // two shared-memory buffers of N complex values fit
constexpr long long kMixedMaxN64 = 7168;  // the same for FP64 (complex128) values
struct MixedArgs {
  const void* in;     // float2 (FP32) or double2 (FP64) elements
  void* out;
  const void* tw;     // W_N^m, m < N, same element type
  int N, C;           // length; transforms per CTA
  long long batch;
  int nrad;
  int rad[kMixedMaxPasses];
  // per pass: N/R and Ns with their reciprocals ceil(2^32 / d) (0 for d = 1):
  // q = umulhi(n, m) is exact for n * d < 2^32, which every index here meets
  unsigned nb[kMixedMaxPasses], nb_m[kMixedMaxPasses];
  unsigned ns[kMixedMaxPasses], ns_m[kMixedMaxPasses];
  unsigned tws[kMixedMaxPasses];   // per pass: twiddle stride N / (Ns R) into W_N^m
  int conj_in, scale_out;
  double sx, sy;      // output scale (1/N of Eq. 2 exact to FP64 for the FP64 kernel)
  float fsx, fsy;     // the same rounded to FP32 for the FP32 kernel
};
// Mixed-radix lengths with a compile-time three-pass schedule (mixed_ct.cu).
struct MixedCtInfo {
  long long N;
  int r0, r1, r2;
  int C;           // transforms per CTA
  int threads;     // threads per CTA
  bool pad;        // padded shared-memory index (msidx)
  const void* fn;  // kernel void(MixedArgs)
};
const MixedCtInfo* mixed_ct_lookup(long long N);

int mixed_radices(long long N, int* rad);
bool mixed_schedule(MixedArgs& a, long long N);
int mixed_plan_init(fft_plan* p);

// Strided passes of the mixed-radix recurrence (mixed4.cu): a batch of
// sub-transforms of length m.N ("columns") whose element n sits at
// col * cs + n * ns from the batch's base, C = 2^csh adjacent columns per
// CTA.  Two such passes make the four-step split of a length beyond one
// on-chip pass (the column pass multiplies its output by W_Nt^{col * k}) and
// the rows-then-columns 2-D transform.
struct Mixed4Args {
  MixedArgs m;                 // sub-length schedule, W_{m.N} table, in/out, conj and output scale
  long long in_bs, out_bs;     // element offset of batch b: b * bs
  long long in_cs, in_ns, out_cs, out_ns;
  long long ncols;             // columns per batch
  long long tiles_per_batch;   // ceil(ncols / C)
  long long ntiles;            // tiles_per_batch * batches
  const void* ft_lo;           // four-step twiddle W_Nt^e = ft_lo[e & (2^ft_s - 1)] * ft_hi[e >> ft_s]
  const void* ft_hi;           // of e = col * k on the output (NULL: none)
  int ft_s;
};
struct Mixed4Pass {
  Mixed4Args a;
  const void* fn;
  int threads, smem;
  long long grid;
  int in_role, out_role;       // 0 the caller's input, 1 its output, 2 the workspace
};
constexpr int kMixed4MaxPasses = 2;
// FP32 sub-lengths with a compile-time schedule (mixed4_ct.cu)
struct Mixed4CtInfo {
  long long L;
  int r0, r1, r2;  // radices (r2 == 1: two passes)
  int csh;         // 2^csh columns per CTA
  const void* fn;  // kernel void(Mixed4Args)
};
const Mixed4CtInfo* mixed4_ct_lookup(long long L);
// kernel for element type (FP64 or FP32), 2^csh columns per CTA, padded index
const void* mixed4_kernel_fn(bool fp64, int csh, bool pad);
int mixed4_plan_1d(fft_plan* p);
int mixed4_plan_2d(fft_plan* p);
int mixed4_exec(fft_plan* p, const void* in, void* out, int conj, double sx, double sy, int scale_out,
                cudaStream_t s);
cudaError_t launch_gen_twiddles_step(void* tab, bool fp64, long long N, long long count, long long step,
                                     cudaStream_t s);
int mixed_exec(fft_plan* p, const void* in, void* out, int conj, double sx, double sy, int scale_out,
               cudaStream_t s);
cudaError_t launch_gen_twiddles_n(float2* tab, long long N, long long count, cudaStream_t s);
cudaError_t launch_gen_twiddles_n64(double2* tab, long long N, long long count, cudaStream_t s);

cudaError_t launch_gen_stage_twiddles(float2* tab, int lg, cudaStream_t s, bool rev = false, int lgm = 4);
cudaError_t launch_gen_power_twiddles(float2* tab, int lgN, long long count, long long step, cudaStream_t s);
// Real-to-complex transforms of N = 2M reals, M a two-pass four-step length
// with rows of 2^6..2^12 points: the even/odd split folded into the row pass
// (real_fold.cu).
struct TileKernelInfo;
const TileKernelInfo* r2c_fold_kernel_info(int lg2);
// complex to real: the split folded into the inner column pass (columns of
// 2^lg1 points, C per CTA), or NULL
const TileKernelInfo* c2r_fold_kernel_info(int lg1, int C);
int r2c_fold_launch(const TileKernelInfo* k, const TileArgs& a, long long M, int N1, long long batch,
                    const float2* r_lo, const float2* r_hi, int r_s, int scale, float s_int, float s_end,
                    cudaStream_t s);
cudaError_t launch_r2c_split(const float2* z, float2* x, long long M, long long batch, const float2* lo,
                             const float2* hi, int s, float s_int, float s_end, cudaStream_t st);
cudaError_t launch_c2r_split(const float2* x, float2* z, long long M, long long batch, const float2* lo,
                             const float2* hi, int s, float end_mul, cudaStream_t st);
cudaError_t launch_r2c_split64(const double2* z, double2* x, long long M, long long batch, const double2* lo,
                               const double2* hi, int s, double s_int, double s_end, cudaStream_t st);
cudaError_t launch_c2r_split64(const double2* x, double2* z, long long M, long long batch, const double2* lo,
                               const double2* hi, int s, double end_mul, cudaStream_t st);

}  // namespace gbfft

struct fft_plan {
  int kind;
  int64_t n;       // transform length (1-D), ny*nx (2-D), total points (many)
  int64_t batch;   // transforms (1-D), images (2-D), count (many)
  int64_t ny, nx;  // 2-D sides
  int dir, prec;
  int device;

  // single pass: lg; four-step: lg1 = log2 N1 (column length), lg2 = log2 N2
  // (row length); 2-D: lg1 = log2 ny, lg2 = log2 nx.
  int lg, lg1, lg2;
  int c1, c2;  // transforms per CTA of the first / second pass
  const gbfft::TileKernelInfo* k1;
  const gbfft::TileKernelInfo* k2;
  const gbfft::TileKernelInfo* ktma;  // persistent TMA-staged single-pass kernel (or NULL)
  const gbfft::TileKernelInfo* kdif2; // two-CTA radix-2 split kernel (or NULL)
  const gbfft::TileKernelInfo* kpf;   // persistent L2-prefetching single-pass kernel (or NULL)
  const gbfft::TileKernelInfo* kpfs;  // its variant staging the next transform by a bulk copy (or NULL;
                                      // kpf is then the fallback for inputs not 16-byte aligned)
  long long pf_grid;                  // its resident-CTA grid
  const gbfft::TileKernelInfo* kradix;  // single pass with radix-8 / radix-4 passes (config radix), or NULL
  void* d_radtw;                        // its stage table (schedule of largest radix 2^radix_lgm)
  int radix_lgm;
  const gbfft::TileKernelInfo* krc;   // fused range-compression kernel of the length (or NULL)
  void* d_rctw;                       // its remainder-last stage table (NULL: the length's own table)
  long long rc_grid;                  // its grid when persistent (0: one tile per CTA)

  // real-data plans (KIND_REAL, n = N reals, M = N/2): fused kernels for
  // M <= 2^14, else the complex length-M plan `inner` plus the split kernels
  // through `zbuf` (batch*M complex values after the inner workspace)
  const gbfft::TileKernelInfo* kr2c;
  const gbfft::TileKernelInfo* kc2r;
  const gbfft::TileKernelInfo* krfold;   // real-to-complex: split folded into the inner row pass (or NULL)
  const gbfft::TileKernelInfo* kcfold;   // complex-to-real: split folded into the inner column pass (or NULL)
  fft_plan* inner;
  void* d_rtw;        // W_N^k, k < M, two-level: r_lo[k & (2^r_s - 1)] * r_hi[k >> r_s]
  const float2* r_lo;
  const float2* r_hi;
  int r_s;
  float2* zbuf;

  // mixed-radix plans (KIND_MIXED)
  gbfft::MixedArgs mixed;
  int mixed_threads, mixed_smem, mixed_pad;
  const gbfft::MixedCtInfo* mixed_ct;   // compile-time schedule for this length (FP32), or NULL
  gbfft::Mixed4Pass m4[gbfft::kMixed4MaxPasses];   // KIND_MIXED_PASSES
  int m4n;
  long long m4_n1, m4_n2;   // four-step: column length N1, row length N2 (N = N1 N2); 2-D: ny, nx
  const float2* pre_tw;               // its W_N^n table, n < N/2
  long long tma_grid;                 // its resident-CTA grid

  // all twiddle tables live in one device allocation
  void* d_tables;
  const float2* tw1;  // stage table for the first pass length
  const float2* tw2;  // stage table for the second pass length
  const float2* ft_lo;
  const float2* ft_hi;
  int ft_s;

  // tensor-core radix-16 path (prec != FFT_PREC_FP32)
  void* d_tc;   // full twiddle tables of the tensor-core passes
  const gbfft::TileKernelInfo* ktc1;
  const gbfft::TileKernelInfo* ktc2;
  const float2* tctw1;
  const float2* tctw2;

  size_t ws_bytes;
  void* ws;
  int ws_owned;

  int* d_status;  // device status word (bounded waits)

  gbfft::ManyPlan* many;
  gbfft::FusedPlan* fused;  // both passes in one persistent launch (fused.cu)
  int launches;

  // multi-pass plans (four-step with two or three passes, 2-D)
  gbfft::PassDesc pass[gbfft::kMaxPasses];
  int npass;
  int lg3;            // three-pass split: log2 N3
  const float2* tw3;  // stage table of the third length
  const float2* ft2_lo;  // two-level table of the second four-step level
  const float2* ft2_hi;
  int ft2_s;
};
