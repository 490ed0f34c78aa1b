// fused.cu -- the two passes of the four-step split in ONE persistent launch,
// with the intermediate kept in L2.
//
// The paper's two-exchange scheme (Sec. 2.3.2) writes the intermediate to
// global memory after the first pass and reads it back in the second, so a
// two-pass transform moves every point through DRAM twice.  Here the batch is
// cut into slabs of whole transforms (about 16 MB each) and the passes are
// pipelined slab by slab through a ring of R = 3 workspace slots:
//     A(0), A(1) B(0), A(2) B(1), ..., A(S-1) B(S-2), B(S-1)
// A(s) = column tiles of slab s (input -> slot s mod R, with the W_N twiddle),
// B(s) = row tiles of slab s (slot -> output, transposed).  A slot is rewritten
// only after the row tiles that read it are done, so the 3 x 16 MB of
// workspace stays resident in L2 (about 126 MB usable) while inputs and
// outputs stream with evict-first hints: DRAM sees roughly one read and one
// write per point.
// With three slots, A(s) waits for B(s-3), which sits a whole group of items
// earlier in the sequence, so CTAs working through the sequence in order do
// not stall on work dispatched just before them.
//
// CTAs claim items in sequence order from a queue head (each CTA holds its
// current item and the one it claimed next).  Every item waits only for items
// earlier in the sequence (B(s) for A(s); A(s) for B(s-R)), so the earliest
// unfinished item is always being worked on and the waits end.  They are still bounded (clock64 budget); a timeout records
// FFT_ERR_TIMEOUT in the plan's status word.  Counters grow monotonically
// within one exec and are cleared by a memset issued with every exec (so exec
// can be captured in a CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "gbfft_internal.h"
#include "tile_fft.cuh"

namespace gbfft {

constexpr int kFusedThreads = 256;
constexpr int kFusedSlots = 3;

struct FusedItem {
  int kind;   // 0 column tile (pass A), 1 row tile (pass B)
  int slab;
  int tile;   // tile index within the slab's pass
};

struct FusedArgs {
  TileArgs A, B;           // per-pass templates; in/out/tile bases set per item
  const FusedItem* items;
  long long nitems;
  long long N;             // transform length
  long long slab_T;        // transforms per slab
  long long batch;
  int tilesA, tilesB;      // tiles per transform of each pass
  float2* ws;              // kFusedSlots slots of slab_T * N points
  unsigned long long* head;  // queue head (items are claimed in sequence order)
  int* doneA;              // [kFusedSlots]
  int* doneB;              // [kFusedSlots]
  int* status;
  long long wait_budget;
};

// the split and tile widths of the fused kernel for length 2^lgN: 256-thread
// CTAs, each pass tile 4096 points
__host__ __device__ constexpr int fused_lg1(int lgN) { return lgN / 2; }
__host__ __device__ constexpr int fused_lg2(int lgN) { return lgN - lgN / 2; }

__device__ __forceinline__ bool fused_wait(const int* flag, int target, long long budget) {
  const long long t0 = clock64();
  while (true) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= target) return true;
    if (clock64() - t0 > budget) return false;
    __nanosleep(32);
  }
}

__device__ __forceinline__ long long slab_count(const FusedArgs& f, int s) {
  const long long rem = f.batch - (long long)s * f.slab_T;
  return rem < f.slab_T ? rem : f.slab_T;
}

// items of one kind completed in slot (s mod R) once slab s is finished
__device__ __forceinline__ int fused_target(const FusedArgs& f, int s, int tiles_per_transform) {
  const int gen = s / kFusedSlots;
  return (int)((long long)gen * f.slab_T * tiles_per_transform + slab_count(f, s) * tiles_per_transform);
}

template <int LGN>
__global__ void __launch_bounds__(kFusedThreads, 3) fused_kernel(const FusedArgs f) {
  constexpr int LG1 = fused_lg1(LGN), LG2 = fused_lg2(LGN);
  constexpr int C1 = 4096 >> LG1, C2 = 4096 >> LG2;
  extern __shared__ float2 smem[];
  __shared__ long long s_next;
  if (threadIdx.x == 0) s_next = atomicAdd(f.head, 1ULL);
  __syncthreads();
  long long i = s_next;
  while (i < f.nitems) {
    // claim the following item now; its index is read after this item's
    // closing barrier (items are claimed in sequence order)
    if (threadIdx.x == 0) s_next = atomicAdd(f.head, 1ULL);
    const FusedItem it = f.items[i];
    const int slot = it.slab % kFusedSlots;
    float2* slot_base = f.ws + (long long)slot * f.slab_T * f.N;
    const long long first_tr = (long long)it.slab * f.slab_T;
    if (it.kind == 0) {
      if (it.slab >= kFusedSlots) {
        // the row tiles of slab s - R must have read this slot
        if (threadIdx.x == 0 &&
            !fused_wait(f.doneB + slot, fused_target(f, it.slab - kFusedSlots, f.tilesB), f.wait_budget))
          atomicExch(f.status, FFT_ERR_TIMEOUT);
        __syncthreads();
      }
      const long long tr = it.tile / f.tilesA, g = it.tile % f.tilesA;
      TileArgs a = f.A;
      a.in = f.A.in + (first_tr + tr) * f.N;
      a.out = slot_base + tr * f.N;
      tile_body<LG1, C1, true, true>(a, g, smem);
      // publish the tile: every thread fences its own workspace stores, the
      // barrier collects the CTA, then the counter moves
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(f.doneA + slot, 1);
    } else {
      if (threadIdx.x == 0 && !fused_wait(f.doneA + slot, fused_target(f, it.slab, f.tilesA), f.wait_budget))
        atomicExch(f.status, FFT_ERR_TIMEOUT);
      __syncthreads();
      const long long tr = it.tile / f.tilesB, g = it.tile % f.tilesB;
      TileArgs b = f.B;
      b.in = slot_base + tr * f.N;
      b.out = f.B.out + (first_tr + tr) * f.N;
      tile_body<LG2, C2, false, true>(b, g, smem);
      // every read of the slot is done once all threads pass the barrier
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(f.doneB + slot, 1);
      }
    }
    __syncthreads();  // s_next is published; shared memory free for the next item
    i = s_next;
  }
}

template <int LGN>
constexpr int fused_smem() {
  return cmax(TileCfg<fused_lg1(LGN), (4096 >> fused_lg1(LGN)), true, true>::SMEM_BYTES,
              TileCfg<fused_lg2(LGN), (4096 >> fused_lg2(LGN)), false, true>::SMEM_BYTES);
}

struct FusedKernel {
  const void* fn;
  int smem;
};

static FusedKernel fused_kernel_for(int lgN) {
  switch (lgN) {
    case 13: return {(const void*)&fused_kernel<13>, fused_smem<13>()};
    case 14: return {(const void*)&fused_kernel<14>, fused_smem<14>()};
    case 15: return {(const void*)&fused_kernel<15>, fused_smem<15>()};
    case 16: return {(const void*)&fused_kernel<16>, fused_smem<16>()};
    case 17: return {(const void*)&fused_kernel<17>, fused_smem<17>()};
    case 18: return {(const void*)&fused_kernel<18>, fused_smem<18>()};
  }
  return {nullptr, 0};
}

struct FusedPlan {
  void* d_mem = nullptr;   // items + counters
  FusedItem* items = nullptr;
  int* counters = nullptr;
  FusedArgs args{};
  FusedKernel k{};
  int grid = 0;
};

void fused_plan_free(fft_plan* p) {
  if (!p->fused) return;
  if (p->fused->d_mem) cudaFree(p->fused->d_mem);
  delete p->fused;
  p->fused = nullptr;
}

bool fused_supported(int lgN) { return fused_kernel_for(lgN).fn != nullptr; }

// Builds the fused plan for `batch` transforms of length 2^lgN; the stage and
// W_N twiddle tables (tw1 = 2^lg1, tw2 = 2^lg2, ft for N) are already built.
int fused_plan_init(fft_plan* p, int lgN, long long slab_bytes) {
  const FusedKernel k = fused_kernel_for(lgN);
  if (!k.fn) return FFT_ERR_UNSUPPORTED;
  const int lg1 = fused_lg1(lgN), lg2 = fused_lg2(lgN);
  const long long N = 1LL << lgN, N1 = 1LL << lg1, N2 = 1LL << lg2;
  const int C1 = 4096 >> lg1, C2 = 4096 >> lg2;
  long long slab_T = std::max<long long>(1, slab_bytes / (N * 8));
  slab_T = std::min<long long>(slab_T, p->batch);
  const int S = (int)((p->batch + slab_T - 1) / slab_T);
  const int tilesA = (int)(N2 / C1), tilesB = (int)(N1 / C2);
  std::vector<FusedItem> items;
  auto push_slab = [&](int kind, int s) {
    const long long cnt = std::min<long long>(slab_T, p->batch - (long long)s * slab_T);
    const long long n_tiles = cnt * (kind == 0 ? tilesA : tilesB);
    for (long long t = 0; t < n_tiles; ++t) items.push_back(FusedItem{kind, s, (int)t});
  };
  push_slab(0, 0);
  for (int s = 1; s < S; ++s) {
    push_slab(0, s);
    push_slab(1, s - 1);
  }
  push_slab(1, S - 1);

  FusedPlan* fp = new (std::nothrow) FusedPlan;
  if (!fp) return FFT_ERR_ALLOC;
  p->fused = fp;
  const size_t b_items = (sizeof(FusedItem) * items.size() + 255) & ~(size_t)255;
  if (cudaMalloc(&fp->d_mem, b_items + 256) != cudaSuccess) return FFT_ERR_ALLOC;
  static_assert((2 + 2 * kFusedSlots) * sizeof(int) <= 256, "counters fit the tail of the allocation");
  fp->items = (FusedItem*)fp->d_mem;
  fp->counters = (int*)((char*)fp->d_mem + b_items);
  if (cudaMemcpy(fp->items, items.data(), sizeof(FusedItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return FFT_ERR_CUDA;
  if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem) != cudaSuccess)
    return FFT_ERR_CUDA;
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, kFusedThreads, k.smem) != cudaSuccess ||
      per_sm < 1)
    return FFT_ERR_CUDA;
  fp->k = k;
  fp->grid = (int)std::min<long long>((long long)per_sm * sms, (long long)items.size());

  FusedArgs& f = fp->args;
  memset(&f, 0, sizeof(f));
  f.items = fp->items;
  f.nitems = (long long)items.size();
  f.N = N;
  f.slab_T = slab_T;
  f.batch = p->batch;
  f.tilesA = tilesA;
  f.tilesB = tilesB;
  f.head = (unsigned long long*)fp->counters;
  f.doneA = fp->counters + 2;
  f.doneB = fp->counters + 2 + kFusedSlots;
  f.status = p->d_status;
  f.wait_budget = 4000000000LL;
  // pass A: columns [g*C1, g*C1+C1) of x[N2*n1 + n2] within one transform,
  // scaled by W_N^{n2*k1}, to the slot as Y[k1][n2]
  TileArgs& A = f.A;
  A.tw = p->tw1;
  A.tiles_per_batch = 1LL << 40;
  A.in_gstride = A.out_gstride = C1;
  A.in_sc = A.out_sc = 1;
  A.in_sn = A.out_sn = N2;
  A.ncols = N2;
  A.ft_lo = p->ft_lo;
  A.ft_hi = p->ft_hi;
  A.ft_lgN = lgN;
  A.ft_s = p->ft_s;
  A.stream_in = 1;
  A.stream_out = 0;
  // pass B: rows [g*C2, g*C2+C2) of Y, to X[k1 + N1*k2]
  TileArgs& B = f.B;
  B.tw = p->tw2;
  B.tiles_per_batch = 1LL << 40;
  B.in_gstride = (long long)C2 * N2;
  B.in_sc = N2;
  B.in_sn = 1;
  B.out_gstride = C2;
  B.out_sc = 1;
  B.out_sn = N1;
  B.ncols = N1;
  B.stream_in = 0;
  B.stream_out = 1;
  p->ws_bytes = (size_t)kFusedSlots * (size_t)slab_T * (size_t)N * 8;
  p->launches = 1;
  p->lg1 = lg1;
  p->lg2 = lg2;
  p->c1 = C1;
  p->c2 = C2;
  return FFT_OK;
}

int fused_exec(fft_plan* p, const float2* in, float2* out, int conj, float sx, float sy, int scale,
               cudaStream_t s) {
  FusedPlan* fp = p->fused;
  if (!p->ws) return FFT_ERR_NO_WORKSPACE;
  FusedArgs f = fp->args;
  f.A.in = in;
  f.A.conj_in = conj;
  f.B.out = out;
  f.B.scale_out = scale;
  f.B.sx = sx;
  f.B.sy = sy;
  f.ws = (float2*)p->ws;
  if (cudaMemsetAsync(fp->counters, 0, sizeof(int) * (2 + 2 * kFusedSlots), s) != cudaSuccess) return FFT_ERR_CUDA;
  void* args[] = {(void*)&f};
  if (cudaLaunchKernel(fp->k.fn, dim3(fp->grid), dim3(kFusedThreads), args, (size_t)fp->k.smem, s) != cudaSuccess)
    return FFT_ERR_CUDA;
  return FFT_OK;
}

}  // namespace gbfft
