// tile_fft_tma.cuh -- persistent, TMA-staged variant of the batched on-chip
// FFT (contiguous transforms in and out).
//
// Same Stockham passes as tile_fft.cuh, but the global->on-chip load is taken
// off the threads: each CTA loops over tiles, and while its registers and
// shared memory work on tile t, one elected thread has already issued a
// cp.async.bulk (TMA) copy of tile t+grid into a staging buffer, completed on
// an mbarrier.  Loads therefore stream continuously from HBM instead of in
// bursts between compute phases (the paper's Sec. 2.3.2 concern, reducing the
// cost of global-memory access, on hardware with an asynchronous copy engine).
//
// Shared memory per CTA:
//   S  staging tile, C*L complex, unpadded (TMA destination; first pass reads it)
//   X  exchange buffer between passes:
//        EX == 8: C*LP complex, padded 8-byte exchange (as tile_fft.cuh)
//        EX == 4: L floats, the real and imaginary halves exchanged one after
//                 the other through an XOR-swizzled word index
//                 n ^ (((n >> 5) * 9) & 31), which is bank-conflict-free for
//                 every pass pattern at L = 2^14 (two-way at most elsewhere).
//                 Used where the full 8-byte exchange would not leave room
//                 for the staging tile.
//
// Every wait on the mbarrier is bounded (clock64 budget); on expiry the CTA
// records FFT_ERR_TIMEOUT in the plan's status word and returns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbfft.h"
#include "tile_fft.cuh"

namespace gbfft {

__device__ __forceinline__ int swz4(int n) { return n ^ (((n >> 5) * 9) & 31); }

template <int LG, int C, int EX>
struct TmaCfg {
  static constexpr int L = 1 << LG;
  static constexpr int P = L < 16 ? L : 16;
  static constexpr int T = C * L / P;
  static constexpr int NST = radix_nst(LG);
  static constexpr int LP = TileCfg<LG, C, false, false>::LP;
  static constexpr int S_BYTES = C * L * 8;
  static constexpr int X_BYTES = NST > 1 ? (EX == 8 ? C * LP * 8 : C * L * 4) : 0;
  static constexpr int SMEM_BYTES = S_BYTES + X_BYTES;
  // CTAs per SM the register budget must allow (shared memory allows the
  // same): 3 for the 256-thread tiles, 2 for 2^13, 1 for 2^14.  With more
  // than one, one CTA's compute overlaps another's staging wait.
  static constexpr int MIN_BLOCKS = (LG == 13) ? 2 : (LG == 14 ? 1 : 3);
};

// (c, j) of butterfly i of this thread in pass S (j-fast mapping).
template <int LG, int C, int S>
__device__ __forceinline__ void tma_bfly(int tid, int i, int& c, int& j) {
  constexpr int L = 1 << LG, P = L < 16 ? L : 16, T = C * L / P;
  constexpr int LR = L >> radix_lgr(LG, S);
  const int b = tid + i * T;
  c = b / LR;
  j = b % LR;
}

// Twiddle + R-point DFT of pass S on the thread's NB butterflies.
template <int LG, int C, int S>
__device__ __forceinline__ void tma_compute(float2* v, const float2* tw, int tid) {
  constexpr int L = 1 << LG, P = L < 16 ? L : 16;
  constexpr int LGR = radix_lgr(LG, S), R = 1 << LGR;
  constexpr int NS = 1 << radix_lgns(LG, S);
  constexpr int NB = P / R;
  if constexpr (NS > 1) {
    const float2* t = tw + stage_tw_off(LG, S);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      int c, j;
      tma_bfly<LG, C, S>(tid, i, c, j);
      apply_stage_twiddle<R>(v + i * R, t, NS, j & (NS - 1));
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) dft_fwd<R>(v + i * R);
}

// Output position of element q of butterfly (c, j) after pass S.
template <int LG, int S>
__device__ __forceinline__ int tma_out_pos(int j, int q) {
  constexpr int LGR = radix_lgr(LG, S), LGNS = radix_lgns(LG, S), NS = 1 << LGNS;
  return ((j >> LGNS) << (LGNS + LGR)) + (j & (NS - 1)) + q * NS;
}

// Exchange pass S's outputs into pass S+1's inputs through X.
template <int LG, int C, int EX, int S>
__device__ __forceinline__ void tma_exchange(float2* v, void* Xraw, int tid) {
  using Cfg = TmaCfg<LG, C, EX>;
  constexpr int L = Cfg::L, P = Cfg::P, LP = Cfg::LP;
  constexpr int R0 = 1 << radix_lgr(LG, S), NB0 = P / R0;
  constexpr int R1 = 1 << radix_lgr(LG, S + 1), NB1 = P / R1, LR1 = L / R1;
  if constexpr (EX == 8) {
    float2* X = (float2*)Xraw;
    if constexpr (S > 0) __syncthreads();   // previous exchange fully read
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
      int c, j;
      tma_bfly<LG, C, S>(tid, i, c, j);
      float2* wp = X + c * LP + pidx(tma_out_pos<LG, S>(j, 0));
#pragma unroll
      for (int q = 0; q < R0; ++q) wp[pidx_c(q * (1 << radix_lgns(LG, S)))] = v[i * R0 + q];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB1; ++i) {
      int c, j;
      tma_bfly<LG, C, S + 1>(tid, i, c, j);
      const float2* rp = X + c * LP + pidx(j);
#pragma unroll
      for (int r = 0; r < R1; ++r) v[i * R1 + r] = rp[pidx_c(r * LR1)];
    }
  } else {
    static_assert(C == 1, "split exchange is compiled for one transform per CTA");
    float* X = (float*)Xraw;
    float t[P];
    if constexpr (S > 0) __syncthreads();
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
      int c, j;
      tma_bfly<LG, C, S>(tid, i, c, j);
#pragma unroll
      for (int q = 0; q < R0; ++q) X[swz4(tma_out_pos<LG, S>(j, q))] = v[i * R0 + q].x;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB1; ++i) {
      int c, j;
      tma_bfly<LG, C, S + 1>(tid, i, c, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) t[i * R1 + r] = X[swz4(j + r * LR1)];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
      int c, j;
      tma_bfly<LG, C, S>(tid, i, c, j);
#pragma unroll
      for (int q = 0; q < R0; ++q) X[swz4(tma_out_pos<LG, S>(j, q))] = v[i * R0 + q].y;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB1; ++i) {
      int c, j;
      tma_bfly<LG, C, S + 1>(tid, i, c, j);
#pragma unroll
      for (int r = 0; r < R1; ++r) v[i * R1 + r] = make_float2(t[i * R1 + r], X[swz4(j + r * LR1)]);
    }
  }
}

// Passes S.. of one tile: compute, exchange, recurse; the last pass stores.
template <int LG, int C, int EX, int S>
__device__ __forceinline__ void tma_passes(float2* v, void* X, const TileArgs& a, float2* gout, long long col0,
                                           int tid) {
  using Cfg = TmaCfg<LG, C, EX>;
  constexpr int L = Cfg::L, NST = Cfg::NST;
  tma_compute<LG, C, S>(v, a.tw, tid);
  if constexpr (S + 1 < NST) {
    tma_exchange<LG, C, EX, S>(v, X, tid);
    tma_passes<LG, C, EX, S + 1>(v, X, a, gout, col0, tid);
  } else {
    constexpr int R = 1 << radix_lgr(LG, S), NS = L / R;
    static_assert((L < 16 ? L : 16) == R, "last pass holds one butterfly per thread");
    int c, j;
    tma_bfly<LG, C, S>(tid, 0, c, j);
    if (a.scale_out) {
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = make_float2(v[q].x * a.sx, v[q].y * a.sy);
    }
    if (col0 + c < a.ncols) {
      float2* p = gout + (long long)c * L + j;
#pragma unroll
      for (int q = 0; q < R; ++q) __stcs(p + q * NS, v[q]);
    }
  }
}

// grid = persistent CTAs; tile t covers transforms [t*C, t*C + C) of the batch.
template <int LG, int C, int EX>
__global__ void __launch_bounds__(TmaCfg<LG, C, EX>::T, TmaCfg<LG, C, EX>::MIN_BLOCKS)
    tile_fft_tma_kernel(const TileArgs a, long long ntiles, int* status) {
  using Cfg = TmaCfg<LG, C, EX>;
  constexpr int L = Cfg::L, P = Cfg::P, NST = Cfg::NST;
  constexpr int R0 = 1 << radix_lgr(LG, 0), NB0 = P / R0, LR0 = L / R0;
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t mbar;
  float2* S = (float2*)smraw;
  void* X = smraw + Cfg::S_BYTES;
  const int tid = threadIdx.x;

  if (tid == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto issue = [&](long long t) {
    const long long col0 = t * C;
    const long long cols = (a.ncols - col0) < C ? (a.ncols - col0) : C;
    tma_load_1d(S, a.in + col0 * L, (uint32_t)(cols * L * 8), &mbar);
  };

  long long tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) issue(tile);
  uint32_t parity = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    if (!mbar_wait(&mbar, parity)) {
      if (tid == 0) atomicExch(status, FFT_ERR_TIMEOUT);
      mbar_wait(&mbar, parity);  // second bounded wait for the copy in flight
      return;
    }
    parity ^= 1u;
    // pass 0 inputs straight from the staging tile
    float2 v[P];
#pragma unroll
    for (int i = 0; i < NB0; ++i) {
      int c, j;
      tma_bfly<LG, C, 0>(tid, i, c, j);
#pragma unroll
      for (int r = 0; r < R0; ++r) v[i * R0 + r] = S[c * L + j + r * LR0];
    }
    if (a.conj_in) {
#pragma unroll
      for (int p = 0; p < P; ++p) v[p].y = -v[p].y;
    }
    __syncthreads();  // staging tile consumed: refill it with the next tile
    if (tid == 0 && tile + gridDim.x < ntiles) {
      fence_proxy_async();
      issue(tile + gridDim.x);
    }
    const long long col0 = tile * C;
    // (the barrier after the next tile's staging reads also orders this
    // tile's last exchange reads before the next exchange writes)
    tma_passes<LG, C, EX, 0>(v, X, a, a.out + col0 * L, col0, tid);
  }
}

}  // namespace gbfft
