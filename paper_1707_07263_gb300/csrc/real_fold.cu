// real_fold.cu -- real-data transforms of N = 2M reals with M = N1 * N2 a
// two-pass four-step length (2^15..2^21): the even/odd split folded into the
// row pass of the complex transform (real to complex) or into its column pass
// (complex to real), so that the transform takes two passes over memory
// instead of three.
//
// The row of N reals is read as M complex values z[m] = x[2m] + i x[2m+1]
// (Sec. 2.1's even/odd split) and Z = Eq. 1 of z (length M) is computed by the
// four-step split: a column pass leaves Y[k1][n2] (with the W_M^{n2 k1}
// twiddle) in the workspace, and the row pass transforms every row k1 of Y to
// Z[k1 + N1 k2].  The split then needs Z[k] and Z[M - k] together:
//     X[k] = E + W_N^k O,  E = (Z[k] + conj Z[M-k]) / 2,  O = (Z[k] - conj Z[M-k]) / (2i),
// and M - k = (N1 - k1) + N1 (N2 - 1 - k2) lies in row N1 - k1 (row 0 and row
// N1/2 are their own mirrors).  A tile of this kernel therefore takes H
// mirror pairs of rows (8 for rows of up to 2^10 points, 4 for 2^11, 2 for
// 2^12) -- rows u, u+1, ... and N1 - u, N1 - u - 1, ..., with rows 0 and N1/2
// as the pair of u = 0 -- runs their 2H row FFTs with the same Stockham
// passes as the row pass (tile_fft.cuh, last pass left in shared memory,
// transposed so that a warp reads 2H rows at one k2 without bank conflicts),
// and computes every X[k] of those rows from shared memory, stored as runs of
// H consecutive k1 (8 bytes each).  X[M] comes from Z[0].
#include <cuda_runtime.h>

#include "gbfft_internal.h"
#include "tile_fft.cuh"
#include "tile_registry.h"

namespace gbfft {

// Mirror pairs of rows per tile: 8 for rows of 2^6..2^10 points, fewer for
// longer rows so that the tile fits shared memory (rows of 2^11: 4, 2^12: 2).
constexpr int fold_pairs(int lg2) { return lg2 <= 10 ? 8 : (lg2 == 11 ? 4 : 2); }

struct RFoldArgs {
  long long M;             // complex length (N / 2)
  int N1;                  // rows of the four-step view (power of two >= 16)
  int tiles_per_row;       // N1 / (2H)
  const float2* r_lo;      // W_N^k = r_lo[k & (2^r_s - 1)] * r_hi[k >> r_s], k < M
  const float2* r_hi;
  int r_s;
  int scale;               // 1: X[1..M-1] times s_int, X[0] and X[M] times s_end
  float s_int, s_end;
};

template <int LG2>
struct FoldCfg {
  static constexpr int H = fold_pairs(LG2), C = 2 * H;
  using Tile = TileCfg<LG2, C, false, false>;
  static constexpr int T = Tile::T;
  // the exchange tile, or the transposed rows left by the last pass if larger
  static constexpr int SMEM = cmax(Tile::SMEM_BYTES, (1 << LG2) * (C + 1) * 8);
};

template <int LG2>
__global__ void __launch_bounds__(FoldCfg<LG2>::T) r2c_fold_kernel(const TileArgs ta, const RFoldArgs f) {
  using Cfg = FoldCfg<LG2>;
  constexpr int N2 = 1 << LG2, H = Cfg::H, C = Cfg::C, T = Cfg::T;
  extern __shared__ float2 smem[];
  __shared__ long long s_off[C];
  __shared__ int s_k1[C];
  const long long tile = blockIdx.x;
  const long long b = tile / f.tiles_per_row;
  const int g = (int)(tile - b * f.tiles_per_row);
  if (threadIdx.x < C) {
    const int c = threadIdx.x, u = g * H + (c & (H - 1));
    const int k1 = c < H ? u : (u == 0 ? f.N1 / 2 : f.N1 - u);
    s_k1[c] = k1;
    s_off[c] = (long long)k1 * N2;
  }
  __syncthreads();
  TileArgs a = ta;
  a.col_off = s_off;
  a.ncols = C;
  float2 v[Cfg::Tile::P];
  tile_stage<LG2, C, false, false, 0, true, 0, 6>(v, smem, a, ta.in + b * ta.in_bstride, nullptr, 0, b, nullptr);

  // every Z of the C rows is in shared memory, Z_c[k2] at k2 * (C + 1) + c
  float2* xr = ta.out + b * (f.M + 1);
  const unsigned lo_mask = (1u << f.r_s) - 1u;
  for (int idx = threadIdx.x; idx < C * N2; idx += T) {
    const int c = idx & (C - 1), k2 = idx / C;
    const int k1 = s_k1[c];
    const bool self = (g == 0 && (c & (H - 1)) == 0);   // rows 0 and N1/2 mirror themselves
    const int pc = self ? c : (c ^ H);
    const int pk2 = (k1 == 0) ? ((N2 - k2) & (N2 - 1)) : (N2 - 1 - k2);
    const float2 zk = smem[k2 * (C + 1) + c];
    const float2 zm = smem[pk2 * (C + 1) + pc];
    const unsigned k = (unsigned)k1 + (unsigned)f.N1 * (unsigned)k2;
    const float2 w = cmul(__ldg(f.r_lo + (k & lo_mask)), __ldg(f.r_hi + (k >> f.r_s)));
    const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    float2 x = cadd(e, cmul(w, o));
    if (f.scale) {
      const float sc = k == 0 ? f.s_end : f.s_int;
      x = make_float2(x.x * sc, x.y * sc);
    }
    __stcs(xr + k, x);
    if (k == 0) {
      // X[M] = E[0] - O[0] (W_N^M = -1), real
      const float xm = zk.x - zk.y;
      __stcs(xr + f.M, make_float2(f.scale ? xm * f.s_end : xm, 0.f));
    }
  }
}

#define GBFFT_FOLD(LG) \
  {(const void*)&r2c_fold_kernel<LG>, FoldCfg<LG>::T, FoldCfg<LG>::SMEM, LG, FoldCfg<LG>::C, MAP_JJ}

// The fold kernel for rows of 2^lg2 points (2^6..2^12), or NULL.
const TileKernelInfo* r2c_fold_kernel_info(int lg2) {
  static const TileKernelInfo tab[] = {GBFFT_FOLD(6),  GBFFT_FOLD(7),  GBFFT_FOLD(8), GBFFT_FOLD(9),
                                       GBFFT_FOLD(10), GBFFT_FOLD(11), GBFFT_FOLD(12)};
  if (lg2 < 6 || lg2 > 12) return nullptr;
  return &tab[lg2 - 6];
}

// Complex-to-real transforms of the same lengths: the split that builds
// Z[m] = E + i O from X[m] and X[M - m] runs inside the column pass of the
// inverse complex transform (tile_fft.cuh, first-pass mode 7), which reads X
// straight from the rows of M + 1 values; X[M - m] lies in the mirror column
// N2 - n2 of the same transform, usually an L2 hit.  The column pass then
// continues as the complex plan's own (four-step twiddle, workspace), and the
// row pass is the complex plan's.
template <int LG1, int C>
__global__ void __launch_bounds__(TileCfg<LG1, C, true, true>::T) c2r_fold_kernel(const TileArgs a) {
  extern __shared__ float2 smem[];
  tile_body<LG1, C, true, true, false, 7>(a, (long long)blockIdx.x, smem);
}

#define GBFFT_CFOLD(LG, C) \
  {(const void*)&c2r_fold_kernel<LG, C>, TileCfg<LG, C, true, true>::T, TileCfg<LG, C, true, true>::SMEM_BYTES, LG, \
   C, MAP_CC}

// The folded column kernel for columns of 2^lg1 points, C per CTA (the inner
// plans' column tiles: 2^7 and 2^8 with 16 columns, 2^10 with 8), or NULL.
const TileKernelInfo* c2r_fold_kernel_info(int lg1, int C) {
  static const TileKernelInfo tab[] = {GBFFT_CFOLD(7, 16), GBFFT_CFOLD(8, 16), GBFFT_CFOLD(10, 8)};
  for (const TileKernelInfo& k : tab)
    if (k.lg == lg1 && k.C == C) return &k;
  return nullptr;
}

int r2c_fold_launch(const TileKernelInfo* k, const TileArgs& a, long long M, int N1, long long batch,
                    const float2* r_lo, const float2* r_hi, int r_s, int scale, float s_int, float s_end,
                    cudaStream_t s) {
  RFoldArgs f;
  f.M = M;
  f.N1 = N1;
  f.tiles_per_row = N1 / k->C;
  f.r_lo = r_lo;
  f.r_hi = r_hi;
  f.r_s = r_s;
  f.scale = scale;
  f.s_int = s_int;
  f.s_end = s_end;
  const long long tiles = (long long)f.tiles_per_row * batch;
  if (tiles < 1 || tiles > 0x7fffffffLL) return FFT_ERR_UNSUPPORTED;
  void* args[] = {(void*)&a, (void*)&f};
  return cudaLaunchKernel(k->fn, dim3((unsigned)tiles), dim3(k->threads), args, (size_t)k->smem_bytes, s) ==
                 cudaSuccess
             ? FFT_OK
             : FFT_ERR_CUDA;
}

}  // namespace gbfft
