// tc_fft.cuh -- radix-16 passes on the tensor cores.
//
// A radix-16 pass applies the 16-point DFT matrix F (F[q][r] = W_16^{qr}) to
// every butterfly's 16 twiddled inputs.  Writing F = Cm - i Sm with
// Cm[q][r] = cos(2*pi*qr/16) and Sm[q][r] = sin(2*pi*qr/16), the complex product
// Y = F X becomes four real 16x16 products:
//     Yr = Cm Xr + Sm Xi,      Yi = Cm Xi - Sm Xr.
// Each is one mma.sync.m16n8k16 per 8 butterflies (Cm / Sm as the A operand,
// the butterflies' real or imaginary parts as the B columns), BF16 or FP16
// operands with FP32 accumulation.  The split variants write every operand
// as hi + lo (hi = round(x), lo = round(x - hi)) and keep three of the four
// cross products, hi*hi + hi*lo + lo*hi, recovering about twice the operand
// precision.  Twiddles, the remainder pass and the four-step twiddle stay FP32.
//
// Data distribution in a tensor-core pass (warp w, lane = 4*gid + tig):
//   inputs  lane holds, for each of 4 groups of 8 butterflies
//           b = 32w + 8g + gid, the elements r in {2tig, 2tig+1, 2tig+8, 2tig+9}
//           (exactly the B-fragment layout);
//   outputs lane holds q in {gid, gid+8} of butterflies 32w + 8g + 2tig + {0,1}
//           (the accumulator layout).
// Passes exchange through a shared tile indexed by the XOR swizzle tcidx()
// (no padding), which a bank model shows keeps these fragment-ordered
// accesses, and the FP32 remainder pass's, at the two-wavefront minimum.
// The last pass stores pairs of adjacent outputs as 16-byte vectors.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tile_fft.cuh"

namespace gbfft {

enum { TC_BF16 = 1, TC_FP16 = 2, TC_BF16_SPLIT = 3, TC_FP16_SPLIT = 4 };

template <int PREC>
struct TcPrec {
  static constexpr bool BF16 = (PREC == TC_BF16 || PREC == TC_BF16_SPLIT);
  static constexpr bool SPLIT = (PREC >= TC_BF16_SPLIT);
};

// two floats -> one 32-bit register of two 16-bit values (lo in the low half)
template <bool BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  uint32_t d;
  if constexpr (BF16)
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  else
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

template <bool BF16>
__device__ __forceinline__ float2 unpack2(uint32_t v) {
  if constexpr (BF16) {
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
  } else {
    __half2 h;
    memcpy(&h, &v, 4);
    return __half22float2(h);
  }
}

// hi/lo split of a pair: hi = round(x), lo = round(x - hi)
template <bool BF16>
__device__ __forceinline__ void split2(float lo, float hi, uint32_t& h, uint32_t& l) {
  h = pack2<BF16>(lo, hi);
  const float2 f = unpack2<BF16>(h);
  l = pack2<BF16>(lo - f.x, hi - f.y);
}

template <bool BF16>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (BF16)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// cos(2*pi*m/16), m = 0..15
__constant__ float c_cos16[16] = {1.f, GBFFT_C8, GBFFT_R2, GBFFT_S8, 0.f, -GBFFT_S8, -GBFFT_R2, -GBFFT_C8,
                                  -1.f, -GBFFT_C8, -GBFFT_R2, -GBFFT_S8, 0.f, GBFFT_S8, GBFFT_R2, GBFFT_C8};
__device__ __forceinline__ float cos16(int m) { return c_cos16[m & 15]; }
__device__ __forceinline__ float sin16(int m) { return cos16(m - 4); }

// A fragments of Cm and Sm (and their lo parts for the split variants):
// A[0] = Cm hi, A[1] = Sm hi, A[2] = Cm lo, A[3] = Sm lo.
template <int PREC>
__device__ __forceinline__ void tc_dft_fragments(uint32_t (&A)[4][4]) {
  constexpr bool BF16 = TcPrec<PREC>::BF16;
  const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int reg = 0; reg < 4; ++reg) {
    const int row = gid + ((reg & 1) ? 8 : 0);
    const int col = 2 * tig + ((reg & 2) ? 8 : 0);
    const float c0 = cos16(row * col), c1 = cos16(row * (col + 1));
    const float s0 = sin16(row * col), s1 = sin16(row * (col + 1));
    split2<BF16>(c0, c1, A[0][reg], A[2][reg]);
    split2<BF16>(s0, s1, A[1][reg], A[3][reg]);
  }
}

// Full twiddle table for tensor-core passes: pass s (Ns > 1, radix 16) stores
// 15 rows of Ns entries, row r-1 column k = W_{16 Ns}^{r k}.
__host__ __device__ constexpr int tc_tw_off(int lg, int s) {
  return s == 0 ? 0 : tc_tw_off(lg, s - 1) + ((radix_lgns(lg, s - 1) > 0) ? 15 * (1 << radix_lgns(lg, s - 1)) : 0);
}
__host__ __device__ constexpr int tc_tw_size(int lg) { return tc_tw_off(lg, radix_nst(lg)); }

template <int LG, int C, bool CF>
__device__ __forceinline__ void tc_map(int b, int& c, int& j) {
  constexpr int LR = (1 << LG) / 16;
  if constexpr (CF) {
    c = b % C;
    j = b / C;
  } else {
    c = b / LR;
    j = b % LR;
  }
}

// One radix-16 pass S on the tensor cores.
template <int LG, int C, bool IN_CF, bool OUT_CF, int S, int PREC>
__device__ __forceinline__ void tc_pass(float2* sm, const TileArgs& a, const float2* gin, float2* gout,
                                        long long col0, const uint32_t (&A)[4][4]) {
  using Cfg = TileCfg<LG, C, IN_CF, OUT_CF, 1>;
  constexpr bool BF16 = TcPrec<PREC>::BF16, SPLIT = TcPrec<PREC>::SPLIT;
  constexpr int L = Cfg::L, NST = Cfg::NST, LP = Cfg::LP;
  static_assert(radix_lgr(LG, S) == 4, "tensor-core passes are radix 16");
  constexpr int LGNS = radix_lgns(LG, S), NS = 1 << LGNS, LR = L / 16;
  constexpr bool FIRST = (S == 0), LAST = (S == NST - 1);
  constexpr bool CF = (FIRST && IN_CF) || (LAST && OUT_CF);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;

  float2 x[4][4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    int c, j;
    tc_map<LG, C, CF>(warp * 32 + g * 8 + gid, c, j);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 2 * tig + (e & 1) + ((e & 2) ? 8 : 0);
      if constexpr (FIRST) {
        const bool ok = (col0 + c) < a.ncols;
        const float2* p = gin + c * a.in_sc + (long long)(j + r * LR) * a.in_sn;
        x[g][e] = ok ? (a.stream_in ? __ldcs(p) : __ldcg(p)) : make_float2(0.f, 0.f);
        if (a.conj_in) x[g][e].y = -x[g][e].y;
      } else {
        x[g][e] = sm[c * LP + tcidx(j + r * LR)];
      }
      if constexpr (NS > 1) {
        if (r > 0) x[g][e] = cmul(x[g][e], __ldg(a.tw + tc_tw_off(LG, S) + (r - 1) * NS + (j & (NS - 1))));
      }
    }
  }

  float2 y[4][4];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    uint32_t br[2], bi[2], brl[2], bil[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if constexpr (SPLIT) {
        split2<BF16>(x[g][2 * h].x, x[g][2 * h + 1].x, br[h], brl[h]);
        split2<BF16>(x[g][2 * h].y, x[g][2 * h + 1].y, bi[h], bil[h]);
      } else {
        br[h] = pack2<BF16>(x[g][2 * h].x, x[g][2 * h + 1].x);
        bi[h] = pack2<BF16>(x[g][2 * h].y, x[g][2 * h + 1].y);
      }
    }
    float dr[4] = {0.f, 0.f, 0.f, 0.f}, di[4] = {0.f, 0.f, 0.f, 0.f};
    const uint32_t nr0 = br[0] ^ 0x80008000u, nr1 = br[1] ^ 0x80008000u;
    mma16816<BF16>(dr, A[0], br[0], br[1]);   // Cm Xr
    mma16816<BF16>(dr, A[1], bi[0], bi[1]);   // + Sm Xi
    mma16816<BF16>(di, A[0], bi[0], bi[1]);   // Cm Xi
    mma16816<BF16>(di, A[1], nr0, nr1);       // - Sm Xr
    if constexpr (SPLIT) {
      const uint32_t nl0 = brl[0] ^ 0x80008000u, nl1 = brl[1] ^ 0x80008000u;
      mma16816<BF16>(dr, A[0], brl[0], brl[1]);
      mma16816<BF16>(dr, A[2], br[0], br[1]);
      mma16816<BF16>(dr, A[1], bil[0], bil[1]);
      mma16816<BF16>(dr, A[3], bi[0], bi[1]);
      mma16816<BF16>(di, A[0], bil[0], bil[1]);
      mma16816<BF16>(di, A[2], bi[0], bi[1]);
      mma16816<BF16>(di, A[1], nl0, nl1);
      mma16816<BF16>(di, A[3], nr0, nr1);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) y[g][e] = make_float2(dr[e], di[e]);
  }

  if constexpr (LAST) {
    // outputs e = 0, 1 (and 2, 3) are butterflies 2*tig and 2*tig+1 at the same
    // q: adjacent j (j-fast) or adjacent columns (c-fast, out_sc == 1), so
    // each pair goes out as one 16-byte store
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = gid + (h ? 8 : 0);
        int c, j;
        tc_map<LG, C, CF>(warp * 32 + g * 8 + 2 * tig, c, j);
        const int k = j + q * NS;
        float2 v0 = y[g][2 * h], v1 = y[g][2 * h + 1];
        if (Cfg::EPI && a.ft_lgN) {
          const unsigned mask = (1u << a.ft_s) - 1u;
          const unsigned m0 = (unsigned)(col0 + c) * (unsigned)k;
          v0 = cmul(v0, cmul(__ldg(a.ft_lo + (m0 & mask)), __ldg(a.ft_hi + (m0 >> a.ft_s))));
          const unsigned m1 = CF ? (unsigned)(col0 + c + 1) * (unsigned)k : (unsigned)(col0 + c) * (unsigned)(k + 1);
          v1 = cmul(v1, cmul(__ldg(a.ft_lo + (m1 & mask)), __ldg(a.ft_hi + (m1 >> a.ft_s))));
        }
        if (a.scale_out) {
          v0 = make_float2(v0.x * a.sx, v0.y * a.sy);
          v1 = make_float2(v1.x * a.sx, v1.y * a.sy);
        }
        if ((col0 + c) < a.ncols) {
          float4* p = (float4*)(gout + c * a.out_sc + (long long)k * a.out_sn);
          const float4 w = make_float4(v0.x, v0.y, v1.x, v1.y);
          if (a.stream_out)
            __stcs(p, w);
          else
            __stcg(p, w);
        }
      }
  } else {
    if constexpr (!FIRST) __syncthreads();
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int q = gid + ((e & 2) ? 8 : 0);
        int c, j;
        tc_map<LG, C, CF>(warp * 32 + g * 8 + 2 * tig + (e & 1), c, j);
        const int pos = ((j >> LGNS) << (LGNS + 4)) + (j & (NS - 1)) + q * NS;
        sm[c * LP + tcidx(pos)] = y[g][e];
      }
    __syncthreads();
  }
}

// FP32 remainder pass or tensor-core radix-16 pass, then the next one.
template <int LG, int C, bool IN_CF, bool OUT_CF, int S, int PREC>
__device__ __forceinline__ void tc_stage(float2* sm, const TileArgs& a, const float2* gin, float2* gout,
                                         long long col0, const float2* epi_tab, const uint32_t (&A)[4][4]) {
  using Cfg = TileCfg<LG, C, IN_CF, OUT_CF, 1>;
  if constexpr (radix_lgr(LG, S) == 4) {
    tc_pass<LG, C, IN_CF, OUT_CF, S, PREC>(sm, a, gin, gout, col0, A);
  } else {
    float2 v[Cfg::P];
    tile_pass<LG, C, IN_CF, OUT_CF, S, false, 0, 1>(v, sm, a, gin, gout, col0, 0, epi_tab);
  }
  if constexpr (S + 1 < Cfg::NST) tc_stage<LG, C, IN_CF, OUT_CF, S + 1, PREC>(sm, a, gin, gout, col0, epi_tab, A);
}

template <int LG, int C, bool IN_CF, bool OUT_CF, int PREC>
__global__ void __launch_bounds__(TileCfg<LG, C, IN_CF, OUT_CF, 1>::T) tc_fft_kernel(const TileArgs a) {
  using Cfg = TileCfg<LG, C, IN_CF, OUT_CF, 1>;
  static_assert(Cfg::T % 32 == 0 && Cfg::P == 16, "tensor-core tiles use whole warps of 16-point threads");
  extern __shared__ float2 smem[];
  const long long tile = (long long)blockIdx.x;
  const long long b = tile / a.tiles_per_batch;
  const long long g = tile - b * a.tiles_per_batch;
  const long long col0 = g * C;
  const float2* gin = a.in + b * a.in_bstride + g * a.in_gstride;
  float2* gout = a.out + b * a.out_bstride + g * a.out_gstride;
  uint32_t A[4][4];
  tc_dft_fragments<PREC>(A);
  tc_stage<LG, C, IN_CF, OUT_CF, 0, PREC>(smem, a, gin, gout, col0, smem + Cfg::SM_TILE, A);
}

}  // namespace gbfft
