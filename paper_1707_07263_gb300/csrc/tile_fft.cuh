// tile_fft.cuh -- the on-chip sub-FFT: one CTA transforms a tile of C
// power-of-two transforms of length L = 2^LG entirely in registers and shared
// memory (paper Sec. 2.3.2: every butterfly level runs in shared memory; global
// memory is touched once to load the piece and once to store it).
//
// Algorithm: Stockham autosort radix-R passes (natural-order output, no bit
// reversal).  With Ns = product of the radices already applied, pass s takes,
// for each butterfly j in [0, L/R):
//     v[r] = a[j + r*L/R] * W_{Ns*R}^{r*(j mod Ns)},   r = 0..R-1
//     V    = R-point DFT of v
//     b[(j div Ns)*Ns*R + (j mod Ns) + q*Ns] = V[q],   q = 0..R-1
// After the last pass Ns*R = L and b holds X(k) of Eq. 1 in natural order.
// Radices: one remainder pass of radix 2/4/8 first (if LG is not a multiple
// of 4), then radix-16 passes.  Each thread owns P = min(16, L) points.
//
// Data movement: the first pass reads straight from global memory into
// registers, the last pass writes straight from registers to global memory;
// the passes in between exchange through a padded shared-memory tile
// (index n -> n + n/16, plus a per-configuration row pad) that keeps every
// warp-wide 8-byte access at the 2-wavefront minimum (the paper's Sec. 2.3.3
// pads its 16x33 array for the same reason; GB300 has 32 banks of 4 bytes).
//
// Two thread mappings per pass:
//   j-fast: consecutive lanes take consecutive butterflies j of one
//           transform -- coalesced when a transform's points are contiguous.
//   c-fast: consecutive lanes take the same j of adjacent transforms c --
//           coalesced when the C transforms are adjacent columns (the
//           paper's column pass over 16-wide groups, Sec. 2.3.2).
// IN_CF / OUT_CF select c-fast for the global-facing first / last pass.
//
// Direction (Eq. 2, Eq. 4): the kernels always apply the forward W_N; the
// conjugate direction is obtained as conj(F(conj(x))), i.e. by negating the
// imaginary part on load and on store, and the 1/N of Eq. 2 is folded into
// the store.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbfft.h"
#include "ct_trig.h"
#include "fft_common.cuh"
#include "tma_util.cuh"

namespace gbfft {

// ---------------------------------------------------------------------------
// Radix schedule for L = 2^LG with radices up to 2^lgm (lgm = 4, radix 16, for
// every kernel but the smaller-radix single-pass variants the autotuner may
// pick): the remainder pass first, then full-radix passes (rev = false); or
// the full-radix passes first and the remainder pass last (rev = true: the
// second transform of the fused range-compression kernel, whose first pass
// then needs exactly the points that the first transform's last pass left in
// each thread).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int radix_nst(int lg, int lgm = 4) { return (lg + lgm - 1) / lgm; }
__host__ __device__ constexpr int radix_lgr(int lg, int s, bool rev = false, int lgm = 4) {
  return (lg % lgm != 0 && s == (rev ? radix_nst(lg, lgm) - 1 : 0)) ? (lg % lgm) : lgm;
}
__host__ __device__ constexpr int radix_lgns(int lg, int s, bool rev = false, int lgm = 4) {
  return s == 0 ? 0 : radix_lgns(lg, s - 1, rev, lgm) + radix_lgr(lg, s - 1, rev, lgm);
}
// Offset (in complex entries) of pass s's twiddle basis in the per-length
// table.  Pass s with Ns > 1 stores lgr(s) rows of Ns entries:
//   row e (e = 0..lgr-1), column k:  W_{Ns*R}^{(2^e) * k}.
__host__ __device__ constexpr int stage_tw_off(int lg, int s, bool rev = false, int lgm = 4) {
  return s == 0 ? 0
                : stage_tw_off(lg, s - 1, rev, lgm) +
                      ((radix_lgns(lg, s - 1, rev, lgm) > 0)
                           ? radix_lgr(lg, s - 1, rev, lgm) * (1 << radix_lgns(lg, s - 1, rev, lgm))
                           : 0);
}
__host__ __device__ constexpr int stage_tw_size(int lg, bool rev = false, int lgm = 4) {
  return stage_tw_off(lg, radix_nst(lg, lgm), rev, lgm);
}

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Row pad (complex entries) so that the lane groups of one warp that touch
// different transforms land on disjoint banks (derived from a bank model of
// every pass's access pattern).
__host__ __device__ constexpr int tile_group_count(int lg, int C, bool in_cf, bool out_cf, int s, int lgm = 4) {
  return (s >= radix_nst(lg, lgm))
             ? 1
             : cmax(cmin(C, (((s == 0) && in_cf) || ((s == radix_nst(lg, lgm) - 1) && out_cf))
                                  ? cmin(C, 32)
                                  : (((1 << lg) >> radix_lgr(lg, s, false, lgm)) < 32
                                         ? cmax(1, 32 / ((1 << lg) >> radix_lgr(lg, s, false, lgm)))
                                         : 1)),
                    tile_group_count(lg, C, in_cf, out_cf, s + 1, lgm));
}
__host__ __device__ constexpr int tile_row_pad(int lg, int C, bool in_cf, bool out_cf, int lgm = 4) {
  return ((32 / tile_group_count(lg, C, in_cf, out_cf, 0, lgm)) % 16 - (((1 << lg) + ((1 << lg) >> 4)) % 16) + 32) %
         16;
}

// Shared-memory index of element n of a transform's row:
//   IDX 0  padded: n + n/16 (FP32 kernels);
//   IDX 1  XOR swizzle inside 16-element blocks, no padding (tensor-core
//          kernels, whose fragment-ordered accesses it keeps conflict-free).
template <int IDX>
__host__ __device__ constexpr int tc_row_pad(int C, bool in_cf, bool out_cf) {
  return (in_cf || out_cf) ? (C == 2 ? 4 : 2) : 0;
}

// LGM: log2 of the largest radix, which is also the number of points each
// thread holds (4: radix 16, every kernel but the autotuner's smaller-radix
// single-pass variants, 3: radix 8, 2: radix 4).
template <int LG, int C, bool IN_CF, bool OUT_CF, int IDX = 0, int LGM = 4>
struct TileCfg {
  static constexpr int L = 1 << LG;
  static constexpr int P = L < (1 << LGM) ? L : (1 << LGM);   // points per thread
  static constexpr int T = C * L / P;                         // threads per CTA
  static constexpr int NST = radix_nst(LG, LGM);
  static constexpr int LP = IDX == 0 ? L + (L >> 4) + tile_row_pad(LG, C, IN_CF, OUT_CF, LGM)
                                     : L + tc_row_pad<IDX>(C, IN_CF, OUT_CF);
  static constexpr int SM_TILE = NST > 1 ? C * LP : 0;   // complex entries
  static constexpr bool EPI = IN_CF && OUT_CF;            // column pass: may carry the four-step twiddle
  static constexpr int SM_EPI = EPI ? C * 16 : 0;         // four-step per-column step table
  static constexpr int SMEM_BYTES = (SM_TILE + SM_EPI) * 8;
};

__device__ __forceinline__ int pidx(int n) { return n + (n >> 4); }
// pidx of a compile-time offset.  For every pass, pidx(base + d) ==
// pidx(base) + pidx_c(d) holds for the element offsets d = r*L/R (reads) and
// d = q*Ns (writes): d is a multiple of 16, or base's low four bits plus d stay
// inside one 16-block.  The shared-memory address of each of a butterfly's R
// elements is then one base register plus an immediate.
__host__ __device__ constexpr int pidx_c(int n) { return n + (n >> 4); }
__device__ __forceinline__ int tcidx(int n) { return n ^ ((((n >> 4) * 13) ^ (n >> 6)) & 15); }
template <int IDX>
__device__ __forceinline__ int sidx(int n) {
  if constexpr (IDX == 0)
    return pidx(n);
  else
    return tcidx(n);
}

// ---------------------------------------------------------------------------
// Kernel arguments.  Tile t = (b, g) with b = t / tiles_per_batch and
// g = t % tiles_per_batch; element (c, n) of the tile lives at
//   in  + b*in_bstride  + g*in_gstride  + c*in_sc  + n*in_sn
//   out + b*out_bstride + g*out_gstride + c*out_sc + n*out_sn
// (all in complex units).  Column index g*C + c >= ncols is skipped (ragged
// last tile of a batch).
// ---------------------------------------------------------------------------
struct TileArgs {
  const float2* in;
  float2* out;
  const float2* tw;  // per-length stage twiddle table (stage_tw_size(LG) entries)
  long long tiles_per_batch;
  long long in_bstride, in_gstride, in_sc, in_sn;
  long long out_bstride, out_gstride, out_sc, out_sn;
  long long ncols;
  // Four-step twiddle W_N^{(g*C+c) * k} on the output (k = output index),
  // N = 2^ft_lgN, from the two-level table W_N^m = lo[m & (2^ft_s-1)] * hi[m >> ft_s].
  const float2* ft_lo;
  const float2* ft_hi;
  int ft_lgN;  // 0: no four-step twiddle
  int ft_s;
  int conj_in;      // negate imaginary parts on load
  int scale_out;    // multiply outputs by (sx, sy) component-wise
  float sx, sy;
  int stream_in;    // 1: read with evict-first (.cs) hint; 0: keep in L2 (.cg)
  int stream_out;   // 1: write with evict-first (.cs) hint
  // Per-column element offsets (OFFS variants only): column c of the tile
  // starts at in + col_off[c] / out + col_off[c]; in_sc/out_sc are unused.
  const long long* col_off;
  // Optional outer batch: the batch index bq = tile / tiles_per_batch splits
  // into b2 = bq / nb1 and b = bq % nb1, adding b2*in_b2stride (out_b2stride).
  // nb1 = 0 means no outer batch.
  long long nb1, in_b2stride, out_b2stride;
  // Four-step twiddle multiplier: 0 = the column index g*C + c, 1 = the
  // (inner) batch index b.
  int ft_by_batch;
  // Radix-2 decimation-in-frequency split across two CTAs (PRE == 1 passes):
  // element n of the half-length transform k1 is
  //   (x[n] + (-1)^k1 x[n + pre_half]) * W_{2 pre_half}^{n k1},
  // with W_{2 pre_half}^n read from pre_tw; k1 arrives as the pass's bidx.
  long long pre_half;
  const float2* pre_tw;
  // Frequency-domain filter of range compression (Sec. 3, Sec. 4: FFT-based
  // SAR processing), complex64 in natural frequency order.  Fused one-pass
  // kernel (POST == 1): output k of the forward transform is multiplied by
  // filt[k].  Last pass of a multi-pass plan (j-fast in, c-fast out), when
  // filt != NULL: the element stored at offset o from `out` is multiplied by
  // filt[o & filt_mask] (filt_mask = N - 1, rows N apart) before the scaling.
  const float2* filt;
  long long filt_mask;
  int filt_conj;    // 1: multiply by conj(filt[k]) instead (the adjoint of range compression)
  // Stage table of the remainder-last schedule (REV passes).
  const float2* tw_rev;
  // Real-data transforms of length N = 2L (rows of L complex values = 2L
  // reals): r_w[k] = W_N^k, k < L.
  const float2* r_w;
  // Complex-to-real first pass (PRE == 5): 1 doubles the real parts of X[0]
  // and X[L] (with the scale 1 instead of 1/L this is the adjoint of the
  // real-to-complex transform).  The real-to-complex last pass (POST == 3)
  // takes scale_out: outputs X[1..L-1] times sx, X[0] and X[L] times sy (the
  // adjoint of the complex-to-real transform has sx = 2/N, sy = 1/N).
  int r_end2;
  // Complex-to-real split folded into a four-step column pass (PRE == 7):
  // W_N^m = r_w[m & (2^r_s - 1)] * r_hi[m >> r_s], m < M (two levels).
  const float2* r_hi;
  int r_s;
};

// Filter value of range compression at frequency index k (conjugated for the
// adjoint).
__device__ __forceinline__ float2 filt_at(const TileArgs& a, long long k) {
  const float2 f = __ldg(a.filt + k);
  return a.filt_conj ? make_float2(f.x, -f.y) : f;
}

// Z[m] = E + i O of a complex-to-real split for the R inputs
// m = m0 + r M/R of one butterfly: E = (X[m] + conj X[M-m]) / 2,
// O = (X[m] - conj X[M-m]) conj(W_N^m) / 2, with W_N^m = w0 W_{2R}^r
// (W_{2R}^r = exp(-i pi r / R) as compile-time constants).
template <int R, int r = 0>
__device__ __forceinline__ void c2r_combine(float2* v, const float2* x1, const float2* x2, float2 w0) {
  if constexpr (r < R) {
    constexpr float hc = (float)ct_cos(r, 2 * R), hs = (float)ct_sin(r, 2 * R);
    const float2 w = cmul(w0, make_float2(hc, -hs));   // hs = sin(pi r / R)
    const float2 e = make_float2(0.5f * (x1[r].x + x2[r].x), 0.5f * (x1[r].y - x2[r].y));
    const float2 d = make_float2(0.5f * (x1[r].x - x2[r].x), 0.5f * (x1[r].y + x2[r].y));
    const float2 o = cmul(d, make_float2(w.x, -w.y));
    v[r] = make_float2(e.x - o.y, e.y + o.x);
    c2r_combine<R, r + 1>(v, x1, x2, w0);
  }
}

template <int R>
__device__ __forceinline__ void apply_stage_twiddle(float2* v, const float2* t, int NS, int k) {
  if constexpr (R >= 2) {
    float2 w[R];
    w[1] = __ldg(t + k);
    if constexpr (R >= 4) w[2] = __ldg(t + NS + k);
    if constexpr (R >= 8) w[4] = __ldg(t + 2 * NS + k);
    if constexpr (R >= 16) w[8] = __ldg(t + 3 * NS + k);
    if constexpr (R >= 4) w[3] = cmul(w[1], w[2]);
    if constexpr (R >= 8) {
      w[5] = cmul(w[4], w[1]);
      w[6] = cmul(w[4], w[2]);
      w[7] = cmul(w[4], w[3]);
    }
    if constexpr (R >= 16) {
#pragma unroll
      for (int r = 1; r < 8; ++r) w[8 + r] = cmul(w[8], w[r]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r]);
  }
}

// One pass S of the tile: gather, twiddle, R-point DFT, scatter (with the
// barriers that separate it from its neighbours).
//   PRE  0: first pass reads global memory; 1: two-CTA radix-2 split;
//        2: first pass reads a TMA-staged box; 4: the first pass's inputs are
//        already in registers (left there by a POST == 2 transform), no conj_in;
//        5: first pass builds Z[n] = E[n] + i O[n] of a complex-to-real
//        transform from X[n] and X[L - n] of rows of L + 1 values (C2R);
//        6: first pass reads an unpadded copy of the C rows that a bulk copy
//        left at the start of the exchange buffer `sm` (tile_fft_pfs_kernel);
//        7: as 5 for the column pass of a four-step complex-to-real plan:
//        element m = n1 N2 + n2 of the length-M input (n1 down the column,
//        n2 = col0 + c, M = L * ncols) is built from X[m] and X[M - m].
//   POST 0: last pass stores to global memory; 2: last pass multiplies output
//        k by filt[k] and conjugates it, in registers; 3: last pass leaves
//        output k in shared memory at sidx(k) (natural order) and splits the
//        real-to-complex pairs of the same row; 6: last pass leaves output k
//        of column c in shared memory at k * (C + 1) + c (transposed: lanes of
//        consecutive k write, and lanes of consecutive c read, without bank
//        conflicts) and stops there (the caller combines rows; `sm` must hold
//        L * (C + 1) entries); 7: last pass of a row pass (j-fast in, c-fast
//        out) leaves its scaled outputs as a dense tile sm[k * C + c] for a
//        tensor-TMA store by the caller; 4: as 0, and
//        once every thread has read its inputs from `sm`, one thread starts
//        the bulk copy of the next tile's rows (source `gin`, none if NULL)
//        into `sm`, completing on the mbarrier stored just past the tile.
//   REV: remainder-last radix schedule (tables from a.tw_rev).  A POST == 2
//        transform (radix-16 last pass: thread j holds k = j + q*L/16) feeds a
//        PRE == 4, REV transform (radix-16 first pass: thread j reads n = j +
//        r*L/16) without an exchange; lengths below 16 are one pass either way.
template <int LG, int C, bool IN_CF, bool OUT_CF, int S, bool OFFS = false, int PRE = 0, int IDX = 0,
          int POST = 0, bool REV = false, int LGM = 4>
__device__ __forceinline__ void tile_pass(float2 (&v)[TileCfg<LG, C, IN_CF, OUT_CF, 0, LGM>::P], float2* sm,
                                          const TileArgs& a, const float2* gin, float2* gout,
                                          long long col0, long long bidx, const float2* epi_tab) {
  using Cfg = TileCfg<LG, C, IN_CF, OUT_CF, IDX, LGM>;
  constexpr int L = Cfg::L, P = Cfg::P, T = Cfg::T, NST = Cfg::NST, LP = Cfg::LP;
  constexpr int LGR = radix_lgr(LG, S, REV, LGM), R = 1 << LGR;
  constexpr int LGNS = radix_lgns(LG, S, REV, LGM), NS = 1 << LGNS;
  constexpr bool FIRST = (S == 0), LAST = (S == NST - 1);
  constexpr bool CF = (FIRST && IN_CF) || (LAST && OUT_CF);
  constexpr int NB = P / R;   // butterflies per thread in this pass
  constexpr int LR = L / R;
  const int tid = threadIdx.x;

  int cc[NB], jj[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if constexpr (CF) {
      cc[i] = tid % C;
      jj[i] = (tid / C) * NB + i;
    } else {
      const int b = tid + i * T;
      cc[i] = b / LR;
      jj[i] = b % LR;
    }
  }

  // ---- gather the R inputs of each butterfly ----
  if constexpr (FIRST && PRE == 4) {
    static_assert(NB == 1 && (R == 16 || R == L), "register hand-over needs a one-butterfly first pass");
  } else if constexpr (FIRST) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const bool ok = (col0 + cc[i]) < a.ncols;
      // a j-fast input is always a contiguous row (in_sn == 1 for every plan
      // that uses it), so its element offsets are compile-time constants
      const long long isn = IN_CF ? a.in_sn : 1;
      const float2* p = (OFFS ? gin + (ok ? a.col_off[cc[i]] : 0) : gin + cc[i] * a.in_sc) + (long long)jj[i] * isn;
      const long long step = (long long)LR * isn;
      if constexpr (PRE == 6) {
        const float2* sp = sm + cc[i] * L + jj[i];
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = ok ? sp[r * LR] : make_float2(0.f, 0.f);
      } else if constexpr (PRE == 5) {
        // complex-to-real: E = (X[n] + conj X[L-n]) / 2,
        // O = (X[n] - conj X[L-n]) W_N^{-n} / 2, Z = E + i O; Im X[0] and
        // Im X[L] do not enter.  Rows hold L + 1 values (in_sc).  All loads
        // are issued before any arithmetic.
        float2 x1[R], x2[R], w[R];
        const float2* pm = p + (long long)(L - 2 * jj[i]);   // X[L - n] = pm[-r * step]
#pragma unroll
        for (int r = 0; r < R; ++r) {
          x1[r] = ok ? __ldg(p + r * step) : make_float2(0.f, 0.f);
          x2[r] = ok ? __ldg(pm - r * step) : make_float2(0.f, 0.f);
          w[r] = __ldg(a.r_w + jj[i] + r * LR);
        }
        if (jj[i] == 0) {   // n == 0 only for r == 0
          const float em = (float)(1 + a.r_end2);   // 2 for the adjoint of real-to-complex
          x1[0] = make_float2(x1[0].x * em, 0.f);
          x2[0] = make_float2(x2[0].x * em, 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float2 e = make_float2(0.5f * (x1[r].x + x2[r].x), 0.5f * (x1[r].y - x2[r].y));
          const float2 d = make_float2(0.5f * (x1[r].x - x2[r].x), 0.5f * (x1[r].y + x2[r].y));
          const float2 o = cmul(d, make_float2(w[r].x, -w[r].y));
          v[i * R + r] = make_float2(e.x - o.y, e.y + o.x);
        }
      } else if constexpr (PRE == 7) {
        // the same split down a column: X[m] and X[M - m] lie in mirror
        // columns (N2 - n2), read straight from the rows of M + 1 values;
        // W_N^m from the two-level table
        // (the step between the R inputs is M / R, so W_N^{m0 + r M/R} =
        // W_N^{m0} W_{2R}^r: one table product per butterfly, then constants)
        static_assert(IN_CF && !OFFS, "complex-to-real column pass");
        const long long M = (long long)L * a.ncols;
        const long long m0 = col0 + cc[i] + (long long)jj[i] * isn;   // m of r = 0
        const float2* pm = p + (M - 2 * m0);                            // X[M - m] = pm[-r * step]
        const unsigned lo_mask = (1u << a.r_s) - 1u;
        const float2 w0 = cmul(__ldg(a.r_w + ((unsigned)m0 & lo_mask)), __ldg(a.r_hi + ((unsigned)m0 >> a.r_s)));
        float2 x1[R], x2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          x1[r] = ok ? __ldg(p + r * step) : make_float2(0.f, 0.f);
          x2[r] = ok ? __ldg(pm - r * step) : make_float2(0.f, 0.f);
        }
        if (m0 == 0) {   // m == 0 only for r == 0
          const float em = (float)(1 + a.r_end2);
          x1[0] = make_float2(x1[0].x * em, 0.f);
          x2[0] = make_float2(x2[0].x * em, 0.f);
        }
        c2r_combine<R>(v + i * R, x1, x2, w0);
      } else if constexpr (PRE == 2) {
        // column tile already staged in shared memory by a tensor TMA copy,
        // laid out [n][c] (gin points at it)
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = gin[(jj[i] + r * LR) * C + cc[i]];
      } else if constexpr (PRE == 1) {
        // (x[n] +- x[n + half]) of the two-CTA radix-2 split; the twiddle
        // W^{n k1} is applied after the conjugation below
        const float2* p2 = p + a.pre_half;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float2 x0 = __ldcs(p + r * step), x1 = __ldcs(p2 + r * step);
          v[i * R + r] = bidx ? csub(x0, x1) : cadd(x0, x1);
        }
      } else if (a.stream_in) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = ok ? __ldcs(p + r * step) : make_float2(0.f, 0.f);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = ok ? __ldcg(p + r * step) : make_float2(0.f, 0.f);
      }
    }
    if (a.conj_in) {
#pragma unroll
      for (int p = 0; p < P; ++p) v[p].y = -v[p].y;
    }
    if constexpr (PRE == 1) {
      if (bidx) {
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
          for (int r = 0; r < R; ++r) v[i * R + r] = cmul(v[i * R + r], __ldg(a.pre_tw + jj[i] + r * LR));
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      if constexpr (IDX == 0) {
        const float2* rp = sm + cc[i] * LP + pidx(jj[i]);
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = rp[pidx_c(r * LR)];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = sm[cc[i] * LP + sidx<IDX>(jj[i] + r * LR)];
      }
    }
  }
  if constexpr (LAST && POST == 4 && !FIRST) {
    // every thread holds its last-pass inputs: the buffer now receives the
    // next tile's rows while this pass computes and stores
    __syncthreads();
    if (threadIdx.x == 0 && gin) {
      fence_proxy_async();   // order the generic-proxy reads above before the async-proxy write
      tma_load_1d(sm, gin, (uint32_t)(C * L * 8), reinterpret_cast<uint64_t*>(sm + Cfg::SM_TILE));
    }
  }

  // ---- twiddles W_{Ns*R}^{r*(j mod Ns)} ----
  if constexpr (NS > 1) {
    const float2* t = (REV ? a.tw_rev : a.tw) + stage_tw_off(LG, S, REV, LGM);
#pragma unroll
    for (int i = 0; i < NB; ++i) apply_stage_twiddle<R>(v + i * R, t, NS, jj[i] & (NS - 1));
  }

  // ---- R-point DFT in registers ----
#pragma unroll
  for (int i = 0; i < NB; ++i) dft_fwd<R>(v + i * R);

  // ---- scatter outputs ----
  if constexpr (LAST && POST == 7) {
    static_assert(NB == 1 && IDX == 0 && OUT_CF && !IN_CF && !REV && !OFFS, "row pass: outputs to a dense tile");
    // the scaled outputs of the C rows as a dense [k][c] tile at sm (C * L
    // entries, inside the exchange tile): adjacent lanes (adjacent c, or the
    // next k) write adjacent words; the caller stores the tile with tensor TMA
    __syncthreads();   // all reads of this pass are done
    if (a.scale_out) {
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = make_float2(v[q].x * a.sx, v[q].y * a.sy);
    }
    float2* wp = sm + jj[0] * C + cc[0];
#pragma unroll
    for (int q = 0; q < R; ++q) wp[q * NS * C] = v[q];
    __syncthreads();
  } else if constexpr (LAST && POST == 6) {
    static_assert(NB == 1 && IDX == 0 && !OUT_CF && !REV, "rows left in shared memory: contiguous rows");
    // (the caller provides at least L * (C + 1) entries at sm: for C >= 16
    // the exchange tile itself, otherwise a larger allocation)
    __syncthreads();   // all reads of this pass are done
    float2* wp = sm + jj[0] * (C + 1) + cc[0];
#pragma unroll
    for (int q = 0; q < R; ++q) wp[q * NS * (C + 1)] = v[q];
    __syncthreads();
  } else if constexpr (LAST && POST == 3) {
    // real-to-complex split: thread j holds Z[k], k = j + q*NS; the partner
    // Z[L - k] of every one of them lives in thread NS - j (q' = R - 1 - q),
    // or in thread 0 itself for j = 0, so one exchange gives each thread all
    // it needs:  X[k] = E + W_N^k O,  E = (Z[k] + conj Z[L-k]) / 2,
    //            O = (Z[k] - conj Z[L-k]) / (2i),  plus X[L] from Z[0].
    static_assert(NB == 1 && IDX == 0 && !OUT_CF && !REV, "real split: contiguous rows");
    const int c = cc[0], j = jj[0];
    __syncthreads();   // all reads of this pass are done
    float2* wp = sm + c * LP + pidx(j);
#pragma unroll
    for (int q = 0; q < R; ++q) wp[pidx_c(q * NS)] = v[q];
    __syncthreads();
    if ((col0 + c) < a.ncols) {
      const float2* zr = sm + c * LP;
      float2* orow = gout + c * a.out_sc;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int k = j + q * NS;
        const float2 zk = v[q];
        const float2 zm = zr[pidx((L - k) & (L - 1))];
        const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        float2 x = cadd(e, cmul(__ldg(a.r_w + k), o));
        if (a.scale_out) {
          const float sc = k == 0 ? a.sy : a.sx;
          x = make_float2(x.x * sc, x.y * sc);
        }
        if (a.stream_out)
          __stcs(orow + k, x);
        else
          __stcg(orow + k, x);
      }
      if (j == 0) {
        // X[L] = E[0] - O[0] (W_N^L = -1)
        const float2 z0 = v[0];
        const float2 x = make_float2((z0.x - z0.y) * (a.scale_out ? a.sy : 1.f), 0.f);
        if (a.stream_out)
          __stcs(orow + L, x);
        else
          __stcg(orow + L, x);
      }
    }
  } else if constexpr (LAST && POST == 2) {
    static_assert(NB == 1 && IDX == 0 && !OUT_CF && !REV, "fused filter pass: contiguous rows");
    // output k = j + q*NS stays in the thread as conj(filt[k] * X[k])
    const int j = jj[0];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const float2 z = cmul(v[q], filt_at(a, j + q * NS));
      v[q] = make_float2(z.x, -z.y);
    }
  } else if constexpr (LAST && REV) {
    static_assert(IDX == 0 && !OUT_CF && !OFFS && PRE != 1, "remainder-last schedule: contiguous rows");
    // NB butterflies per thread; butterfly i writes k = j_i + q*NS of column c_i
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int c = cc[i], j = jj[i];
      if (a.scale_out) {
#pragma unroll
        for (int q = 0; q < R; ++q) v[i * R + q] = make_float2(v[i * R + q].x * a.sx, v[i * R + q].y * a.sy);
      }
      if ((col0 + c) < a.ncols) {
        float2* p = gout + c * a.out_sc + j;
        if (a.stream_out) {
#pragma unroll
          for (int q = 0; q < R; ++q) __stcs(p + q * NS, v[i * R + q]);
        } else {
#pragma unroll
          for (int q = 0; q < R; ++q) __stcg(p + q * NS, v[i * R + q]);
        }
      }
    }
  } else if constexpr (LAST) {
    static_assert(NB == 1, "last pass is a full-radix pass (or the whole length)");
    // After the last pass NS = L/R and j < NS: output index k = j + q*NS.
    const int c = cc[0], j = jj[0];
    const bool ok = (col0 + c) < a.ncols;
    if (Cfg::EPI && a.ft_lgN) {
      // four-step twiddle W_N^{n2*k}, n2 = col0 + c, k = j + q*NS
      //   = W_N^{n2*j} * W_N^{n2*NS*q}; the second factor is the per-column
      //   table epi_tab[q*C + c] built at kernel start (q-major: adjacent
      //   lanes of the c-fast mapping read adjacent entries, no bank conflict).
      const unsigned n2 = a.ft_by_batch ? (unsigned)bidx : (unsigned)(col0 + c);
      const unsigned m = n2 * (unsigned)j;
      const unsigned mask = (1u << a.ft_s) - 1u;
      const float2 base = cmul(__ldg(a.ft_lo + (m & mask)), __ldg(a.ft_hi + (m >> a.ft_s)));
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = cmul(v[q], cmul(base, epi_tab[q * C + c]));
    }
    if constexpr (!IN_CF && OUT_CF && !OFFS && PRE == 0) {
      if (a.filt) {
        // multi-pass range compression: the stored element's offset from
        // `out` modulo N is its frequency index
        const long long o = (long long)(gout - a.out) + c * a.out_sc + (long long)j * a.out_sn;
        const long long st = (long long)NS * a.out_sn;
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = cmul(v[q], filt_at(a, (o + q * st) & a.filt_mask));
      }
    }
    if (a.scale_out) {
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = make_float2(v[q].x * a.sx, v[q].y * a.sy);
    }
    if (ok) {
      // a j-fast output is contiguous (out_sn == 1), or every other element
      // for the two-CTA split (PRE == 1); c-fast outputs use the runtime stride
      const long long osn = OUT_CF ? a.out_sn : (PRE == 1 ? 2 : 1);
      float2* p = (OFFS ? gout + a.col_off[c] : gout + c * a.out_sc) + (long long)j * osn;
      const long long step = (long long)NS * osn;
      if (a.stream_out) {
#pragma unroll
        for (int q = 0; q < R; ++q) __stcs(p + q * step, v[q]);
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) __stcg(p + q * step, v[q]);
      }
    }
  } else {
    // all reads of this pass (or, for PRE == 4, of the previous transform's
    // last pass) are done
    if constexpr (!FIRST || PRE == 4 || PRE == 6) __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = jj[i];
      const int base = ((j >> LGNS) << (LGNS + LGR)) + (j & (NS - 1));
      if constexpr (IDX == 0) {
        float2* wp = sm + cc[i] * LP + pidx(base);
#pragma unroll
        for (int q = 0; q < R; ++q) wp[pidx_c(q * NS)] = v[i * R + q];
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) sm[cc[i] * LP + sidx<IDX>(base + q * NS)] = v[i * R + q];
      }
    }
    __syncthreads();
  }
}

template <int LG, int C, bool IN_CF, bool OUT_CF, int S, bool OFFS = false, int PRE = 0, int POST = 0,
          bool REV = false, int LGM = 4>
__device__ __forceinline__ void tile_stage(float2 (&v)[TileCfg<LG, C, IN_CF, OUT_CF, 0, LGM>::P], float2* sm,
                                           const TileArgs& a, const float2* gin, float2* gout,
                                           long long col0, long long bidx, const float2* epi_tab) {
  tile_pass<LG, C, IN_CF, OUT_CF, S, OFFS, PRE, 0, POST, REV, LGM>(v, sm, a, gin, gout, col0, bidx, epi_tab);
  if constexpr (S + 1 < TileCfg<LG, C, IN_CF, OUT_CF, 0, LGM>::NST)
    tile_stage<LG, C, IN_CF, OUT_CF, S + 1, OFFS, PRE, POST, REV, LGM>(v, sm, a, gin, gout, col0, bidx, epi_tab);
}

// One tile of a pass: tile index `tile` of the launch described by `a`, using
// `smem` (TileCfg::SMEM_BYTES).  Shared by the one-tile-per-CTA kernel below
// and the persistent uneven-batch kernel.
template <int LG, int C, bool IN_CF, bool OUT_CF, bool OFFS = false, int PRE = 0, int POST = 0, int LGM = 4>
__device__ __forceinline__ void tile_body(const TileArgs& a, long long tile, float2* smem) {
  using Cfg = TileCfg<LG, C, IN_CF, OUT_CF, 0, LGM>;
  float2* sm = smem;
  float2* epi_tab = smem + Cfg::SM_TILE;

  long long b = tile / a.tiles_per_batch;
  const long long g = tile - b * a.tiles_per_batch;
  long long b2 = 0;
  if (a.nb1) {
    b2 = b / a.nb1;
    b -= b2 * a.nb1;
  }
  const long long col0 = g * C;
  const float2* gin = a.in + b2 * a.in_b2stride + b * a.in_bstride + g * a.in_gstride;
  float2* gout = a.out + b2 * a.out_b2stride + b * a.out_bstride + g * a.out_gstride;

  if (Cfg::EPI && a.ft_lgN) {
    // per-column step factors W_N^{n2*NS_last*q}, q = 0..15
    constexpr int NS_LAST = 1 << radix_lgns(LG, Cfg::NST - 1, false, LGM);
    for (int e = threadIdx.x; e < C * 16; e += Cfg::T) {
      const int q = e / C, c = e - q * C;   // entry q*C + c
      const unsigned n2 = a.ft_by_batch ? (unsigned)b : (unsigned)(col0 + c);
      const unsigned m = n2 * (unsigned)NS_LAST * (unsigned)q;
      const unsigned mm = m & ((1u << a.ft_lgN) - 1u);
      const unsigned mask = (1u << a.ft_s) - 1u;
      epi_tab[e] = cmul(__ldg(a.ft_lo + (mm & mask)), __ldg(a.ft_hi + (mm >> a.ft_s)));
    }
    if constexpr (Cfg::NST == 1) __syncthreads();
  }

  float2 v[Cfg::P];
  tile_stage<LG, C, IN_CF, OUT_CF, 0, OFFS, PRE, POST, false, LGM>(v, sm, a, gin, gout, col0, b, epi_tab);
}

// Two CTAs per transform of length 2^(LG+1) (radix-2 decimation in
// frequency, Sec. 2.1's butterfly applied once across the halves):
//   X[2 k2 + k1] = sum_n W_{N/2}^{n k2} [(x[n] + (-1)^k1 x[n + N/2]) W_N^{n k1}]
// CTA (b, k1) computes the half-length transform of the bracket for transform
// b and writes every other output (out_sn = 2, offset k1).  Each CTA of a
// pair reads both halves of the input; the second read of every element is
// usually an L2 hit.  Halving the per-CTA size lets two CTAs share an SM.
template <int LG>
__global__ void __launch_bounds__(TileCfg<LG, 1, false, false>::T, (LG >= 13 ? 2 : 3))
    tile_fft_dif2_kernel(const TileArgs a) {
  extern __shared__ float2 smem[];
  const long long b = (long long)blockIdx.x >> 1;
  const int k1 = blockIdx.x & 1;
  float2 v[TileCfg<LG, 1, false, false>::P];
  tile_stage<LG, 1, false, false, 0, false, 1>(v, smem, a, a.in + b * a.in_bstride, a.out + b * a.out_bstride + k1, 0,
                                               k1, nullptr);
}

// LGM < 4: the same pass with radix-8 (LGM = 3) or radix-4 (LGM = 2) passes
// and as many points per thread (single-pass variants the autotuner may pick;
// stage table built for that schedule).
template <int LG, int C, bool IN_CF, bool OUT_CF, int LGM = 4>
__global__ void __launch_bounds__(TileCfg<LG, C, IN_CF, OUT_CF, 0, LGM>::T)
    tile_fft_kernel(const TileArgs a) {
  extern __shared__ float2 smem[];
  tile_body<LG, C, IN_CF, OUT_CF, false, 0, 0, LGM>(a, (long long)blockIdx.x, smem);
}

// Persistent single-pass variant for one transform per CTA (C == 1, contiguous
// rows): CTA b takes tiles b, b + grid, ...  Before transforming a tile, its
// threads ask L2 for the next one (prefetch.global.L2, one 128-byte line per
// thread per step), so that the next load phase hits L2 and the DRAM reads
// overlap this tile's passes instead of following them.
template <int LG>
__global__ void __launch_bounds__(TileCfg<LG, 1, false, false>::T)
    tile_fft_pf_kernel(const TileArgs a, long long ntiles) {
  extern __shared__ float2 smem[];
  using Cfg = TileCfg<LG, 1, false, false>;
  constexpr int BYTES = Cfg::L * 8;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long nt = t + gridDim.x;
    if (nt < ntiles) {
      const char* p = (const char*)(a.in + nt * a.in_gstride);
#pragma unroll
      for (int off = threadIdx.x * 128; off < BYTES; off += Cfg::T * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
    }
    tile_body<LG, 1, false, false>(a, t, smem);
    __syncthreads();   // the next tile's first exchange overwrites this one's
  }
}

// Persistent single pass (C = 1) whose exchange buffer doubles as the staging
// buffer of the next transform: when the last pass of transform t has read its
// inputs from shared memory, one thread starts a bulk copy (TMA, evict-first)
// of transform t + grid into the same buffer, which lands while the last pass
// computes and stores; transform t + grid's first pass then reads shared
// memory instead of waiting on global loads.  Transform t + grid is also
// prefetched into L2 when transform t starts, so that the copy reads L2.
// Shared memory: the exchange tile plus one mbarrier (8 bytes, 16 reserved).
// The wait on the barrier is bounded: on expiry the CTA records
// FFT_ERR_TIMEOUT in `status`, waits once more (bounded) for the copy in
// flight, and returns.
template <int LG>
constexpr int pfs_smem_bytes() { return TileCfg<LG, 1, false, false>::SMEM_BYTES + 16; }

template <int LG>
__global__ void __launch_bounds__(TileCfg<LG, 1, false, false>::T)
    tile_fft_pfs_kernel(const TileArgs a, long long ntiles, int* status) {
  extern __shared__ float2 smem[];
  using Cfg = TileCfg<LG, 1, false, false>;
  static_assert(Cfg::NST > 1 && Cfg::SM_TILE >= Cfg::L, "the staged copy must fit the exchange buffer");
  constexpr int BYTES = Cfg::L * 8;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Cfg::SM_TILE);
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && (long long)blockIdx.x < ntiles)
    tma_load_1d(smem, a.in + (long long)blockIdx.x * a.in_gstride, BYTES, mbar);
  uint32_t parity = 0;
  float2 v[Cfg::P];
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long nt = t + gridDim.x;
    const float2* next = nt < ntiles ? a.in + nt * a.in_gstride : nullptr;
    if (next) {
      const char* p = (const char*)next;
#pragma unroll
      for (int off = threadIdx.x * 128; off < BYTES; off += Cfg::T * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
    }
    if (!mbar_wait(mbar, parity)) {
      if (threadIdx.x == 0) atomicExch(status, FFT_ERR_TIMEOUT);
      mbar_wait(mbar, parity);   // second bounded wait for the copy in flight
      return;
    }
    parity ^= 1;
    // (no closing barrier: the next transform starts with the wait on its copy,
    // which the last pass issued after every thread had read the buffer)
    tile_stage<LG, 1, false, false, 0, false, 6, 4>(v, smem, a, next, a.out + t * a.out_gstride, t, 0, nullptr);
  }
}

// Resident CTAs per SM the fused kernel is compiled for: 64 registers per
// thread at every size (measured on GB300: more registers than the default
// heuristic picks speed up 2^13 and 2^14; 48 at 256 threads spills and
// does not help 2^12).
__host__ __device__ constexpr int rc_min_blocks(int threads) { return threads <= 256 ? 4 : (threads <= 512 ? 2 : 1); }

// Range compression of C contiguous rows per CTA (fast convolution, the
// FFT-based SAR step of Sec. 3 and Sec. 4): y = IDFT(H * DFT(x)) with one
// read and one write of every value.  The forward transform (Eq. 1) ends with
// conj(H X) in registers; a second forward transform of it (remainder-last
// schedule, which starts from those registers), conjugated and scaled by 1/L
// on the store (a.sx = 1/L, a.sy = -1/L), is Eq. 2 of H X.
// Shared memory: C * LP entries.
// One CTA per SM at 2^14: the kernel is persistent there and prefetches the
// next row into L2 (as tile_fft_pf_kernel); shorter rows take one tile per CTA.
__host__ __device__ constexpr bool rc_persistent(int lg) { return lg == 14; }

template <int LG, int C>
__global__ void __launch_bounds__(TileCfg<LG, C, false, false>::T, rc_min_blocks(TileCfg<LG, C, false, false>::T))
    tile_rc_kernel(const TileArgs a, long long ntiles) {
  extern __shared__ float2 smem[];
  using Cfg = TileCfg<LG, C, false, false>;
  float2 v[Cfg::P];
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if constexpr (rc_persistent(LG)) {
      const long long nt = t + gridDim.x;
      if (nt < ntiles) {
        const char* p = (const char*)(a.in + nt * a.in_gstride);
#pragma unroll
        for (int off = threadIdx.x * 128; off < C * Cfg::L * 8; off += Cfg::T * 128)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
      }
    }
    {
      const long long b = t / a.tiles_per_batch;
      const long long g = t - b * a.tiles_per_batch;
      const float2* gin = a.in + b * a.in_bstride + g * a.in_gstride;
      tile_stage<LG, C, false, false, 0, false, 0, 2>(v, smem, a, gin, nullptr, g * C, b, nullptr);
    }
    {
      // The tile index is passed through an opaque move, so that the output
      // address is computed here instead of being held in registers through
      // the first transform (which spills at 2^14, 64 registers per thread).
      long long tt;
      asm volatile("mov.b64 %0, %1;" : "=l"(tt) : "l"(t));
      const long long b = tt / a.tiles_per_batch;
      const long long g = tt - b * a.tiles_per_batch;
      float2* gout = a.out + b * a.out_bstride + g * a.out_gstride;
      tile_stage<LG, C, false, false, 0, false, 4, 0, true>(v, smem, a, nullptr, gout, g * C, b, nullptr);
    }
    if constexpr (!rc_persistent(LG)) break;
    __syncthreads();   // the next tile's first exchange overwrites this one's
  }
}

// Real-to-complex transform of rows of N = 2L reals (Sec. 2.1's split of a
// sequence into even and odd samples): the row read as L complex values
// z[m] = x[2m] + i x[2m+1] is transformed on chip (Z = Eq. 1 of length L) and
// the last pass turns Z into X[0..L] (POST == 3), written to rows of L + 1
// complex values (out_sc).  One read and one write of every value.
template <int LG, int C>
__global__ void __launch_bounds__(TileCfg<LG, C, false, false>::T) tile_r2c_kernel(const TileArgs a) {
  extern __shared__ float2 smem[];
  using Cfg = TileCfg<LG, C, false, false>;
  const long long tile = blockIdx.x;
  const long long b = tile / a.tiles_per_batch;
  const long long g = tile - b * a.tiles_per_batch;
  float2 v[Cfg::P];
  tile_stage<LG, C, false, false, 0, false, 0, 3>(v, smem, a, a.in + b * a.in_bstride + g * a.in_gstride,
                                                  a.out + b * a.out_bstride + g * a.out_gstride, g * C, b, nullptr);
}

// Complex-to-real transform (the inverse of tile_r2c_kernel): rows of L + 1
// values X[0..L] (in_sc) become rows of N = 2L reals.  The first pass builds
// Z[n] = E[n] + i O[n] from X[n] and X[L - n] (PRE == 5) and the tile runs
// the inverse length-L transform by conjugation (conj_in = 1, a.sx = 1/L,
// a.sy = -1/L); z[m] = x[2m] + i x[2m+1] is stored as L complex values.
template <int LG, int C>
__global__ void __launch_bounds__(TileCfg<LG, C, false, false>::T, rc_min_blocks(TileCfg<LG, C, false, false>::T))
    tile_c2r_kernel(const TileArgs a) {
  extern __shared__ float2 smem[];
  using Cfg = TileCfg<LG, C, false, false>;
  const long long tile = blockIdx.x;
  const long long b = tile / a.tiles_per_batch;
  const long long g = tile - b * a.tiles_per_batch;
  float2 v[Cfg::P];
  tile_stage<LG, C, false, false, 0, false, 5, 0>(v, smem, a, a.in + b * a.in_bstride + g * a.in_gstride,
                                                  a.out + b * a.out_bstride + g * a.out_gstride, g * C, b, nullptr);
}

}  // namespace gbfft
