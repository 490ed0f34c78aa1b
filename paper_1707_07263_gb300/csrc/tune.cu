// tune.cu -- the autotuner: time candidate plan configurations on the caller's
// buffers and keep the fastest.  The paper fixes its partition thresholds by
// hand for the C2070 (Sec. 2.3.2, Sec. 3); here the split, the number of
// passes, the columns per CTA, the staging kernel and, for one on-chip pass,
// the largest radix (with it the points per thread and the threads per CTA)
// are measured per shape on the GPU at hand.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "gbfft_internal.h"
#include "tile_registry.h"

namespace gbfft {
int set_err(int code);
}

using namespace gbfft;

static void add_cols(std::vector<fft_plan_config>& out, fft_plan_config base, int lg_a, int lg_b, int cols_a_max,
                     int cols_b_max) {
  // columns per CTA: powers of two 2..64 keeping C * L <= 2^14 (compiled range)
  for (int ca = 2; ca <= 64; ca *= 2) {
    if ((ca << lg_a) > (1 << 14) || ca > cols_a_max) continue;
    for (int cb = 2; cb <= 64; cb *= 2) {
      if ((cb << lg_b) > (1 << 14) || cb > cols_b_max) continue;
      fft_plan_config c = base;
      c.c1 = ca;
      c.c2 = cb;
      out.push_back(c);
    }
  }
}

static std::vector<fft_plan_config> candidates(int lgN) {
  std::vector<fft_plan_config> v;
  fft_plan_config z;
  memset(&z, 0, sizeof(z));
  z.tma = -1;
  z.fused = 0;
  {
    fft_plan_config c = z;
    c.fused = 1;
    v.push_back(c);  // rejected by plan creation where no fused kernel exists
  }
  if (lgN <= 14) {
    fft_plan_config c = z;
    c.npass = 1;
    c.tma = 0;
    v.push_back(c);
    c.tma = 1;
    v.push_back(c);
    if (lgN >= 12) {
      c.tma = 2;  // persistent register path with an L2 prefetch of the next transform
      v.push_back(c);
      c.tma = 3;  // ... and a bulk copy of it into the exchange buffer
      v.push_back(c);
    }
    c.tma = 0;
    c.halves = 2;  // rejected where no split kernel exists
    v.push_back(c);
    c.halves = 0;
    // largest radix 8 or 4 (as many points per thread, so 2x / 4x the
    // threads per CTA); rejected where not compiled
    for (int r = 4; r <= 8; r *= 2) {
      c.radix = r;
      v.push_back(c);
    }
  }
  if (lgN >= 10) {
    for (int lg1 = lgN / 2 - 2; lg1 <= (lgN + 1) / 2 + 2; ++lg1) {
      const int lg2 = lgN - lg1;
      if (lg1 < 5 || lg2 < 5 || lg1 > 14 || lg2 > 14) continue;
      fft_plan_config c = z;
      c.npass = 2;
      c.lg1 = lg1;
      add_cols(v, c, lg1, lg2, 1 << lg2, 1 << lg1);
      c.tma = 1;  // default columns, tensor-TMA staged column pass
      v.push_back(c);
    }
  }
  if (lgN >= 15) {
    const int d1 = (lgN + 2) / 3;
    for (int l1 = d1 - 1; l1 <= d1 + 1; ++l1)
      for (int l2 = (lgN - l1) / 2 - 1; l2 <= (lgN - l1 + 1) / 2 + 1; ++l2) {
        const int l3 = lgN - l1 - l2;
        if (l1 < 5 || l2 < 5 || l3 < 5 || l1 > 14 || l2 > 14 || l3 > 14) continue;
        fft_plan_config c = z;
        c.npass = 3;
        c.lg1 = l1;
        c.lg2 = l2;
        v.push_back(c);  // default columns
        c.tma = 1;       // ... with tensor-TMA staged column passes
        v.push_back(c);
        c.tma = -1;
        for (int ca = 16; ca <= 32; ca *= 2)
          for (int cb = 16; cb <= 32; cb *= 2)
            for (int cc = 8; cc <= 32; cc *= 2) {
              if ((ca << l1) > (1 << 14) || (cb << l2) > (1 << 14) || (cc << l3) > (1 << 14)) continue;
              fft_plan_config d = c;
              d.c1 = ca;
              d.c2 = cb;
              d.c3 = cc;
              v.push_back(d);
            }
      }
  }
  return v;
}

extern "C" GBFFT_API int fft_autotune(int64_t n, int64_t batch, int prec, void* in, void* out, void* ws,
                                      size_t ws_bytes, void* stream, int iters, fft_plan_config* best,
                                      float* best_us) {
  if (n < 2 || (n & (n - 1)) || batch < 1 || !in || !out || !best || !best_us || iters < 1)
    return set_err(FFT_ERR_INVALID_ARG);
  int lgN = 0;
  while ((1LL << lgN) < n) ++lgN;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<fft_plan_config> cands;
  if (prec == FFT_PREC_FP32) {
    cands = candidates(lgN);
  }
  fft_plan_config dflt;
  memset(&dflt, 0, sizeof(dflt));
  dflt.tma = -1;
  dflt.fused = -1;
  cands.insert(cands.begin(), dflt);  // the planner's default is always a candidate
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return set_err(FFT_ERR_CUDA);
  float best_t = 1e30f;
  bool found = false;
  for (const fft_plan_config& c : cands) {
    fft_plan* p = fft_plan_create_config(n, batch, FFT_FORWARD, prec, &c);
    if (!p) continue;  // no compiled kernel for this candidate
    const size_t need = fft_plan_workspace_bytes(p);
    if (need && (!ws || ws_bytes < need)) {
      fft_destroy(p);
      continue;
    }
    if (need) fft_plan_set_workspace(p, ws);
    bool ok = true;
    for (int w = 0; w < 3 && ok; ++w) ok = fft_exec(p, in, out, stream) == FFT_OK;
    cudaEventRecord(e0, s);
    for (int i = 0; i < iters && ok; ++i) ok = fft_exec(p, in, out, stream) == FFT_OK;
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ok = false;
    if (ok) {
      const float t = ms * 1000.f / iters;
      if (t < best_t) {
        best_t = t;
        fft_plan_get_config(p, best);
        found = true;
      }
    }
    fft_destroy(p);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (!found) return set_err(FFT_ERR_UNSUPPORTED);
  *best_us = best_t;
  return FFT_OK;
}

// Uneven batches: the queue gap, the resident CTAs per SM and the split of every
// four-step length present (fft_many_config).  The paper's thresholds for
// splitting a transform are fixed by hand (Sec. 2.3.2, Sec. 3); here they are
// timed on the batch at hand, one persistent launch per candidate.
extern "C" GBFFT_API int fft_autotune_many(const int64_t* lengths, int64_t count, int prec, void* in, void* out,
                                           void* ws, size_t ws_bytes, void* stream, int iters, fft_many_config* best,
                                           float* best_us) {
  if (!lengths || count < 1 || !in || !out || !best || !best_us || iters < 1) return set_err(FFT_ERR_INVALID_ARG);
  if (prec != FFT_PREC_FP32) return set_err(FFT_ERR_UNSUPPORTED);
  bool present[4] = {false, false, false, false};
  for (int64_t i = 0; i < count; ++i)
    for (int L = 13; L <= 16; ++L)
      if (lengths[i] == (1LL << L)) present[L - 13] = true;
  // splits: every valid lg1 for the four-step lengths present, the default otherwise
  std::vector<std::vector<int>> opts(4);
  for (int i = 0; i < 4; ++i) {
    const int L = 13 + i;
    if (present[i]) {
      for (int lg1 = 7; lg1 <= 8; ++lg1)
        if (L - lg1 >= 6 && L - lg1 <= 8) opts[i].push_back(lg1);
    } else {
      opts[i].push_back(0);
    }
  }
  std::vector<fft_many_config> cands;
  const int gaps[] = {1, 2, 3, 4, 6, 8};
  for (int g : gaps)
    for (int ctas = 2; ctas <= 4; ++ctas)
      for (int a : opts[0])
        for (int b : opts[1])
          for (int c : opts[2])
            for (int d : opts[3]) {
              fft_many_config cf;
              memset(&cf, 0, sizeof(cf));
              cf.gap = g;
              cf.ctas_per_sm = ctas;
              cf.lg1[0] = a;
              cf.lg1[1] = b;
              cf.lg1[2] = c;
              cf.lg1[3] = d;
              cands.push_back(cf);
            }
  fft_many_config dflt;
  memset(&dflt, 0, sizeof(dflt));
  cands.insert(cands.begin(), dflt);   // the planner's default is always a candidate
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return set_err(FFT_ERR_CUDA);
  float best_t = 1e30f;
  bool found = false;
  for (const fft_many_config& c : cands) {
    fft_plan* p = fft_plan_create_many_config(lengths, count, FFT_FORWARD, prec, &c);
    if (!p) continue;
    const size_t need = fft_plan_workspace_bytes(p);
    if (need && (!ws || ws_bytes < need)) {
      fft_destroy(p);
      continue;
    }
    if (need) fft_plan_set_workspace(p, ws);
    bool ok = true;
    for (int w = 0; w < 3 && ok; ++w) ok = fft_exec(p, in, out, stream) == FFT_OK;
    cudaEventRecord(e0, s);
    for (int i = 0; i < iters && ok; ++i) ok = fft_exec(p, in, out, stream) == FFT_OK;
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ok = false;
    if (ok && fft_status(p, stream) != FFT_OK) ok = false;   // a bounded wait ran out: not a valid candidate
    if (ok) {
      const float t = ms * 1000.f / iters;
      if (t < best_t) {
        best_t = t;
        fft_plan_get_many_config(p, best);
        found = true;
      }
    }
    fft_destroy(p);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (!found) return set_err(FFT_ERR_UNSUPPORTED);
  *best_us = best_t;
  return FFT_OK;
}
