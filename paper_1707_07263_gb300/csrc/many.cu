// many.cu -- transforms of uneven power-of-two lengths (2^1..2^16), packed back
// to back, in ONE persistent launch.
//
// The plan turns the batch into a queue of tile work items, each sized for a
// 256-thread CTA (at most 4096 points):
//   kind 0  batch tile: up to C = 4096/L transforms of the same length L <= 2^12,
//           each found through a per-column offset (the transforms need not
//           be adjacent);
//   kind 1  four-step column tile (C columns of length N1, with the W_N^{n2*k1}
//           twiddle) of a transform with 2^13 <= N <= 2^16;
//   kind 2  four-step row tile of such a transform, written transposed.
// Queue order: the kind-1 tiles of the four-step transforms (largest first),
// each transform's kind-2 tiles following its kind-1 tiles once about two
// grids' worth of further items have been queued, then the batch tiles
// (largest first).  The distance lets the column tiles finish before their row
// tiles are dequeued, and keeps the intermediate of the transforms in flight
// (~two grids of 4096-point tiles, ~30 MB) in L2 between the two passes.
// CTAs pop items with one atomicAdd on a queue head, claiming the next item
// while working on the current one.  A kind-2 tile waits until all kind-1
// tiles of its transform have been written (a per-transform completion
// counter); since those were dequeued earlier by CTAs that never wait, the
// wait always ends -- it is still bounded (clock64 budget) and a timeout sets
// FFT_ERR_TIMEOUT in the plan's status word instead of hanging.  The queue head and counters are
// cleared by a memset issued with every exec, so exec can be captured into a
// CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "gbfft_internal.h"
#include "tile_fft.cuh"

namespace gbfft {

struct ManyItem {
  int kind;   // 0 batch tile, 1 four-step column tile, 2 four-step row tile
  int lg;     // tile transform length (log2)
  int ncols;  // valid columns of the tile
  int tr;     // kind 0: first slot in the offset table; kinds 1/2: transform index
  int g;      // kinds 1/2: tile index within the pass
  int need;   // kind 2: column tiles of this transform to wait for
};

struct ManyTransform {
  long long off;     // element offset of the transform in the packed data
  long long ws_off;  // element offset of its workspace
  int lgN, lg1, lg2, c1, c2;
  int tab;           // index of its two-level W_N table
};

struct ManyArgs {
  const float2* in;
  float2* out;
  float2* ws;
  const ManyItem* items;
  const ManyTransform* trs;
  const long long* offs;
  const float2* stage_tw;      // stage tables, lengths 2^1..2^12 back to back
  const int* stage_tw_off;     // [13] offset of the table for length 2^lg
  const float2* ft_tab;        // two-level tables per four-step length
  const int* ft_off;           // [17] offset of (lo, hi) for lgN; lo then hi
  int* head;
  int* done;
  int* status;
  int nitems;
  int conj;
  int inv;
  long long wait_budget;
};

struct ManyPlan {
  fft_many_config cfg{};   // resolved configuration
  void* d_mem = nullptr;   // items, transforms, offsets, tables, counters
  size_t counters_bytes = 0;
  int* d_counters = nullptr;
  ManyArgs args{};
  int nitems = 0;
  int grid = 0;
  long long total = 0;
};

constexpr int kManyThreads = 256;

// The four-step split of 2^13..2^16 inside the persistent kernel: column
// tiles of length 2^lg1 (32 or 16 columns; lg1 = 7, 8) and row tiles of length
// 2^(lgN - lg1) (lengths 2^6..2^8).  Default lg1: 7, 7, 8, 8.  (A 64-column
// tile of 2^6 would raise the kernel's shared memory from 41.5 to 49.7 KB per
// CTA, taking a third of the L1 that caches the twiddle tables at four CTAs
// per SM: measured 14 % slower on the 4096-transform batch.)
constexpr int many_default_lg1(int lgN) { return lgN <= 14 ? 7 : 8; }
constexpr bool many_split_ok(int lgN, int lg1) { return lg1 >= 7 && lg1 <= 8 && lgN - lg1 >= 6 && lgN - lg1 <= 8; }
constexpr int kManyDefaultGap = 4;   // half resident grids between column and row tiles
constexpr int kManyMaxGap = 16;

template <int LG, int C, bool ICF, bool OCF>
constexpr int many_smem() { return TileCfg<LG, C, ICF, OCF>::SMEM_BYTES; }

template <int LG>
constexpr int many_batch_smem() {
  if constexpr (LG == 0) {
    return 0;
  } else {
    return cmax(TileCfg<LG, (LG >= 4) ? (4096 >> LG) : 256, false, false>::SMEM_BYTES, many_batch_smem<LG - 1>());
  }
}

// dynamic shared memory: the largest tile any item kind needs
constexpr int kManySmem = cmax(many_batch_smem<12>(),
                               cmax(cmax(many_smem<7, 32, true, true>(), many_smem<8, 16, true, true>()),
                                    cmax(cmax(many_smem<6, 64, false, true>(), many_smem<7, 32, false, true>()),
                                         many_smem<8, 16, false, true>())));

__device__ __forceinline__ bool many_wait(const int* flag, int target, long long budget) {
  const long long t0 = clock64();
  while (true) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v >= target) return true;
    if (clock64() - t0 > budget) return false;
    __nanosleep(64);
  }
}

template <int LG>
__device__ __forceinline__ void many_batch_tile(const ManyArgs& m, const ManyItem& it, TileArgs& a, float2* smem,
                                                long long* s_off) {
  constexpr int C = (LG >= 4) ? (4096 >> LG) : 256;
  for (int c = threadIdx.x; c < C; c += kManyThreads) s_off[c] = c < it.ncols ? m.offs[it.tr + c] : 0;
  __syncthreads();
  a.in = m.in;
  a.out = m.out;
  a.tw = m.stage_tw + m.stage_tw_off[LG];
  a.tiles_per_batch = 1LL << 40;
  a.in_sn = a.out_sn = 1;
  a.ncols = it.ncols;
  a.col_off = s_off;
  const float sc = m.inv ? 1.0f / (float)(1 << LG) : 1.0f;
  a.scale_out = (m.conj || m.inv) ? 1 : 0;
  a.sx = sc;
  a.sy = m.conj ? -sc : sc;
  tile_body<LG, C, false, false, true>(a, 0, smem);
}

template <int LG1>
__device__ __forceinline__ void many_col_tile(const ManyArgs& m, const ManyItem& it, const ManyTransform& t,
                                              TileArgs& a, float2* smem) {
  constexpr int C = 4096 >> LG1;
  const long long N2 = 1LL << t.lg2;
  a.in = m.in + t.off;
  a.out = m.ws + t.ws_off;
  a.tw = m.stage_tw + m.stage_tw_off[LG1];
  a.tiles_per_batch = 1LL << 40;
  a.in_gstride = a.out_gstride = C;
  a.in_sc = a.out_sc = 1;
  a.in_sn = a.out_sn = N2;
  a.ncols = N2;
  a.ft_lo = m.ft_tab + m.ft_off[t.lgN];
  a.ft_hi = a.ft_lo + (1 << ((t.lgN + 1) / 2));
  a.ft_lgN = t.lgN;
  a.ft_s = (t.lgN + 1) / 2;
  a.stream_out = 0;
  tile_body<LG1, C, true, true>(a, it.g, smem);
}

template <int LG2>
__device__ __forceinline__ void many_row_tile(const ManyArgs& m, const ManyItem& it, const ManyTransform& t,
                                              TileArgs& a, float2* smem) {
  constexpr int C = 4096 >> LG2;
  const long long N1 = 1LL << t.lg1, N2 = 1LL << LG2;
  a.in = m.ws + t.ws_off;
  a.out = m.out + t.off;
  a.tw = m.stage_tw + m.stage_tw_off[LG2];
  a.tiles_per_batch = 1LL << 40;
  a.in_gstride = C * N2;
  a.in_sc = N2;
  a.in_sn = 1;
  a.out_gstride = C;
  a.out_sc = 1;
  a.out_sn = N1;
  a.ncols = N1;
  a.stream_in = 0;
  const float sc = m.inv ? 1.0f / (float)(1LL << t.lgN) : 1.0f;
  a.scale_out = (m.conj || m.inv) ? 1 : 0;
  a.sx = sc;
  a.sy = m.conj ? -sc : sc;
  tile_body<LG2, C, false, true>(a, it.g, smem);
  // The tile's C rows of the intermediate (C * N2 = 4096 points, 32 KB,
  // contiguous) have been read by every thread: tile_body's first exchange
  // barrier follows all its loads.  Nothing reads them again in this
  // execution, so drop the lines from L2 instead of letting them be written
  // back to DRAM later (measured before: 838 MB written for 466 MB of output).
  static_assert(C * (1 << LG2) * 8 == kManyThreads * 128, "one 128-byte line per thread");
  const char* rows = (const char*)(m.ws + t.ws_off + (long long)it.g * C * N2);
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(rows + threadIdx.x * 128) : "memory");
}

__global__ void __launch_bounds__(kManyThreads, 4) many_kernel(const ManyArgs m) {
  extern __shared__ float2 smem[];
  __shared__ int s_next;
  __shared__ long long s_off[256];
  if (threadIdx.x == 0) s_next = atomicAdd(m.head, 1);
  __syncthreads();
  int idx = s_next;
  while (idx < m.nitems) {
    // claim the following item now (its index is read after this item's
    // closing barrier); items are still claimed in queue order, and a CTA's
    // claimed-but-unstarted item starts as soon as its current one ends, so
    // the earliest unfinished item is always being worked on
    __syncthreads();
    if (threadIdx.x == 0) s_next = atomicAdd(m.head, 1);
    const ManyItem it = m.items[idx];
    TileArgs a;
    memset(&a, 0, sizeof(a));
    a.stream_in = 1;
    a.stream_out = 1;
    if (it.kind == 0) {
      a.conj_in = m.conj;
      switch (it.lg) {
        case 1: many_batch_tile<1>(m, it, a, smem, s_off); break;
        case 2: many_batch_tile<2>(m, it, a, smem, s_off); break;
        case 3: many_batch_tile<3>(m, it, a, smem, s_off); break;
        case 4: many_batch_tile<4>(m, it, a, smem, s_off); break;
        case 5: many_batch_tile<5>(m, it, a, smem, s_off); break;
        case 6: many_batch_tile<6>(m, it, a, smem, s_off); break;
        case 7: many_batch_tile<7>(m, it, a, smem, s_off); break;
        case 8: many_batch_tile<8>(m, it, a, smem, s_off); break;
        case 9: many_batch_tile<9>(m, it, a, smem, s_off); break;
        case 10: many_batch_tile<10>(m, it, a, smem, s_off); break;
        case 11: many_batch_tile<11>(m, it, a, smem, s_off); break;
        case 12: many_batch_tile<12>(m, it, a, smem, s_off); break;
      }
    } else if (it.kind == 1) {
      const ManyTransform t = m.trs[it.tr];
      a.conj_in = m.conj;
      if (t.lg1 == 7) many_col_tile<7>(m, it, t, a, smem);
      else many_col_tile<8>(m, it, t, a, smem);
      // publish: every thread's stores are visible before the counter moves
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(m.done + it.tr, 1);
    } else {
      const ManyTransform t = m.trs[it.tr];
      if (threadIdx.x == 0) {
        if (!many_wait(m.done + it.tr, it.need, m.wait_budget)) atomicExch(m.status, FFT_ERR_TIMEOUT);
      }
      __syncthreads();
      if (t.lg2 == 6) many_row_tile<6>(m, it, t, a, smem);
      else if (t.lg2 == 7) many_row_tile<7>(m, it, t, a, smem);
      else many_row_tile<8>(m, it, t, a, smem);
    }
    __syncthreads();  // smem is reused by the next item; s_next is published
    idx = s_next;
  }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Fault injection for the bounded-wait test, compiled only into the test
// library libgbfft_testhooks.so (nvcc -DGBFFT_TEST_HOOKS); the product
// library libgbfft.so has no such switch.  In the test library, a plan created
// while GBFFT_FAULT_MISSING_PRODUCER=1 is set gets one row tile that waits for
// a column tile that does not exist, with a ~1 ms wait budget, so the timeout
// path is exercised without any GPU fault.
#ifdef GBFFT_TEST_HOOKS
static bool fault_missing_producer() {
  const char* e = getenv("GBFFT_FAULT_MISSING_PRODUCER");
  return e && atoi(e) != 0;
}
#else
static bool fault_missing_producer() { return false; }
#endif

// Resolves a configuration against the defaults; FFT_ERR_INVALID_ARG if a
// field is out of range.  ctas_per_sm is lowered to `occupancy` later.
int many_resolve_config(const fft_many_config* in, fft_many_config* out) {
  fft_many_config c{};
  c.gap = kManyDefaultGap;
  c.ctas_per_sm = 0;
  for (int i = 0; i < 4; ++i) c.lg1[i] = many_default_lg1(13 + i);
  if (in) {
    if (in->gap > kManyMaxGap) return FFT_ERR_INVALID_ARG;
    if (in->gap > 0) c.gap = in->gap;
    if (in->ctas_per_sm > 0) c.ctas_per_sm = in->ctas_per_sm;
    for (int i = 0; i < 4; ++i) {
      if (in->lg1[i] <= 0) continue;
      if (!many_split_ok(13 + i, in->lg1[i])) return FFT_ERR_INVALID_ARG;
      c.lg1[i] = in->lg1[i];
    }
  }
  *out = c;
  return FFT_OK;
}

int many_plan_init(fft_plan* p, const int64_t* lengths, int64_t count, const fft_many_config* cfg_in) {
  if (count > (1 << 24)) return FFT_ERR_INVALID_ARG;
  fft_many_config cfg;
  if (many_resolve_config(cfg_in, &cfg) != FFT_OK) return FFT_ERR_INVALID_ARG;
  std::vector<int> lg(count);
  long long total = 0;
  for (int64_t i = 0; i < count; ++i) {
    const int64_t n = lengths[i];
    if (n < 2 || n > (1 << 16) || (n & (n - 1))) return FFT_ERR_INVALID_ARG;
    int l = 0;
    while ((1LL << l) < n) ++l;
    lg[i] = l;
    total += n;
  }
  std::vector<long long> off(count);
  {
    long long o = 0;
    for (int64_t i = 0; i < count; ++i) {
      off[i] = o;
      o += lengths[i];
    }
  }
  // batch tiles: group transforms of equal length (<= 2^12), largest first
  std::vector<ManyItem> batch_items;
  std::vector<long long> slots;
  std::vector<ManyTransform> trs;
  long long ws_total = 0;
  for (int L = 12; L >= 1; --L) {
    const int C = (L >= 4) ? (4096 >> L) : 256;
    std::vector<long long> grp;
    for (int64_t i = 0; i < count; ++i)
      if (lg[i] == L) grp.push_back(off[i]);
    for (size_t s = 0; s < grp.size(); s += C) {
      ManyItem it{};
      it.kind = 0;
      it.lg = L;
      it.ncols = (int)std::min<size_t>(C, grp.size() - s);
      it.tr = (int)slots.size();
      for (int c = 0; c < it.ncols; ++c) slots.push_back(grp[s + c]);
      batch_items.push_back(it);
    }
  }
  // resident CTAs of the persistent launch (sets the queue distance below)
  if (cudaFuncSetAttribute(many_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kManySmem) != cudaSuccess)
    return FFT_ERR_CUDA;
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, many_kernel, kManyThreads, kManySmem) != cudaSuccess ||
      per_sm < 1)
    return FFT_ERR_CUDA;
  cfg.ctas_per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, per_sm) : per_sm;
  const size_t resident = (size_t)cfg.ctas_per_sm * (size_t)sms;
  // items queued between a transform's column and row tiles (in units of
  // half the resident grid)
  const size_t gap = (size_t)cfg.gap * resident / 2;

  // four-step transforms, largest first: column tiles in order, each
  // transform's row tiles once `gap` more items have been queued
  std::vector<ManyItem> fourstep;
  std::vector<std::pair<size_t, size_t>> pending;   // (queue position of the last column tile, transform)
  std::vector<std::vector<ManyItem>> rows_of;
  for (int L = 16; L >= 13; --L) {
    for (int64_t i = 0; i < count; ++i) {
      if (lg[i] != L) continue;
      ManyTransform t{};
      t.off = off[i];
      t.ws_off = ws_total;
      t.lgN = L;
      t.lg1 = cfg.lg1[L - 13];
      t.lg2 = L - t.lg1;
      t.c1 = 4096 >> t.lg1;
      t.c2 = 4096 >> t.lg2;
      ws_total += 1LL << L;
      const int tr = (int)trs.size();
      const int ncol_tiles = (int)((1LL << t.lg2) / t.c1);
      const int nrow_tiles = (int)((1LL << t.lg1) / t.c2);
      for (int g = 0; g < ncol_tiles; ++g) fourstep.push_back(ManyItem{1, t.lg1, t.c1, tr, g, 0});
      rows_of.emplace_back();
      for (int g = 0; g < nrow_tiles; ++g) rows_of.back().push_back(ManyItem{2, t.lg2, t.c2, tr, g, ncol_tiles});
      pending.emplace_back(fourstep.size(), (size_t)tr);
      trs.push_back(t);
      // release the row tiles of every transform whose column tiles are far enough back
      size_t k = 0;
      while (k < pending.size() && fourstep.size() - pending[k].first >= gap) ++k;
      for (size_t i = 0; i < k; ++i)
        fourstep.insert(fourstep.end(), rows_of[pending[i].second].begin(), rows_of[pending[i].second].end());
      pending.erase(pending.begin(), pending.begin() + k);
    }
  }
  for (auto& pr : pending) fourstep.insert(fourstep.end(), rows_of[pr.second].begin(), rows_of[pr.second].end());
  std::vector<ManyItem> items;
  items.insert(items.end(), fourstep.begin(), fourstep.end());
  items.insert(items.end(), batch_items.begin(), batch_items.end());
  const bool starve = fault_missing_producer();
  if (starve && !trs.empty()) {
    // injected fault: one row tile waits for a column tile that does not exist
    for (ManyItem& it : items)
      if (it.kind == 2) {
        it.need += 1;
        break;
      }
  }

  // twiddle tables: stage tables for every tile length 1..12, two-level W_N
  // tables for every four-step length 13..16
  int stage_off[13] = {0};
  int st_total = 0;
  for (int L = 1; L <= 12; ++L) {
    stage_off[L] = st_total;
    st_total += stage_tw_size(L) + 1;
  }
  int ft_off[17] = {0};
  int ft_total = 0;
  for (int L = 13; L <= 16; ++L) {
    ft_off[L] = ft_total;
    ft_total += (1 << ((L + 1) / 2)) + (1 << (L - (L + 1) / 2));
  }

  ManyPlan* mp = new (std::nothrow) ManyPlan;
  if (!mp) return FFT_ERR_ALLOC;
  p->many = mp;
  mp->cfg = cfg;
  const size_t b_items = al256(sizeof(ManyItem) * (items.size() + 1));
  const size_t b_trs = al256(sizeof(ManyTransform) * (trs.size() + 1));
  const size_t b_slots = al256(sizeof(long long) * (slots.size() + 1));
  const size_t b_st = al256(sizeof(float2) * (st_total + 1));
  const size_t b_sto = al256(sizeof(int) * 13);
  const size_t b_ft = al256(sizeof(float2) * (ft_total + 1));
  const size_t b_fto = al256(sizeof(int) * 17);
  const size_t b_cnt = al256(sizeof(int) * (trs.size() + 2));
  const size_t total_b = b_items + b_trs + b_slots + b_st + b_sto + b_ft + b_fto + b_cnt;
  char* base = nullptr;
  if (cudaMalloc(&base, total_b) != cudaSuccess) return FFT_ERR_ALLOC;
  mp->d_mem = base;
  char* q = base;
  ManyItem* d_items = (ManyItem*)q; q += b_items;
  ManyTransform* d_trs = (ManyTransform*)q; q += b_trs;
  long long* d_slots = (long long*)q; q += b_slots;
  float2* d_st = (float2*)q; q += b_st;
  int* d_sto = (int*)q; q += b_sto;
  float2* d_ft = (float2*)q; q += b_ft;
  int* d_fto = (int*)q; q += b_fto;
  int* d_cnt = (int*)q;
  if (cudaMemcpy(d_items, items.data(), sizeof(ManyItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      (trs.size() && cudaMemcpy(d_trs, trs.data(), sizeof(ManyTransform) * trs.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      (slots.size() && cudaMemcpy(d_slots, slots.data(), sizeof(long long) * slots.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(d_sto, stage_off, sizeof(stage_off), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_fto, ft_off, sizeof(ft_off), cudaMemcpyHostToDevice) != cudaSuccess)
    return FFT_ERR_CUDA;
  for (int L = 1; L <= 12; ++L)
    if (launch_gen_stage_twiddles(d_st + stage_off[L], L, 0) != cudaSuccess) return FFT_ERR_CUDA;
  for (int L = 13; L <= 16; ++L) {
    const int s = (L + 1) / 2;
    if (launch_gen_power_twiddles(d_ft + ft_off[L], L, 1LL << s, 1, 0) != cudaSuccess ||
        launch_gen_power_twiddles(d_ft + ft_off[L] + (1 << s), L, 1LL << (L - s), 1LL << s, 0) != cudaSuccess)
      return FFT_ERR_CUDA;
  }
  // status word: reuse the plan's convention (a separate small allocation)
  if (cudaMalloc(&p->d_tables, 256) != cudaSuccess) return FFT_ERR_ALLOC;
  p->d_status = (int*)p->d_tables;
  if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return FFT_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return FFT_ERR_CUDA;

  mp->grid = (int)std::min<long long>((long long)resident, (long long)items.size());
  mp->nitems = (int)items.size();
  mp->total = total;
  mp->d_counters = d_cnt;
  mp->counters_bytes = sizeof(int) * (trs.size() + 2);

  ManyArgs& m = mp->args;
  m.items = d_items;
  m.trs = d_trs;
  m.offs = d_slots;
  m.stage_tw = d_st;
  m.stage_tw_off = d_sto;
  m.ft_tab = d_ft;
  m.ft_off = d_fto;
  m.head = d_cnt;
  m.done = d_cnt + 1;
  m.status = p->d_status;
  m.nitems = mp->nitems;
  m.wait_budget = starve ? 2000000LL : 4000000000LL;  // ~1 ms under the injected fault, ~2 s otherwise

  p->n = total;
  p->ws_bytes = (size_t)ws_total * 8;
  p->launches = 1;
  return FFT_OK;
}

int many_get_config(const fft_plan* p, fft_many_config* out) {
  if (!p->many) return FFT_ERR_INVALID_ARG;
  *out = p->many->cfg;
  return FFT_OK;
}

void many_plan_free(fft_plan* p) {
  if (!p->many) return;
  if (p->many->d_mem) cudaFree(p->many->d_mem);
  delete p->many;
  p->many = nullptr;
}

int many_exec(fft_plan* p, const float2* in, float2* out, int dir, cudaStream_t s) {
  ManyPlan* mp = p->many;
  if (!mp) return FFT_ERR_INVALID_ARG;
  if (p->ws_bytes && !p->ws) return FFT_ERR_NO_WORKSPACE;
  ManyArgs m = mp->args;
  m.in = in;
  m.out = out;
  m.ws = (float2*)p->ws;
  const int inv = dir & FFT_INVERSE, adj = (dir & FFT_ADJOINT) ? 1 : 0;
  m.conj = inv ^ adj;
  m.inv = inv;
  if (cudaMemsetAsync(mp->d_counters, 0, mp->counters_bytes, s) != cudaSuccess) return FFT_ERR_CUDA;
  void* args[] = {(void*)&m};
  if (cudaLaunchKernel((const void*)many_kernel, dim3(mp->grid), dim3(kManyThreads), args, kManySmem, s) !=
      cudaSuccess)
    return FFT_ERR_CUDA;
  return FFT_OK;
}

}  // namespace gbfft
