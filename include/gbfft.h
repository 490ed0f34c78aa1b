/*
 * gbfft.h -- C ABI of the GB300 (sm_103a) complex FFT library: power-of-two
 * lengths (1-D, 2-D, uneven batches, real data) and 7-smooth lengths.
 *
 * What the library computes (paper Sec. 2.1):
 *   forward  (Eq. 1):  X(k) = sum_{n=0}^{N-1} x(n) W_N^{nk},            W_N = exp(-2*pi*i/N)
 *   inverse  (Eq. 2):  x(n) = (1/N) sum_{k=0}^{N-1} X(k) W_N^{-nk}
 *   adjoint  (Eq. 4):  the conjugate-direction sum without the 1/N, i.e. F^H.
 * Outputs are in natural order.  Data are complex64: interleaved (re, im)
 * float32 pairs, contiguous; a batch of B transforms of length N is B*N
 * complex values with transform b at offset b*N.  2-D images are row-major
 * (element (y, x) at y*nx + x).  FFT_PREC_FP64 plans take complex128 (re, im
 * double pairs) instead; real-data plans (fft_plan_create_r2c) take rows of
 * float32 and give rows of n/2 + 1 complex64.
 *
 * Memory: every data pointer passed to fft_exec* is owned by the caller and
 * is device memory, or page-locked host memory the device can address
 * (fft_pointer_usable), at least 8-byte aligned (16 for FFT_PREC_FP64;
 * FFT_ERR_ALIGN otherwise).  in == out (in place) is allowed for every plan
 * kind except real-data plans.  The library allocates only at
 * plan creation (the twiddle tables) and in fft_plan_set_workspace(plan, NULL);
 * fft_exec* never allocates, never synchronises the stream and is safe to
 * capture into a CUDA graph.
 *
 * Errors: calls return 0 (FFT_OK) or a negative FFT_ERR_* code; plan
 * constructors return NULL on error.  The code of the last failing call on
 * the calling host thread is kept in fft_last_error().  Argument errors are
 * detected on the host before anything is launched, including plan pointers
 * that are not live plans (see fft_destroy).
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GBFFT_API __attribute__((visibility("default")))
#else
#define GBFFT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_plan fft_plan; /* opaque, owned by the library */

/* Directions.  FFT_ADJOINT is a flag: FFT_ADJOINT alone is the adjoint of the
 * forward transform (conjugate direction, no scale, Eq. 4), and
 * FFT_INVERSE | FFT_ADJOINT is the adjoint of the inverse (forward direction
 * with 1/N). */
enum { FFT_FORWARD = 0, FFT_INVERSE = 1, FFT_ADJOINT = 2 };

/* Arithmetic of the radix-16 passes.  FP32 is the plain path.  The TC_*
 * variants run each radix-16 DFT as a small dense product on the tensor cores
 * (BF16 or FP16 operands, FP32 accumulation); *_SPLIT adds hi+lo operand
 * splitting (three products) to win back accuracy.  Twiddles stay FP32. */
enum {
  FFT_PREC_FP32 = 0,
  FFT_PREC_TC_BF16 = 1,
  FFT_PREC_TC_FP16 = 2,
  FFT_PREC_TC_BF16_SPLIT = 3,
  FFT_PREC_TC_FP16_SPLIT = 4,
  /* complex128 data and FP64 arithmetic; 1-D plans of 7-smooth length
   * n = 2^a 3^b 5^c 7^d (powers of two included): one on-chip pass for
   * 2 <= n <= 7168, two strided passes (four-step, workspace) for
   * 7168 < n <= 7168^2 when n = N1 N2 with N1, N2 <= 7168 (powers of two up
   * to 2^24); 2-D plans of 7-smooth sides up to 7168; in and out 16-byte
   * aligned */
  FFT_PREC_FP64 = 5
};

enum {
  FFT_OK = 0,
  FFT_ERR_INVALID_ARG = -1,   /* n not a supported length, batch < 1, bad dir/prec, NULL */
  FFT_ERR_ALIGN = -2,         /* data pointer not 8-byte aligned */
  FFT_ERR_NO_WORKSPACE = -3,  /* plan needs a workspace and none was set */
  FFT_ERR_CUDA = -4,          /* a CUDA runtime call or launch failed */
  FFT_ERR_TIMEOUT = -5,       /* a bounded device-side wait ran out */
  FFT_ERR_UNSUPPORTED = -6,   /* valid request this build does not implement */
  FFT_ERR_ALLOC = -7          /* host or device allocation failed at plan time */
};

/* Largest supported 1-D length (2^28) and 2-D side (2^14). */
#define FFT_MAX_LOG2N 28
#define FFT_MAX_LOG2_SIDE 14

/* Plan for `batch` 1-D transforms of length n: a power of two, 2 <= n <= 2^28,
 * or (FP32 and FP64) a product n = 2^a 3^b 5^c 7^d (mixed radix: Eq. 1 holds
 * for any n and the Cooley-Tukey split of Sec. 2.1 for any factorisation;
 * a config must be NULL).  Mixed-radix lengths up to 14336 run as one on-chip
 * pass of radix-16/8/4/2/3/5/7 stages; longer ones, up to 14336^2, as the
 * four-step split n = N1 N2 (N1 the largest divisor of n at most sqrt(n)
 * whose cofactor N2 is at most 14336): a strided column pass with the twiddle
 * W_n^{n2 k1}, then a row pass, through a workspace (fft_plan_kind 6).  A
 * 7-smooth n with no such split, or beyond 14336^2, gives FFT_ERR_UNSUPPORTED.
 * FP64 plans take the same routes with 7168 in place of 14336, for powers of
 * two as well (see FFT_PREC_FP64).
 * dir is the direction fft_exec uses (FFT_FORWARD, FFT_INVERSE, optionally
 * with FFT_ADJOINT); prec one of FFT_PREC_*.  Lengths up to 2^14 run as one
 * on-chip pass per transform (Sec. 2.3.2: short data is not partitioned);
 * longer ones are split N = N1*N2 into a column pass with twiddle scaling and
 * a row pass through global memory (Sec. 2.3.2: two exchanges between shared
 * and global memory); from 2^22 the rows are split once more (three passes).
 * Multi-pass plans need a workspace (fft_plan_workspace_bytes).
 * Builds the twiddle tables on the current device (FP64 sincospi rounded
 * once to FP32; Sec. 2.3.1 look-up table).  Returns NULL on error. */
GBFFT_API fft_plan* fft_plan_create(int64_t n, int64_t batch, int dir, int prec);

/* Plan for `batch` 2-D transforms of ny-by-nx row-major images: 1-D
 * transforms of every row, then of every column (Sec. 2.3.2: rows, then
 * columns).  Power-of-two sides 2 <= ny, nx <= 2^14 run on the radix-16 tile
 * kernels (every precision but FP64): a row pass and one or two column
 * passes, or, for sides of 2^10..2^12 (ny >= 2^11, or 1024 x 1024), two row
 * passes that each store their result transposed (the second transforms the
 * columns as rows); a workspace of one image batch where fft_plan_workspace_bytes
 * says so.  Sides that are 7-smooth but not both
 * powers of two (FP32, up to 14336), and every FP64 plan (7-smooth sides up
 * to 7168), run as a row pass and a column pass of the strided mixed-radix
 * kernel, the column pass in place in the output (no workspace; fft_plan_kind
 * 6).  A side with a prime factor above 7, or below 2, is FFT_ERR_INVALID_ARG;
 * a valid side beyond those limits, or tensor-core precisions with a side
 * that is not a power of two, FFT_ERR_UNSUPPORTED. */
GBFFT_API fft_plan* fft_plan_create_2d(int64_t ny, int64_t nx, int64_t batch, int dir, int prec);

/* Plan for `batch` real-data transforms of length n: FFT_PREC_FP32 with n a
 * power of two, 4 <= n <= 2^28 (float32 rows, complex64 spectra), or
 * FFT_PREC_FP64 with n even, n >= 4 and n/2 a 7-smooth FP64 length (float64
 * rows, complex128 spectra, 16-byte aligned; the complex128 plan of length
 * n/2 plus FP64 split kernels).  Other precisions: FFT_ERR_INVALID_ARG for
 * lengths that are not powers of two, else FFT_ERR_UNSUPPORTED.  Run it with
 * fft_exec_dir:
 *   FFT_FORWARD (real to complex): in = batch rows of n floats, out = batch
 *     rows of n/2 + 1 complex64 values X[k] = Eq. 1 of the row, k = 0..n/2
 *     (the other half is X[n-k] = conj X[k]).
 *   FFT_INVERSE (complex to real): in = batch rows of n/2 + 1 complex64 values,
 *     out = batch rows of n floats, Eq. 2 (with 1/n) of the Hermitian
 *     extension; Im X[0] and Im X[n/2] are ignored.
 * The row of n reals is read as n/2 complex values x[2m] + i x[2m+1] (Sec. 2.1
 * splits a sequence into even and odd samples the same way); one complex
 * transform of length n/2 and one split step give the result.  n <= 2^15: one
 * fused kernel, one read and one write of every value.  2^16 <= n <= 2^22,
 * real to complex: the complex plan's column pass, then its row pass with the
 * split folded in (rows k1 and n/2/N1 - k1 in one tile), two passes.
 * 2^16 <= n <= 2^21, complex to real: the split folded into the complex
 * plan's column pass (X[m] and X[n/2 - m] read from the same row), then its
 * row pass, two passes.  Other longer n and directions: the complex plan plus
 * one split kernel.  Multi-pass lengths need a workspace
 * (fft_plan_workspace_bytes).
 * The adjoints (for backpropagation; adjoint with respect to the real inner
 * product <u, v> = Re sum conj(u) v, which is PyTorch's gradient convention):
 *   FFT_ADJOINT (adjoint of FFT_FORWARD): in = rows of n/2 + 1 complex64 g,
 *     out = rows of n floats  y[m] = Re sum_{k=0}^{n/2} g[k] W_n^{-mk}
 *     (Eq. 4 over the kept bins; Im g[0] and Im g[n/2] do not enter).
 *   FFT_INVERSE | FFT_ADJOINT (adjoint of FFT_INVERSE): in = rows of n floats
 *     g, out = rows of n/2 + 1 complex64: Eq. 1 of g with bins 1..n/2-1 times
 *     2/n and bins 0 and n/2 times 1/n.
 * Both run in the same kernels as the transforms (the bin weights and the
 * scale are arguments of the split step), at the same cost.
 * Pointers 8-byte aligned, device memory or memory fft_pointer_usable accepts;
 * in == out is not allowed. */
GBFFT_API fft_plan* fft_plan_create_r2c(int64_t n, int64_t batch, int prec);

/* Plan for `count` 1-D transforms of uneven power-of-two lengths lengths[i]
 * (2^1..2^16), packed back to back: transform i starts at the prefix sum of
 * the lengths before it.  The host array is copied; the caller keeps it. */
GBFFT_API fft_plan* fft_plan_create_many(const int64_t* lengths, int64_t count, int dir, int prec);

/* Configuration of an uneven-batch plan (the knobs of fft_autotune_many).  The
 * plan runs as one persistent launch over a queue of tiles of at most 4096
 * points: batch tiles of equal-length transforms up to 2^12, and the column
 * and row tiles of a four-step split N = N1 * N2 (Sec. 2.3.2) for 2^13..2^16.
 *   gap:         the row tiles of a four-step transform are queued this many
 *                half resident grids after its column tiles (1..16; <= 0 =
 *                default 4).  Short gaps keep the intermediate in L2 but make
 *                row tiles wait; long gaps do the opposite.
 *   ctas_per_sm: resident CTAs per SM of the persistent launch (<= 0 = the
 *                occupancy limit of the kernel, 4; larger values are lowered
 *                to that limit).
 *   lg1[i]:      log2 N1 of the split for transforms of length 2^(13+i):
 *                2^13: 7, 2^14: 7 or 8, 2^15: 7 or 8, 2^16: 8
 *                (<= 0 = defaults 7, 7, 8, 8).  Other values are invalid. */
typedef struct fft_many_config {
  int gap, ctas_per_sm;
  int lg1[4];
} fft_many_config;

/* As fft_plan_create_many, with an explicit configuration (NULL = defaults).
 * NULL with FFT_ERR_INVALID_ARG for a configuration outside the ranges above. */
GBFFT_API fft_plan* fft_plan_create_many_config(const int64_t* lengths, int64_t count, int dir, int prec,
                                                const fft_many_config* cfg);

/* The resolved configuration of an uneven-batch plan (FFT_ERR_INVALID_ARG for
 * other plan kinds). */
GBFFT_API int fft_plan_get_many_config(const fft_plan* plan, fft_many_config* out);

/* Autotuner of uneven-batch plans: builds the plan for (lengths, count, prec)
 * under every configuration of the search space -- gap in {1, 2, 3, 4, 6, 8},
 * CTAs per SM from 2 to the occupancy limit, and every valid split for each
 * four-step length that occurs in `lengths` -- times each with CUDA events
 * over `iters` executions (after 3 untimed ones) on the caller's device
 * buffers in/out (the packed data, sum(lengths) complex64 each) and workspace
 * ws of ws_bytes (>= the plan's fft_plan_workspace_bytes), and writes the
 * fastest configuration to *best and its mean time in microseconds to
 * *best_us.  Synchronises `stream`; overwrites the buffers; creates plans, so
 * call it outside any stream capture.  FP32 only. */
GBFFT_API int fft_autotune_many(const int64_t* lengths, int64_t count, int prec, void* in, void* out, void* ws,
                                size_t ws_bytes, void* stream, int iters, fft_many_config* best, float* best_us);

/* Runs the plan on `stream` (a cudaStream_t; NULL = legacy default stream)
 * in the plan's direction.  Asynchronous: returns once the launches are
 * queued.  in/out: the packed data (complex64; complex128 for FFT_PREC_FP64;
 * see fft_plan_create_r2c for real-data plans) in device memory or in memory
 * fft_pointer_usable accepts.  FFT_ERR_NO_WORKSPACE if a multi-pass plan has
 * no workspace; a bounded device-side wait that ran out shows later in
 * fft_status, not here. */
GBFFT_API int fft_exec(fft_plan* plan, const void* in, void* out, void* stream);

/* As fft_exec, with an explicit direction instead of the plan's (the twiddle
 * tables serve every direction); used for the adjoint in backpropagation. */
GBFFT_API int fft_exec_dir(fft_plan* plan, const void* in, void* out, int dir, void* stream);

/* SAR range compression (fast convolution; Sec. 3 and Sec. 4 name FFT-based
 * SAR processing as the method's application): each of the plan's `batch`
 * rows x_b of length n becomes
 *     y_b = IFFT( H .* FFT(x_b) )      (Eq. 1, pointwise product, Eq. 2)
 * with one n-point frequency-domain filter H for every row (for a matched
 * filter, the conjugated spectrum of the transmitted pulse).
 *   plan:  a 1-D FP32 plan of fft_plan_create / fft_plan_create_config (not a
 *          fused two-pass configuration); its direction is not used.
 *   in, out: batch*n complex64 values, 8-byte aligned, device memory or memory
 *          fft_pointer_usable accepts; in == out allowed.
 *   filt:  n complex64 values in natural frequency order (k < n/2: k/n cycles
 *          per sample; k >= n/2: k/n - 1), 8-byte aligned, same kinds of memory.
 * n <= 2^14: one fused kernel; each row is read once and written once, the
 * product and both transforms on chip (separate calls move every value through
 * memory three times).  Longer n: the plan's passes run twice, the product
 * fused into the last pass of the first run; `out` holds the intermediate and
 * the plan's workspace is used.  Asynchronous on `stream`, no allocation,
 * capturable.  FFT_ERR_UNSUPPORTED for 2-D, uneven-batch, tensor-core and
 * fused two-pass plans. */
GBFFT_API int fft_exec_filter(fft_plan* plan, const void* in, void* out, const void* filt, void* stream);

/* As fft_exec_filter, with a direction: FFT_FORWARD is fft_exec_filter, and
 * FFT_ADJOINT computes the adjoint of range compression,
 *     y_b = IFFT( conj(H) .* FFT(x_b) )
 * (the adjoint of F^-1 diag(H) F is F^-1 diag(conj H) F, since F^-1 = F^H / n),
 * which is the backward pass of range compression with respect to x: the same
 * kernels, with the filter conjugated as it is loaded.  Other directions
 * return FFT_ERR_INVALID_ARG. */
GBFFT_API int fft_exec_filter_dir(fft_plan* plan, const void* in, void* out, const void* filt, int dir,
                                  void* stream);

/* Whether the GPU can read and write the `bytes` bytes at `ptr` through that
 * same address, so that fft_exec may take it as `in` or `out`: memory of the
 * current device, managed memory, or page-locked host memory mapped into the
 * device's address space at the same address (cudaHostAlloc or
 * cudaHostRegister under unified addressing, the default on 64-bit hosts).
 * Both ends of the range are checked.  Returns 1 if usable, 0 if not
 * (pageable or unknown host memory, another device's memory, a mapping at a
 * different device address), or a negative error code (FFT_ERR_INVALID_ARG
 * for NULL or bytes == 0).  With mapped host memory the kernels read and
 * write the batch over the host link while they transform it, with no
 * separate copy and no device buffer (the host<->device transfer that Sec. 3
 * and Sec. 4 count in their GPU times). */
GBFFT_API int fft_pointer_usable(const void* ptr, size_t bytes);

/* Explicit plan configuration (npass, lg1, lg2, c1, c2, c3 <= 0 mean
 * "planner default"; tma, fused < 0 mean default).  npass: 1 = one on-chip
 * pass (n <= 2^14), 2 = two passes N = 2^lg1 * 2^(lgN-lg1), 3 = three passes
 * 2^lg1 * 2^lg2 * 2^lg3.  c1, c2, c3: adjacent transforms (columns) per CTA of
 * each pass, 1..64.  tma: 1 = persistent TMA-staged kernels (single pass:
 * cp.async.bulk of contiguous tiles; multi-pass: column passes staged by
 * tensor TMA boxes), 2 = single pass 2^12..2^14 only: persistent register-path
 * kernel that prefetches the next transform into L2 while computing one,
 * 3 = as 2, and once the last pass has read the exchange buffer a bulk copy
 * brings the next transform into it, so the first pass reads shared memory
 * (inputs not 16-byte aligned take the tma = 2 kernel), 0 = register path.  fused: 1 = both passes of a two-pass split in one
 * persistent launch that pipelines slabs of the batch through an L2-resident
 * workspace (2^13..2^18; split and columns fixed by the kernel), 0 = one launch
 * per pass.  halves: single pass only, 2 = two CTAs per transform, each
 * computing the even or odd outputs from a radix-2 split of the input
 * (2^12..2^14), <= 1 = one CTA per transform.  radix: single pass on the
 * register path only (tma <= 0, halves <= 1, FFT_PREC_FP32): the largest
 * radix of the Stockham passes, which is also the number of points each
 * thread holds, and so sets the threads per CTA (transforms per CTA x n /
 * radix): 8 = radix-8 passes (n = 2^5..2^13), 4 = radix-4 passes
 * (n = 2^5..2^12), 16 = radix-16 passes (every other kernel), <= 0 = the
 * planner's choice (radix 8 at n = 2^5 and 2^6 when npass, tma, fused and
 * halves are left at their defaults too, radix 16 otherwise); any other
 * value, or 4 / 8 where no such kernel is compiled, gives
 * FFT_ERR_UNSUPPORTED.  fft_plan_get_config reports 16 unless a smaller radix
 * was chosen.  These are the knobs of the autotuner (fft_autotune). */
typedef struct fft_plan_config {
  int npass, lg1, lg2, c1, c2, c3, tma, fused, halves, radix;
} fft_plan_config;

/* As fft_plan_create, with an explicit configuration (NULL = defaults).
 * Returns NULL with FFT_ERR_UNSUPPORTED if the configuration has no
 * compiled kernel. */
GBFFT_API fft_plan* fft_plan_create_config(int64_t n, int64_t batch, int dir, int prec, const fft_plan_config* cfg);

/* The configuration a 1-D plan was built with. */
GBFFT_API int fft_plan_get_config(const fft_plan* plan, fft_plan_config* out);

/* Autotuner: builds every candidate configuration for (n, batch, prec) --
 * one or two or three passes, the split lengths near the even split, columns
 * per CTA around the default, TMA staging on/off, the largest radix of a
 * single pass (16, 8 or 4) -- times each with CUDA
 * events over `iters` executions (after 3 untimed ones) on the caller's
 * device buffers in/out (n*batch complex64 each) and workspace ws of ws_bytes
 * (>= n*batch*8 bytes), and writes the fastest configuration to *best and its
 * mean time in microseconds to *best_us.  Synchronises `stream`.  The buffers'
 * contents are overwritten.  Plans are created and destroyed internally, so
 * call it outside any stream capture.  Only FFT_PREC_FP32 power-of-two
 * lengths have choices (mixed-radix and FP64 plans take no configuration). */
GBFFT_API int fft_autotune(int64_t n, int64_t batch, int prec, void* in, void* out, void* ws, size_t ws_bytes,
                           void* stream, int iters, fft_plan_config* best, float* best_us);

/* Frees the plan and everything the library allocated for it.  NULL-safe.
 * The library keeps a record of the plans it has handed out: a pointer that
 * is not a live plan (never returned by a constructor, or destroyed already)
 * frees nothing here and sets FFT_ERR_INVALID_ARG, and every other call
 * rejects it with FFT_ERR_INVALID_ARG (or 0 / -1 from the queries). */
GBFFT_API void fft_destroy(fft_plan* plan);

/* Bytes of device workspace fft_exec needs (0 for single-pass and 2-D plans). */
GBFFT_API size_t fft_plan_workspace_bytes(const fft_plan* plan);

/* Gives the plan a caller-owned device workspace of at least
 * fft_plan_workspace_bytes(plan) bytes (256-byte aligned), or, with NULL, makes
 * the library allocate and own one now.  Returns FFT_OK or an error code. */
GBFFT_API int fft_plan_set_workspace(fft_plan* plan, void* dev_ptr);

/* Descriptive queries (for tests and the benchmark). */
GBFFT_API int64_t fft_plan_length(const fft_plan* plan);
GBFFT_API int64_t fft_plan_batch(const fft_plan* plan);
/* Number of kernel launches one fft_exec issues (real-data plans: the largest
 * of the directions; a folded direction issues one fewer than the complex
 * plan plus a split kernel). */
GBFFT_API int fft_plan_launches(const fft_plan* plan);
/* Kind: 0 single on-chip pass, 1 four-step, 2 two-dimensional, 3 uneven batch,
 * 4 real data, 5 mixed radix (one pass), 6 two strided mixed-radix passes
 * (mixed-radix or FP64 four-step, mixed-radix or FP64 2-D). */
GBFFT_API int fft_plan_kind(const fft_plan* plan);
/* Human-readable plan summary into buf (NUL-terminated); returns FFT_OK. */
GBFFT_API int fft_plan_describe(const fft_plan* plan, char* buf, size_t len);

/* Device-side status word of the plan (0 = OK, FFT_ERR_TIMEOUT if a bounded
 * wait gave up).  Synchronises `stream` to read it. */
GBFFT_API int fft_status(fft_plan* plan, void* stream);

/* Allocation-free four-step transform, for callers that cannot allocate device
 * memory when they need a transform (inside an allocator or memory-pool
 * callback, in a plug-in whose host owns all device memory, on real-time paths
 * that allow allocation only at start-up).  The paper has no counterpart; it
 * computes what fft_exec_dir computes on a four-step plan of (n, batch).
 *   n:      power of two, 2^15 <= n <= 2^22;  batch >= 1 and n*batch <= 2^22,
 *           anything larger returns FFT_ERR_INVALID_ARG without launching.
 *   dir:    as fft_exec_dir.  in/out: caller-owned device pointers (8-byte
 *           aligned, in == out allowed).  stream: cudaStream_t or NULL.
 * Nothing is allocated per call: the workspace (32 MiB) and the twiddle tables
 * live in a static device array inside the library.  The CUDA runtime loads a
 * library's device code, and with it this array, onto a device the first time
 * the library is used there (lazy module loading, the default), and that load
 * does allocate device memory.  So make one call on each device at start-up,
 * from a context that may allocate and outside any stream capture: that first
 * call loads the kernels and the array, looks up the array's device address
 * and raises the kernels' shared-memory limit, once per device.  From then on
 * the array stays reserved on that device until the process exits, and calls
 * allocate nothing.  All calls share the array and find the previous call's
 * contents in it (each call rewrites what it reads): calls whose work overlaps
 * on the GPU race on it, so serialise them. */
GBFFT_API int fft_exec_noalloc(int64_t n, int64_t batch, int dir, const void* in, void* out, void* stream);

/* Code of the last failing call on this host thread (FFT_OK if none). */
GBFFT_API int fft_last_error(void);
/* Static description of an error code. */
GBFFT_API const char* fft_error_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
