/*
 * fft_oracle.c -- plain FP64 CPU oracle for the complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path (the CUDA library and
 * its Python binding) may link, load or call this code; only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg do.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (paper, Sec. 2.1):
 *   Eq. 1  X(k) = sum_{n=0}^{N-1} x(n) W_N^{nk},            k = 0..N-1
 *   Eq. 2  x(n) = (1/N) sum_{k=0}^{N-1} X(k) W_N^{-nk},     n = 0..N-1
 * with W_N = exp(-2*pi*i/N) (the paper never writes W_N out; this is the
 * usual forward sign).  Eq. 4, (W^{nk})^* = W^{-nk}, makes the inverse the
 * conjugate-direction sum times 1/N; the adjoint of the forward transform is
 * the same conjugate-direction sum without the 1/N.
 *
 * Direction codes: 0 = forward (Eq. 1), 1 = inverse (Eq. 2),
 *                  2 = adjoint of forward (conjugate direction, no scale).
 *
 * Layout: complex values are interleaved (re, im) doubles; a batch of B
 * transforms of length N is B*N complex values, transform b at offset b*N.
 *
 * Routines:
 *   oracle_dft  -- Eq. 1/2 summed term by term, O(N^2).  The exponent n*k is
 *                  reduced mod N first (Eq. 3, periodicity), so every angle is
 *                  2*pi*m/N with 0 <= m < N.
 *   oracle_dft_bins -- the same sum at chosen outputs k only, O(N) each.
 *   oracle_fft  -- the textbook recursive radix-2 decimation-in-time
 *                  Cooley-Tukey split (the butterfly of Sec. 2.1): even and
 *                  odd samples are transformed separately and combined as
 *                  X(k) = E(k) + W_N^k O(k), X(k+N/2) = E(k) - W_N^k O(k).
 *                  N must be a power of two.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* W_N^m for sign s (s = -1 forward, +1 conjugate direction), m reduced mod N
 * (Eq. 3) so the angle 2*pi*m/N lies in [0, 2*pi). */
static void oracle_w(int64_t m, int64_t n, int s, double *wr, double *wi)
{
    m %= n;
    if (m < 0) m += n;
    double a = 2.0 * M_PI * (double)m / (double)n;
    *wr = cos(a);
    *wi = (double)s * sin(a);
}

static int dir_sign(int dir) { return dir == 0 ? -1 : +1; }
static double dir_scale(int dir, int64_t n) { return dir == 1 ? 1.0 / (double)n : 1.0; }

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

/* Eq. 1 (dir 0), Eq. 2 (dir 1) or the adjoint (dir 2), term by term. */
int oracle_dft(int64_t n, const double *in, double *out, int dir)
{
    if (n < 1 || dir < 0 || dir > 2 || in == out) return -1;
    const int s = dir_sign(dir);
    const double scale = dir_scale(dir, n);
    for (int64_t k = 0; k < n; ++k) {
        double acc_r = 0.0, acc_i = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double wr, wi;
            /* (j*k) mod n without overflow for n <= 2^31 */
            int64_t m = (int64_t)(((unsigned __int128)j * (unsigned __int128)k) % (unsigned __int128)n);
            oracle_w(m, n, s, &wr, &wi);
            const double xr = in[2 * j], xi = in[2 * j + 1];
            acc_r += xr * wr - xi * wi;
            acc_i += xr * wi + xi * wr;
        }
        out[2 * k] = acc_r * scale;
        out[2 * k + 1] = acc_i * scale;
    }
    return 0;
}

/* Eq. 1 (dir 0), Eq. 2 (dir 1) or the adjoint (dir 2) at the listed outputs
 * only: out[b] = scale * sum_j in[j] W^{j * bins[b]}, b < nbins, each summed
 * term by term like oracle_dft.  Single outputs of transforms too long for
 * the O(N^2) sum over every output are checked this way. */
int oracle_dft_bins(int64_t n, const double *in, int64_t nbins, const int64_t *bins, double *out, int dir)
{
    if (n < 1 || nbins < 0 || dir < 0 || dir > 2 || !in || !out || (nbins > 0 && !bins)) return -1;
    const int s = dir_sign(dir);
    const double scale = dir_scale(dir, n);
    for (int64_t b = 0; b < nbins; ++b) {
        const int64_t bin = bins[b];
        if (bin < 0 || bin >= n) return -1;
        double sum_r = 0.0, sum_i = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double wr, wi;
            int64_t e = (int64_t)(((unsigned __int128)j * (unsigned __int128)bin) % (unsigned __int128)n);
            oracle_w(e, n, s, &wr, &wi);
            sum_r += in[2 * j] * wr - in[2 * j + 1] * wi;
            sum_i += in[2 * j] * wi + in[2 * j + 1] * wr;
        }
        out[2 * b] = sum_r * scale;
        out[2 * b + 1] = sum_i * scale;
    }
    return 0;
}

/* Recursive radix-2 DIT on x[0], x[stride], ..., x[(n-1)*stride] -> y[0..n). */
static void fft_rec(int64_t n, const double *x, int64_t stride, double *y, int s)
{
    if (n == 1) {
        y[0] = x[0];
        y[1] = x[1];
        return;
    }
    const int64_t h = n / 2;
    fft_rec(h, x, 2 * stride, y, s);                   /* E: even samples -> y[0..h)  */
    fft_rec(h, x + 2 * stride, 2 * stride, y + 2 * h, s); /* O: odd samples  -> y[h..n) */
    for (int64_t k = 0; k < h; ++k) {
        double wr, wi;
        oracle_w(k, n, s, &wr, &wi);
        const double er = y[2 * k], ei = y[2 * k + 1];
        const double orr = y[2 * (h + k)], oi = y[2 * (h + k) + 1];
        const double tr = wr * orr - wi * oi;
        const double ti = wr * oi + wi * orr;
        y[2 * k] = er + tr;
        y[2 * k + 1] = ei + ti;
        y[2 * (h + k)] = er - tr;
        y[2 * (h + k) + 1] = ei - ti;
    }
}

int oracle_fft(int64_t n, const double *in, double *out, int dir)
{
    if (!is_pow2(n) || dir < 0 || dir > 2 || in == out) return -1;
    fft_rec(n, in, 1, out, dir_sign(dir));
    const double scale = dir_scale(dir, n);
    if (scale != 1.0)
        for (int64_t i = 0; i < 2 * n; ++i) out[i] *= scale;
    return 0;
}

/* Batched forms: transform b reads in + 2*b*n and writes out + 2*b*n. */
int oracle_dft_batch(int64_t n, int64_t batch, const double *in, double *out, int dir)
{
    for (int64_t b = 0; b < batch; ++b) {
        int rc = oracle_dft(n, in + 2 * b * n, out + 2 * b * n, dir);
        if (rc) return rc;
    }
    return 0;
}

int oracle_fft_batch(int64_t n, int64_t batch, const double *in, double *out, int dir)
{
    for (int64_t b = 0; b < batch; ++b) {
        int rc = oracle_fft(n, in + 2 * b * n, out + 2 * b * n, dir);
        if (rc) return rc;
    }
    return 0;
}

/*
 * 2-D transform of an ny-by-nx row-major image (element (y, x) at y*nx + x):
 *   X(ky, kx) = sum_y sum_x x(y, x) W_ny^{y*ky} W_nx^{x*kx}
 * computed as the definition separates: a 1-D transform of every row, then a
 * 1-D transform of every column (the rows-then-columns order of Sec. 2.3.2).
 * The inverse scales by 1/(ny*nx) through the two 1-D inverses.
 */
int oracle_fft2(int64_t ny, int64_t nx, const double *in, double *out, int dir)
{
    if (!is_pow2(ny) || !is_pow2(nx) || dir < 0 || dir > 2 || in == out) return -1;
    int rc = oracle_fft_batch(nx, ny, in, out, dir);
    if (rc) return rc;
    double *col = (double *)malloc(sizeof(double) * 2 * (size_t)ny);
    double *res = (double *)malloc(sizeof(double) * 2 * (size_t)ny);
    if (!col || !res) {
        free(col);
        free(res);
        return -2;
    }
    for (int64_t x = 0; x < nx; ++x) {
        for (int64_t y = 0; y < ny; ++y) {
            col[2 * y] = out[2 * (y * nx + x)];
            col[2 * y + 1] = out[2 * (y * nx + x) + 1];
        }
        oracle_fft(ny, col, res, dir);
        for (int64_t y = 0; y < ny; ++y) {
            out[2 * (y * nx + x)] = res[2 * y];
            out[2 * (y * nx + x) + 1] = res[2 * y + 1];
        }
    }
    free(col);
    free(res);
    return 0;
}
