/*
 * rl_oracle.c -- FP64 CPU oracle for 3D Richardson-Lucy deconvolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) links, loads or calls this file.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark use it.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes follows the paper (arXiv 2510.14143), Section 4,
 * "Richardson-Lucy deconvolution": each iteration (1) blurs the estimate with
 * the PSF, (2) divides the measured volume by that blur, (3) correlates the
 * quotient with the PSF (convolution with the mirrored PSF) and (4) multiplies
 * the estimate by the result.  In the same section the PSF volume is as large
 * as the image and the convolutions run through FFTs.  Where the paper is
 * silent the oracle takes these readings:
 *   - circular boundaries (FFT convolution of same-size arrays, no padding);
 *   - the PSF peak sits at index floor(n/2) on every axis and is moved to
 *     the origin before the transform;
 *   - "flipped PSF" is the circular flip h0(-x mod n), i.e. the adjoint of
 *     the forward convolution (conj(H) in Fourier space);
 *   - initial estimate u0 = max(mean(d), eps) everywhere;
 *   - the ratio's denominator is clamped: r = d / max(b, eps).
 *
 * Everything is double precision, arrays are C-order [nz][ny][nx] (x fastest).
 * FFT convention: forward X[k] = sum_n x[n] exp(-2 pi i k n / N), inverse
 * carries 1/N per axis.  Transforms are full complex transforms; the real
 * part is taken after each inverse (no half-spectrum tricks).
 *
 * FFT: iterative radix-2 decimation-in-time for powers of two; Bluestein's
 * chirp-z method (built on the same radix-2 code) for every other length;
 * an O(N^2) brute-force DFT for tests.
 *
 * Gradient: plain reverse mode over the same steps, storing every iterate.
 * Gaussian PSF: h = A * g / sum(g), g = exp(-(dx^2+dy^2)/(2 sxy^2) - dz^2/(2 sz^2)),
 * (dx,dy,dz) = index - floor(n/2).
 *
 * Beyond the plain iteration, each with its citation and readings at its definition:
 * automatic and metric-guided stopping (Section 4; the relative change, the Poisson
 * likelihood and the scale-invariant PSNR of Section 3's metric list), linear
 * ("same"-mode) boundaries for a PSF box smaller than the image, accelerated RL
 * (the Biggs-Andrews extrapolation cited in Section 2), and the Fourier shell
 * correlation, two-volume and single-image (Sections 3 and 4).  Every entry point is
 * pinned by the CPU tests to closed forms, direct loops or brute force.
 *
 * All entry points return 0 on success and a negative value on bad input or
 * allocation failure.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* ---------------------------------------------------------------- FFT 1D */

/* In-place iterative radix-2 DIT FFT, forward (sign=-1) or unnormalised
 * backward (sign=+1).  n must be a power of two. */
static void fft_radix2(cplx *x, int64_t n, int sign)
{
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len / 2;
        for (int64_t k = 0; k < half; ++k) {
            double a = sign * 2.0 * PI * (double)k / (double)len;
            cplx w = cos(a) + I * sin(a);
            for (int64_t s = 0; s < n; s += len) {
                cplx e = x[s + k];
                cplx o = x[s + k + half] * w;
                x[s + k] = e + o;
                x[s + k + half] = e - o;
            }
        }
    }
}

/* Bluestein / chirp-z: length-n DFT as a circular convolution of length
 * m >= 2n-1 (m a power of two) done with radix-2 FFTs.
 * exp(sign*2 pi i k j/n) = w_k w_j conj(w_{k-j}) with w_j = exp(sign*pi i j^2/n). */
static int fft_bluestein(cplx *x, int64_t n, int sign)
{
    int64_t m = 1;
    while (m < 2 * n - 1) m <<= 1;
    cplx *w = malloc(sizeof(cplx) * (size_t)n);
    cplx *a = calloc((size_t)m, sizeof(cplx));
    cplx *b = calloc((size_t)m, sizeof(cplx));
    if (!w || !a || !b) { free(w); free(a); free(b); return -2; }
    for (int64_t j = 0; j < n; ++j) {
        /* reduce j^2 modulo 2n so the angle stays small and exact */
        int64_t jj = (int64_t)(((__int128)j * j) % (2 * n));
        double ang = sign * PI * (double)jj / (double)n;
        w[j] = cos(ang) + I * sin(ang);
    }
    for (int64_t j = 0; j < n; ++j) a[j] = x[j] * w[j];
    b[0] = conj(w[0]);
    for (int64_t j = 1; j < n; ++j) { b[j] = conj(w[j]); b[m - j] = conj(w[j]); }
    fft_radix2(a, m, -1);
    fft_radix2(b, m, -1);
    for (int64_t j = 0; j < m; ++j) a[j] *= b[j];
    fft_radix2(a, m, +1);
    for (int64_t k = 0; k < n; ++k) x[k] = w[k] * a[k] / (double)m;
    free(w); free(a); free(b);
    return 0;
}

/* Forward (inverse=0) or inverse (inverse=1, with 1/n) DFT of one line. */
static int fft_line(cplx *x, int64_t n, int inverse)
{
    int sign = inverse ? +1 : -1;
    int rc = 0;
    if (n == 1) return 0;
    if (is_pow2(n)) fft_radix2(x, n, sign);
    else rc = fft_bluestein(x, n, sign);
    if (inverse) for (int64_t k = 0; k < n; ++k) x[k] /= (double)n;
    return rc;
}

/* x: interleaved (re, im) doubles, length n; transformed in place. */
int orc_fft1(double *x, int64_t n, int inverse)
{
    if (!x || n < 1) return -1;
    return fft_line((cplx *)x, n, inverse);
}

/* Brute-force O(n^2) DFT, out of place. */
int orc_dft1_brute(const double *in, double *out, int64_t n, int inverse)
{
    if (!in || !out || n < 1) return -1;
    const cplx *xi = (const cplx *)in;
    cplx *xo = (cplx *)out;
    int sign = inverse ? +1 : -1;
    for (int64_t k = 0; k < n; ++k) {
        cplx s = 0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t kj = (int64_t)(((__int128)k * j) % n);
            double a = sign * 2.0 * PI * (double)kj / (double)n;
            s += xi[j] * (cos(a) + I * sin(a));
        }
        xo[k] = inverse ? s / (double)n : s;
    }
    return 0;
}

/* ---------------------------------------------------------------- FFT 3D */

/* Transform every line along one axis of a [nz][ny][nx] complex array.
 * stride = distance between consecutive elements of a line, count = lines. */
static int fft_axis(cplx *x, int64_t nz, int64_t ny, int64_t nx, int axis, int inverse)
{
    int64_t n, stride;
    if (axis == 2) { n = nx; stride = 1; }
    else if (axis == 1) { n = ny; stride = nx; }
    else { n = nz; stride = nx * ny; }
    if (n == 1) return 0;
    int64_t lines = nx * ny * nz / n;
    int err = 0;
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * (size_t)n);
        if (!buf) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (int64_t l = 0; l < lines; ++l) {
                /* first element of line l */
                int64_t base;
                if (axis == 2) base = l * nx;
                else if (axis == 1) base = (l / nx) * nx * ny + (l % nx);
                else base = l;
                for (int64_t j = 0; j < n; ++j) buf[j] = x[base + j * stride];
                if (fft_line(buf, n, inverse) != 0) {
#pragma omp atomic write
                    err = -2;
                }
                for (int64_t j = 0; j < n; ++j) x[base + j * stride] = buf[j];
            }
            free(buf);
        }
    }
    return err;
}

static int fft3(cplx *x, int64_t nz, int64_t ny, int64_t nx, int inverse)
{
    int rc = 0;
    for (int axis = 2; axis >= 0 && rc == 0; --axis)
        rc = fft_axis(x, nz, ny, nx, axis, inverse);
    return rc;
}

int orc_fft3(double *x, int64_t nz, int64_t ny, int64_t nx, int inverse)
{
    if (!x || nz < 1 || ny < 1 || nx < 1) return -1;
    return fft3((cplx *)x, nz, ny, nx, inverse);
}

/* ------------------------------------------------------- PSF and helpers */

static int64_t wrap(int64_t i, int64_t n) { int64_t r = i % n; return r < 0 ? r + n : r; }

/* h0(z,y,x) = p((z + nz/2) mod nz, (y + ny/2) mod ny, (x + nx/2) mod nx):
 * moves the PSF peak from floor(n/2) to the origin. */
static void center_to_origin(const double *p, double *h0, int64_t nz, int64_t ny, int64_t nx)
{
    int64_t cz = nz / 2, cy = ny / 2, cx = nx / 2;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                h0[(z * ny + y) * nx + x] =
                    p[(wrap(z + cz, nz) * ny + wrap(y + cy, ny)) * nx + wrap(x + cx, nx)];
}

/* inverse map: p(x) = h0(x - c) */
static void origin_to_center(const double *h0, double *p, int64_t nz, int64_t ny, int64_t nx)
{
    int64_t cz = nz / 2, cy = ny / 2, cx = nx / 2;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                p[(wrap(z + cz, nz) * ny + wrap(y + cy, ny)) * nx + wrap(x + cx, nx)] =
                    h0[(z * ny + y) * nx + x];
}

int orc_center_to_origin(const double *p, double *h0, int64_t nz, int64_t ny, int64_t nx)
{
    if (!p || !h0 || nz < 1 || ny < 1 || nx < 1) return -1;
    center_to_origin(p, h0, nz, ny, nx);
    return 0;
}

/* Direct circular convolution, O(V^2): out(y) = sum_x h0(x) u(y - x). */
int orc_conv3_direct(const double *h0, const double *u, double *out,
                     int64_t nz, int64_t ny, int64_t nx)
{
    if (!h0 || !u || !out || nz < 1 || ny < 1 || nx < 1) return -1;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double s = 0.0;
                for (int64_t a = 0; a < nz; ++a)
                    for (int64_t b = 0; b < ny; ++b)
                        for (int64_t c = 0; c < nx; ++c)
                            s += h0[(a * ny + b) * nx + c] *
                                 u[(wrap(z - a, nz) * ny + wrap(y - b, ny)) * nx + wrap(x - c, nx)];
                out[(z * ny + y) * nx + x] = s;
            }
    return 0;
}

/* ------------------------------------------------------------ RL oracle */

/* Spectrum of the origin-centred PSF: H = DFT3(h0). Hs: interleaved complex, V. */
int orc_psf_spectrum(const double *psf, double *Hs, int64_t nz, int64_t ny, int64_t nx)
{
    if (!psf || !Hs || nz < 1 || ny < 1 || nx < 1) return -1;
    int64_t V = nz * ny * nx;
    double *h0 = malloc(sizeof(double) * (size_t)V);
    if (!h0) return -2;
    center_to_origin(psf, h0, nz, ny, nx);
    cplx *H = (cplx *)Hs;
    for (int64_t i = 0; i < V; ++i) H[i] = h0[i];
    free(h0);
    return fft3(H, nz, ny, nx, 0);
}

/* out = Re IDFT3(M(H) * DFT3(in)), M = identity (conjugate=0) or conj (=1).
 * work: V complex scratch. */
static int spectral_filter(const cplx *H, const double *in, double *out, cplx *work,
                           int64_t nz, int64_t ny, int64_t nx, int conjugate)
{
    int64_t V = nz * ny * nx;
    for (int64_t i = 0; i < V; ++i) work[i] = in[i];
    int rc = fft3(work, nz, ny, nx, 0);
    if (rc) return rc;
    for (int64_t i = 0; i < V; ++i) work[i] *= conjugate ? conj(H[i]) : H[i];
    rc = fft3(work, nz, ny, nx, 1);
    if (rc) return rc;
    for (int64_t i = 0; i < V; ++i) out[i] = creal(work[i]);
    return 0;
}

/* Blur with the PSF (b = h * u, circular) -- the forward model, given H. */
int orc_convolve(const double *Hs, const double *u, double *b, int64_t nz, int64_t ny, int64_t nx,
                 int conjugate)
{
    if (!Hs || !u || !b || nz < 1 || ny < 1 || nx < 1) return -1;
    int64_t V = nz * ny * nx;
    cplx *work = malloc(sizeof(cplx) * (size_t)V);
    if (!work) return -2;
    int rc = spectral_filter((const cplx *)Hs, u, b, work, nz, ny, nx, conjugate);
    free(work);
    return rc;
}

double orc_initial_value(const double *d, int64_t V, double eps)
{
    double s = 0.0;
    for (int64_t i = 0; i < V; ++i) s += d[i];
    double m = s / (double)V;
    return m > eps ? m : eps;
}

/* One RL iteration from u (given H).  Writes u_next and, if non-NULL, the
 * intermediates b = h*u, r = d/max(b,eps), q = h (flipped) * r. */
int orc_rl_iterate(const double *Hs, const double *d, const double *u, double eps,
                   int64_t nz, int64_t ny, int64_t nx,
                   double *u_next, double *b_out, double *r_out, double *q_out)
{
    if (!Hs || !d || !u || !u_next || nz < 1 || ny < 1 || nx < 1) return -1;
    int64_t V = nz * ny * nx;
    cplx *work = malloc(sizeof(cplx) * (size_t)V);
    double *b = malloc(sizeof(double) * (size_t)V);
    double *r = malloc(sizeof(double) * (size_t)V);
    double *q = malloc(sizeof(double) * (size_t)V);
    int rc = -2;
    if (work && b && r && q) {
        const cplx *H = (const cplx *)Hs;
        rc = spectral_filter(H, u, b, work, nz, ny, nx, 0);           /* forward conv */
        if (!rc) {
            for (int64_t i = 0; i < V; ++i) {                           /* ratio */
                double c = b[i] > eps ? b[i] : eps;
                r[i] = d[i] / c;
            }
            rc = spectral_filter(H, r, q, work, nz, ny, nx, 1);        /* back-conv, flipped PSF */
        }
        if (!rc) {
            for (int64_t i = 0; i < V; ++i) u_next[i] = u[i] * q[i];   /* multiplicative update */
            if (b_out) memcpy(b_out, b, sizeof(double) * (size_t)V);
            if (r_out) memcpy(r_out, r, sizeof(double) * (size_t)V);
            if (q_out) memcpy(q_out, q, sizeof(double) * (size_t)V);
        }
    }
    free(work); free(b); free(r); free(q);
    return rc;
}

/* Full RL: n_iter iterations from u0 = max(mean(d), eps). */
int orc_rl(const double *d, const double *psf, int64_t nz, int64_t ny, int64_t nx,
           int n_iter, double eps, double *out)
{
    if (!d || !psf || !out || nz < 1 || ny < 1 || nx < 1 || n_iter < 0 || !(eps > 0)) return -1;
    int64_t V = nz * ny * nx;
    double *Hs = malloc(sizeof(double) * 2 * (size_t)V);
    double *u = malloc(sizeof(double) * (size_t)V);
    if (!Hs || !u) { free(Hs); free(u); return -2; }
    int rc = orc_psf_spectrum(psf, Hs, nz, ny, nx);
    double u0 = orc_initial_value(d, V, eps);
    for (int64_t i = 0; i < V; ++i) u[i] = u0;
    for (int k = 0; k < n_iter && !rc; ++k)
        rc = orc_rl_iterate(Hs, d, u, eps, nz, ny, nx, u, NULL, NULL, NULL);
    if (!rc) memcpy(out, u, sizeof(double) * (size_t)V);
    free(Hs); free(u);
    return rc;
}

/* RL with automatic stopping (the paper's Section 4 ends the iteration once the gain in
 * image quality from one iteration to the next drops under a threshold).
 * Reading: the improvement of iteration k is the relative change of the estimate,
 *   delta_k = ||u_{k+1} - u_k||_2 / ||u_k||_2,
 * checked after every check_every-th iteration (and after the last one); the run stops
 * at the first check with delta_k < tol.  Writes the estimate, the number of iterations
 * done and delta_0 .. delta_{done-1} (history may be NULL). */
int orc_rl_auto(const double *d, const double *psf, int64_t nz, int64_t ny, int64_t nx, int max_iter,
                double eps, double tol, int check_every, double *out, int *n_done, double *history)
{
    if (!d || !psf || !out || !n_done || nz < 1 || ny < 1 || nx < 1 || max_iter < 1 || check_every < 1 ||
        !(eps > 0))
        return -1;
    int64_t V = nz * ny * nx;
    double *Hs = malloc(sizeof(double) * 2 * (size_t)V);
    double *u = malloc(sizeof(double) * (size_t)V);
    double *un = malloc(sizeof(double) * (size_t)V);
    if (!Hs || !u || !un) { free(Hs); free(u); free(un); return -2; }
    int rc = orc_psf_spectrum(psf, Hs, nz, ny, nx);
    double u0 = orc_initial_value(d, V, eps);
    for (int64_t i = 0; i < V; ++i) u[i] = u0;
    int k = 0;
    while (!rc && k < max_iter) {
        rc = orc_rl_iterate(Hs, d, u, eps, nz, ny, nx, un, NULL, NULL, NULL);
        if (rc) break;
        double num = 0.0, den = 0.0;
        for (int64_t i = 0; i < V; ++i) {
            double e = un[i] - u[i];
            num += e * e;
            den += u[i] * u[i];
        }
        double delta = den > 0 ? sqrt(num / den) : 0.0;
        if (history) history[k] = delta;
        memcpy(u, un, sizeof(double) * (size_t)V);
        ++k;
        if ((k % check_every == 0 || k == max_iter) && delta < tol) break;
    }
    if (!rc) {
        memcpy(out, u, sizeof(double) * (size_t)V);
        *n_done = k;
    }
    free(Hs); free(u); free(un);
    return rc;
}

/* Linear ("same"-mode) boundaries: the image lives on its own box only, the PSF (dims
 * kz, ky, kx, peak at floor(k/2)) can be smaller, and the convolution sees zeros outside the
 * box instead of wrapping around:
 *   b(x) = sum_t p(t + c) u(x - t),  c = floor(k/2), u = 0 outside [0, n)   ("same" output),
 *   q(x) = sum_t p(t + c) r(x + t),  r = 0 outside [0, n)                    (its adjoint).
 * Computed by FFT on the padded box M = n + k - 1 per axis, where circular convolution of
 * the zero-padded arrays equals the linear one; the PSF is placed with its peak at the
 * origin of the padded box.  The RL iteration is unchanged otherwise (x_0 = max(mean(d),
 * eps) on the image box, r = d / max(b, eps)).  This is the zero-padded reading of the
 * survey's "next" row; the paper's own workload uses a PSF of the image's size. */
static void same_embed_psf(const double *psf, int64_t kz, int64_t ky, int64_t kx, double *h0, int64_t mz,
                           int64_t my, int64_t mx)
{
    memset(h0, 0, sizeof(double) * (size_t)(mz * my * mx));
    for (int64_t z = 0; z < kz; ++z)
        for (int64_t y = 0; y < ky; ++y)
            for (int64_t x = 0; x < kx; ++x)
                h0[(wrap(z - kz / 2, mz) * my + wrap(y - ky / 2, my)) * mx + wrap(x - kx / 2, mx)] =
                    psf[(z * ky + y) * kx + x];
}

struct same_geom {
    int64_t nz, ny, nx, mz, my, mx;
};

/* out (image box) = crop(Re IDFT3(M(H) DFT3(pad(in)))), M = identity or conj */
static int same_filter(const struct same_geom *g, const cplx *H, const double *in, double *out, cplx *work,
                       int conjugate)
{
    int64_t Vm = g->mz * g->my * g->mx;
    for (int64_t i = 0; i < Vm; ++i) work[i] = 0.0;
    for (int64_t z = 0; z < g->nz; ++z)
        for (int64_t y = 0; y < g->ny; ++y)
            for (int64_t x = 0; x < g->nx; ++x)
                work[(z * g->my + y) * g->mx + x] = in[(z * g->ny + y) * g->nx + x];
    int rc = fft3(work, g->mz, g->my, g->mx, 0);
    if (rc) return rc;
    for (int64_t i = 0; i < Vm; ++i) work[i] *= conjugate ? conj(H[i]) : H[i];
    rc = fft3(work, g->mz, g->my, g->mx, 1);
    if (rc) return rc;
    for (int64_t z = 0; z < g->nz; ++z)
        for (int64_t y = 0; y < g->ny; ++y)
            for (int64_t x = 0; x < g->nx; ++x)
                out[(z * g->ny + y) * g->nx + x] = creal(work[(z * g->my + y) * g->mx + x]);
    return 0;
}

static int same_setup(const double *psf, const int64_t n[3], const int64_t k[3], struct same_geom *g, cplx **H,
                      cplx **work)
{
    g->nz = n[0]; g->ny = n[1]; g->nx = n[2];
    g->mz = n[0] + k[0] - 1; g->my = n[1] + k[1] - 1; g->mx = n[2] + k[2] - 1;
    int64_t Vm = g->mz * g->my * g->mx;
    double *h0 = malloc(sizeof(double) * (size_t)Vm);
    *H = malloc(sizeof(cplx) * (size_t)Vm);
    *work = malloc(sizeof(cplx) * (size_t)Vm);
    if (!h0 || !*H || !*work) { free(h0); free(*H); free(*work); *H = *work = NULL; return -2; }
    same_embed_psf(psf, k[0], k[1], k[2], h0, g->mz, g->my, g->mx);
    for (int64_t i = 0; i < Vm; ++i) (*H)[i] = h0[i];
    free(h0);
    return fft3(*H, g->mz, g->my, g->mx, 0);
}

/* b = same-mode convolution of u (image box n) with psf (box k); flipped: its adjoint. */
int orc_conv_same(const double *psf, const double *u, double *b, int64_t nz, int64_t ny, int64_t nx, int64_t kz,
                  int64_t ky, int64_t kx, int flipped)
{
    if (!psf || !u || !b || nz < 1 || ny < 1 || nx < 1 || kz < 1 || ky < 1 || kx < 1) return -1;
    const int64_t n[3] = {nz, ny, nx}, k[3] = {kz, ky, kx};
    struct same_geom g;
    cplx *H, *work;
    int rc = same_setup(psf, n, k, &g, &H, &work);
    if (!rc) rc = same_filter(&g, H, u, b, work, flipped);
    free(H); free(work);
    return rc;
}

/* RL with linear boundaries: n_iter iterations from x_0 = max(mean(d), eps). */
int orc_rl_same(const double *d, const double *psf, int64_t nz, int64_t ny, int64_t nx, int64_t kz, int64_t ky,
                int64_t kx, int n_iter, double eps, double *out)
{
    if (!d || !psf || !out || nz < 1 || ny < 1 || nx < 1 || kz < 1 || ky < 1 || kx < 1 || n_iter < 0 ||
        !(eps > 0))
        return -1;
    const int64_t n[3] = {nz, ny, nx}, k[3] = {kz, ky, kx};
    int64_t V = nz * ny * nx;
    struct same_geom g;
    cplx *H, *work;
    int rc = same_setup(psf, n, k, &g, &H, &work);
    double *u = malloc(sizeof(double) * (size_t)V), *b = malloc(sizeof(double) * (size_t)V);
    double *q = malloc(sizeof(double) * (size_t)V);
    if (!u || !b || !q) rc = rc ? rc : -2;
    if (!rc) {
        double u0 = orc_initial_value(d, V, eps);
        for (int64_t i = 0; i < V; ++i) u[i] = u0;
        for (int it = 0; it < n_iter && !rc; ++it) {
            rc = same_filter(&g, H, u, b, work, 0);                         /* forward conv */
            if (rc) break;
            for (int64_t i = 0; i < V; ++i) b[i] = d[i] / (b[i] > eps ? b[i] : eps);   /* ratio */
            rc = same_filter(&g, H, b, q, work, 1);                          /* adjoint */
            if (rc) break;
            for (int64_t i = 0; i < V; ++i) u[i] *= q[i];                     /* update */
        }
        if (!rc) memcpy(out, u, sizeof(double) * (size_t)V);
    }
    free(H); free(work); free(u); free(b); free(q);
    return rc;
}

/* Quality metrics for metric-guided stopping (the paper's Section 4 stops RL when the
 * improvement of an image-quality measure between consecutive iterations falls under a
 * threshold; Section 3 lists scale-invariant PSNR among its metrics).
 *   Poisson negative log-likelihood (up to a constant): NLL(u) = sum (c - d ln c),
 *     c = max(h * u, eps), the objective RL maximises the likelihood of.
 *   Scale-invariant PSNR of x against a reference y (Weigert et al. 2018): the affine map
 *     a x + b closest to y in least squares, then 20 log10(range(y) / rmse),
 *     range(y) = max y - min y, rmse = sqrt(min_{a,b} mean((a x + b - y)^2)).  The
 *     minimum has the closed form var(y) - cov(x, y)^2 / var(x) (population moments);
 *     var(x) = 0 leaves var(y).  A zero rmse gives +inf, a zero range -inf. */
double orc_poisson_nll(const double *b, const double *d, int64_t V, double eps)
{
    double s = 0.0;
    for (int64_t i = 0; i < V; ++i) {
        double c = b[i] > eps ? b[i] : eps;
        s += c - d[i] * log(c);
    }
    return s;
}

double orc_psnr_si(const double *x, const double *y, int64_t V)
{
    double mx = 0.0, my = 0.0, ymin = y[0], ymax = y[0];
    for (int64_t i = 0; i < V; ++i) {
        mx += x[i];
        my += y[i];
        if (y[i] < ymin) ymin = y[i];
        if (y[i] > ymax) ymax = y[i];
    }
    mx /= (double)V;
    my /= (double)V;
    double vx = 0.0, vy = 0.0, cxy = 0.0;
    for (int64_t i = 0; i < V; ++i) {
        double ex = x[i] - mx, ey = y[i] - my;
        vx += ex * ex;
        vy += ey * ey;
        cxy += ex * ey;
    }
    vx /= (double)V;
    vy /= (double)V;
    cxy /= (double)V;
    double mse = vx > 0.0 ? vy - cxy * cxy / vx : vy;
    if (mse < 0.0) mse = 0.0;
    return 20.0 * log10((ymax - ymin) / sqrt(mse));
}

/* RL with metric-guided stopping.  After iteration k (which made u_{k+1}) the history
 * row k holds (delta_k, NLL(u_k), PSNR_si(u_{k+1}, ref)); NAN for the PSNR without a
 * reference.  NLL(u_k) comes from iteration k's forward convolution.  At every check
 * (k+1 a multiple of check_every, or k+1 = max_iter) the run stops when the chosen
 * measure's improvement is under tol:
 *   metric 0: delta_k < tol (relative change of the estimate);
 *   metric 1: k >= 1 and (NLL(u_{k-1}) - NLL(u_k)) / |NLL(u_k)| < tol;
 *   metric 2: k >= 1 and PSNR_k - PSNR_{k-1} < tol (decibels; needs ref).
 * out: the last estimate u_{n_done}.
 *
 * monitor_run is that loop for any RL step: step(ctx, u, un, b) makes the next estimate
 * un and leaves the forward blur b = h * u (before the clamp) for the likelihood. */
typedef int (*monitor_step)(void *ctx, const double *u, double *un, double *b);

static int monitor_run(monitor_step step, void *ctx, const double *d, const double *ref, int64_t V, int max_iter,
                       double eps, int metric, double tol, int check_every, double *out, int *n_done, double *hist)
{
    double *u = malloc(sizeof(double) * (size_t)V);
    double *un = malloc(sizeof(double) * (size_t)V);
    double *b = malloc(sizeof(double) * (size_t)V);
    if (!u || !un || !b) { free(u); free(un); free(b); return -2; }
    int rc = 0;
    double u0 = orc_initial_value(d, V, eps);
    for (int64_t i = 0; i < V; ++i) u[i] = u0;
    int k = 0;
    while (!rc && k < max_iter) {
        rc = step(ctx, u, un, b);
        if (rc) break;
        double num = 0.0, den = 0.0;
        for (int64_t i = 0; i < V; ++i) {
            double e = un[i] - u[i];
            num += e * e;
            den += u[i] * u[i];
        }
        double *h = hist + 3 * (size_t)k;
        h[0] = den > 0 ? sqrt(num / den) : 0.0;
        h[1] = orc_poisson_nll(b, d, V, eps);
        h[2] = ref ? orc_psnr_si(un, ref, V) : NAN;
        memcpy(u, un, sizeof(double) * (size_t)V);
        ++k;
        if (k % check_every == 0 || k == max_iter) {
            int stop = 0;
            if (metric == 0) stop = h[0] < tol;
            else if (k >= 2 && metric == 1) stop = (h[-2] - h[1]) / fabs(h[1]) < tol;
            else if (k >= 2 && metric == 2) stop = h[2] - h[-1] < tol;
            if (stop) break;
        }
    }
    if (!rc) {
        memcpy(out, u, sizeof(double) * (size_t)V);
        *n_done = k;
    }
    free(u); free(un); free(b);
    return rc;
}

struct circ_monitor {
    const double *Hs, *d;
    double eps;
    int64_t nz, ny, nx;
};

static int circ_monitor_step(void *ctx, const double *u, double *un, double *b)
{
    const struct circ_monitor *c = ctx;
    return orc_rl_iterate(c->Hs, c->d, u, c->eps, c->nz, c->ny, c->nx, un, b, NULL, NULL);
}

int orc_rl_monitor(const double *d, const double *psf, const double *ref, int64_t nz, int64_t ny, int64_t nx,
                   int max_iter, double eps, int metric, double tol, int check_every, double *out, int *n_done,
                   double *hist)
{
    if (!d || !psf || !out || !n_done || !hist || nz < 1 || ny < 1 || nx < 1 || max_iter < 1 ||
        check_every < 1 || !(eps > 0) || metric < 0 || metric > 2 || (metric == 2 && !ref))
        return -1;
    int64_t V = nz * ny * nx;
    double *Hs = malloc(sizeof(double) * 2 * (size_t)V);
    if (!Hs) return -2;
    int rc = orc_psf_spectrum(psf, Hs, nz, ny, nx);
    struct circ_monitor c = {Hs, d, eps, nz, ny, nx};
    if (!rc) rc = monitor_run(circ_monitor_step, &c, d, ref, V, max_iter, eps, metric, tol, check_every, out, n_done,
                              hist);
    free(Hs);
    return rc;
}

/* The same monitored run with linear ("same"-mode) boundaries: the blur, the ratio, the
 * adjoint and the update of orc_rl_same; every measure is taken over the image box. */
struct same_monitor {
    const struct same_geom *g;
    const cplx *H;
    cplx *work;
    const double *d;
    double *r, *q;
    double eps;
    int64_t V;
};

static int same_monitor_step(void *ctx, const double *u, double *un, double *b)
{
    const struct same_monitor *c = ctx;
    int rc = same_filter(c->g, c->H, u, b, c->work, 0);                          /* forward conv */
    if (rc) return rc;
    for (int64_t i = 0; i < c->V; ++i) c->r[i] = c->d[i] / (b[i] > c->eps ? b[i] : c->eps);   /* ratio */
    rc = same_filter(c->g, c->H, c->r, c->q, c->work, 1);                        /* adjoint */
    if (rc) return rc;
    for (int64_t i = 0; i < c->V; ++i) un[i] = u[i] * c->q[i];                   /* update */
    return 0;
}

int orc_rl_monitor_same(const double *d, const double *psf, const double *ref, int64_t nz, int64_t ny, int64_t nx,
                        int64_t kz, int64_t ky, int64_t kx, int max_iter, double eps, int metric, double tol,
                        int check_every, double *out, int *n_done, double *hist)
{
    if (!d || !psf || !out || !n_done || !hist || nz < 1 || ny < 1 || nx < 1 || kz < 1 || ky < 1 || kx < 1 ||
        max_iter < 1 || check_every < 1 || !(eps > 0) || metric < 0 || metric > 2 || (metric == 2 && !ref))
        return -1;
    const int64_t n[3] = {nz, ny, nx}, k[3] = {kz, ky, kx};
    int64_t V = nz * ny * nx;
    struct same_geom g;
    cplx *H, *work;
    int rc = same_setup(psf, n, k, &g, &H, &work);
    double *r = malloc(sizeof(double) * (size_t)V), *q = malloc(sizeof(double) * (size_t)V);
    if (!r || !q) rc = rc ? rc : -2;
    struct same_monitor c = {&g, H, work, d, r, q, eps, V};
    if (!rc) rc = monitor_run(same_monitor_step, &c, d, ref, V, max_iter, eps, metric, tol, check_every, out, n_done,
                              hist);
    free(H); free(work); free(r); free(q);
    return rc;
}

/* Accelerated Richardson-Lucy.  The paper (Section 2, on the pycudadecon plugin) cites
 * the acceleration of Biggs and Andrews ("Acceleration of iterative image restoration
 * algorithms", Applied Optics 36(8), 1997).  Their first-order vector extrapolation
 * runs the fixed-point step psi (one RL iteration) from a predicted point instead of the
 * last estimate:
 *   y_k     = max(x_k + alpha_k (x_k - x_{k-1}), 0)      prediction along the last move
 *   x_{k+1} = psi(y_k)                                      one RL iteration from y_k
 *   g_k     = x_{k+1} - y_k                                 the change psi made
 *   alpha_k = <g_{k-1}, g_{k-2}> / <g_{k-2}, g_{k-2}>, clamped to [0, 1]; alpha_0 =
 *             alpha_1 = 0 (no two changes yet) and alpha_k = 0 when the denominator is 0.
 * Readings (the paper gives no formula): negative predicted values are set to 0 (RL
 * needs a non-negative point); the clamp of alpha to [0, 1] keeps the prediction between
 * the last estimate and one full step beyond it.
 *
 * accel_run is the extrapolation alone, for any step psi; orc_rl_accel uses the RL step,
 * orc_accel_linear a linear step psi(y) = xs + lambda (y - xs) (per element), whose
 * iterates have closed forms the tests check. */
typedef int (*step_fn)(void *ctx, const double *y, double *x_next);

static int accel_run(step_fn psi, void *ctx, int64_t V, int n_iter, const double *x0, double *out,
                     double *alpha_hist)
{
    double *x = malloc(sizeof(double) * (size_t)V);     /* x_k */
    double *xp = malloc(sizeof(double) * (size_t)V);    /* x_{k-1} */
    double *xn = malloc(sizeof(double) * (size_t)V);    /* x_{k+1} */
    double *y = malloc(sizeof(double) * (size_t)V);     /* y_k */
    double *g1 = malloc(sizeof(double) * (size_t)V);    /* g_{k-1} */
    double *g2 = malloc(sizeof(double) * (size_t)V);    /* g_{k-2} */
    int rc = -2;
    if (x && xp && xn && y && g1 && g2) {
        rc = 0;
        memcpy(x, x0, sizeof(double) * (size_t)V);
        memcpy(xp, x0, sizeof(double) * (size_t)V);
        for (int k = 0; k < n_iter && !rc; ++k) {
            double alpha = 0.0;
            if (k >= 2) {
                double num = 0.0, den = 0.0;
                for (int64_t i = 0; i < V; ++i) {
                    num += g1[i] * g2[i];
                    den += g2[i] * g2[i];
                }
                alpha = den > 0.0 ? num / den : 0.0;
                if (alpha < 0.0) alpha = 0.0;
                if (alpha > 1.0) alpha = 1.0;
            }
            if (alpha_hist) alpha_hist[k] = alpha;
            for (int64_t i = 0; i < V; ++i) {
                double v = x[i] + alpha * (x[i] - xp[i]);
                y[i] = v > 0.0 ? v : 0.0;
            }
            rc = psi(ctx, y, xn);
            if (rc) break;
            for (int64_t i = 0; i < V; ++i) {
                g2[i] = g1[i];
                g1[i] = xn[i] - y[i];
                xp[i] = x[i];
                x[i] = xn[i];
            }
        }
        if (!rc) memcpy(out, x, sizeof(double) * (size_t)V);
    }
    free(x); free(xp); free(xn); free(y); free(g1); free(g2);
    return rc;
}

struct rl_step_ctx {
    const double *Hs, *d;
    double eps;
    int64_t nz, ny, nx;
};

static int rl_step(void *ctx, const double *y, double *x_next)
{
    const struct rl_step_ctx *c = ctx;
    return orc_rl_iterate(c->Hs, c->d, y, c->eps, c->nz, c->ny, c->nx, x_next, NULL, NULL, NULL);
}

/* Accelerated RL: n_iter steps from x_0 = max(mean(d), eps); alpha_hist (may be NULL)
 * receives alpha_0 .. alpha_{n_iter-1}. */
int orc_rl_accel(const double *d, const double *psf, int64_t nz, int64_t ny, int64_t nx, int n_iter,
                 double eps, double *out, double *alpha_hist)
{
    if (!d || !psf || !out || nz < 1 || ny < 1 || nx < 1 || n_iter < 0 || !(eps > 0)) return -1;
    int64_t V = nz * ny * nx;
    double *Hs = malloc(sizeof(double) * 2 * (size_t)V);
    double *x0 = malloc(sizeof(double) * (size_t)V);
    if (!Hs || !x0) { free(Hs); free(x0); return -2; }
    int rc = orc_psf_spectrum(psf, Hs, nz, ny, nx);
    double u0 = orc_initial_value(d, V, eps);
    for (int64_t i = 0; i < V; ++i) x0[i] = u0;
    struct rl_step_ctx c = {Hs, d, eps, nz, ny, nx};
    if (!rc) rc = accel_run(rl_step, &c, V, n_iter, x0, out, alpha_hist);
    free(Hs); free(x0);
    return rc;
}

struct lin_step_ctx {
    const double *xs, *lambda;
    int64_t V;
};

static int lin_step(void *ctx, const double *y, double *x_next)
{
    const struct lin_step_ctx *c = ctx;
    for (int64_t i = 0; i < c->V; ++i) x_next[i] = c->xs[i] + c->lambda[i] * (y[i] - c->xs[i]);
    return 0;
}

/* The extrapolation with the linear step psi(y) = xs + lambda (y - xs), from x0. */
int orc_accel_linear(int64_t V, int n_iter, const double *xs, const double *lambda, const double *x0,
                     double *out, double *alpha_hist)
{
    if (V < 1 || n_iter < 0 || !xs || !lambda || !x0 || !out) return -1;
    struct lin_step_ctx c = {xs, lambda, V};
    return accel_run(lin_step, &c, V, n_iter, x0, out, alpha_hist);
}

/* Accelerated RL with linear boundaries: the same extrapolation, each step a same-mode
 * RL iteration. */
struct same_step_ctx {
    const struct same_geom *g;
    const cplx *H;
    cplx *work;
    const double *d;
    double eps;
    double *b, *q;
};

static int same_rl_step(void *ctx, const double *y, double *x_next)
{
    const struct same_step_ctx *c = ctx;
    const int64_t V = c->g->nz * c->g->ny * c->g->nx;
    int rc = same_filter(c->g, c->H, y, c->b, c->work, 0);
    if (rc) return rc;
    for (int64_t i = 0; i < V; ++i) c->b[i] = c->d[i] / (c->b[i] > c->eps ? c->b[i] : c->eps);
    rc = same_filter(c->g, c->H, c->b, c->q, c->work, 1);
    if (rc) return rc;
    for (int64_t i = 0; i < V; ++i) x_next[i] = y[i] * c->q[i];
    return 0;
}

int orc_rl_accel_same(const double *d, const double *psf, int64_t nz, int64_t ny, int64_t nx, int64_t kz, int64_t ky,
                      int64_t kx, int n_iter, double eps, double *out, double *alpha_hist)
{
    if (!d || !psf || !out || nz < 1 || ny < 1 || nx < 1 || kz < 1 || ky < 1 || kx < 1 || n_iter < 0 ||
        !(eps > 0))
        return -1;
    const int64_t n[3] = {nz, ny, nx}, k[3] = {kz, ky, kx};
    int64_t V = nz * ny * nx;
    struct same_geom g;
    cplx *H, *work;
    int rc = same_setup(psf, n, k, &g, &H, &work);
    double *x0 = malloc(sizeof(double) * (size_t)V), *b = malloc(sizeof(double) * (size_t)V);
    double *q = malloc(sizeof(double) * (size_t)V);
    if (!x0 || !b || !q) rc = rc ? rc : -2;
    if (!rc) {
        double u0 = orc_initial_value(d, V, eps);
        for (int64_t i = 0; i < V; ++i) x0[i] = u0;
        struct same_step_ctx c = {&g, H, work, d, eps, b, q};
        rc = accel_run(same_rl_step, &c, V, n_iter, x0, out, alpha_hist);
    }
    free(H); free(work); free(x0); free(b); free(q);
    return rc;
}

/* Fourier Shell Correlation of two volumes (the paper's FRC/FSC resolution metric,
 * Section 3 "custom algorithms" and Section 4 "Evaluation metrics"):
 *   FSC(s) = Re sum_{k in s} A(k) conj B(k) / sqrt(sum_{k in s} |A(k)|^2 sum_{k in s} |B(k)|^2),
 * A, B the full 3D DFTs.  Shell s = floor(2 * n_shells * rho) for the normalised radius
 * rho = |(fz, fy, fx)|, f = signed frequency / n (cycles per voxel), evaluated exactly in
 * integers (rho^2 is rational); rho >= 1/2 (beyond Nyquist) is left out.  num, da, db: the three sums per shell (may be NULL); fsc: the
 * ratio (0 for an empty shell). */
int orc_fsc(const double *a, const double *b, int64_t nz, int64_t ny, int64_t nx, int n_shells, double *fsc,
            double *num, double *da, double *db)
{
    if (!a || !b || !fsc || nz < 1 || ny < 1 || nx < 1 || n_shells < 1) return -1;
    int64_t V = nz * ny * nx;
    cplx *A = malloc(sizeof(cplx) * (size_t)V), *B = malloc(sizeof(cplx) * (size_t)V);
    double *sn = calloc((size_t)n_shells, sizeof(double)), *sa = calloc((size_t)n_shells, sizeof(double));
    double *sb = calloc((size_t)n_shells, sizeof(double));
    int rc = -2;
    if (A && B && sn && sa && sb) {
        for (int64_t i = 0; i < V; ++i) { A[i] = a[i]; B[i] = b[i]; }
        rc = fft3(A, nz, ny, nx, 0);
        if (!rc) rc = fft3(B, nz, ny, nx, 0);
        if (!rc) {
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        /* signed frequency index in (-n/2, n/2]; rho^2 = num / den exactly */
                        __int128 kz = 2 * z > nz ? z - nz : z, ky = 2 * y > ny ? y - ny : y;
                        __int128 kx = 2 * x > nx ? x - nx : x;
                        __int128 den = (__int128)nz * nz * ny * ny * nx * nx;
                        __int128 rn = kz * kz * ny * ny * nx * nx + ky * ky * nz * nz * nx * nx +
                                      kx * kx * nz * nz * ny * ny;
                        /* s = floor(2 S rho) = isqrt(floor(4 S^2 num / den)) */
                        __int128 q = (__int128)4 * n_shells * n_shells * rn / den;
                        int64_t s = (int64_t)floor(sqrt((double)q));
                        while ((__int128)s * s > q) --s;
                        while ((__int128)(s + 1) * (s + 1) <= q) ++s;
                        if (s >= n_shells) continue; /* rho >= 1/2 */
                        int64_t i = (z * ny + y) * nx + x;
                        sn[s] += creal(A[i] * conj(B[i]));
                        sa[s] += creal(A[i] * conj(A[i]));
                        sb[s] += creal(B[i] * conj(B[i]));
                    }
            for (int s = 0; s < n_shells; ++s) {
                double den = sqrt(sa[s] * sb[s]);
                fsc[s] = den > 0 ? sn[s] / den : 0.0;
                if (num) num[s] = sn[s];
                if (da) da[s] = sa[s];
                if (db) db[s] = sb[s];
            }
        }
    }
    free(A); free(B); free(sn); free(sa); free(sb);
    return rc;
}

/* Single-image FSC (the paper's resolution metric computed from one image, Section 4,
 * "Evaluation metrics", citing Koho et al. 2019): the volume (even dims) splits into its
 * eight parity sub-volumes s_abc(z, y, x) = d(2z + a, 2y + b, 2x + c); the FSC of each of
 * the four pairs of opposite parity (abc with (1-a)(1-b)(1-c)) is taken on the half grid
 * and the four curves are averaged shell by shell.  Readings: plain mean of the four
 * pairs; no correction for the half-voxel diagonal shift between a pair; shells are
 * those of the half grid (its Nyquist is half the full grid's).  out: n_shells values. */
int orc_fsc_split(const double *d, int64_t nz, int64_t ny, int64_t nx, int n_shells, double *out)
{
    if (!d || !out || nz < 2 || ny < 2 || nx < 2 || nz % 2 || ny % 2 || nx % 2 || n_shells < 1) return -1;
    const int64_t hz = nz / 2, hy = ny / 2, hx = nx / 2, H = hz * hy * hx;
    double *a = malloc(sizeof(double) * (size_t)H), *b = malloc(sizeof(double) * (size_t)H);
    double *f = malloc(sizeof(double) * (size_t)n_shells);
    int rc = (a && b && f) ? 0 : -2;
    for (int s = 0; s < n_shells; ++s) out[s] = 0.0;
    for (int pair = 0; pair < 4 && !rc; ++pair) {
        /* one half has z-parity 0 and (y, x) parities from the pair index; the other the
         * complementary parities */
        const int p0[3] = {0, (pair >> 1) & 1, pair & 1};
        for (int64_t z = 0; z < hz; ++z)
            for (int64_t y = 0; y < hy; ++y)
                for (int64_t x = 0; x < hx; ++x) {
                    const int64_t i = (z * hy + y) * hx + x;
                    a[i] = d[((2 * z + p0[0]) * ny + 2 * y + p0[1]) * nx + 2 * x + p0[2]];
                    b[i] = d[((2 * z + 1 - p0[0]) * ny + 2 * y + 1 - p0[1]) * nx + 2 * x + 1 - p0[2]];
                }
        rc = orc_fsc(a, b, hz, hy, hx, n_shells, f, NULL, NULL, NULL);
        for (int s = 0; s < n_shells && !rc; ++s) out[s] += 0.25 * f[s];
    }
    free(a); free(b); free(f);
    return rc;
}

/* Reverse mode through n_iter RL iterations.
 * g_out = dL/du_K.  Writes grad_d = dL/dd (through the ratio at every
 * iteration and through u0 = max(mean(d), eps)) and grad_psf = dL/dp for the
 * centred PSF p.  Either output may be NULL. */
int orc_rl_grad(const double *d, const double *psf, int64_t nz, int64_t ny, int64_t nx,
                int n_iter, double eps, const double *g_out, double *grad_d, double *grad_psf)
{
    if (!d || !psf || !g_out || nz < 1 || ny < 1 || nx < 1 || n_iter < 0 || !(eps > 0)) return -1;
    int64_t V = nz * ny * nx;
    size_t fb = sizeof(double) * (size_t)V;
    int K = n_iter;
    double *Hs = malloc(2 * fb);
    double *us = malloc(fb * (size_t)(K + 1));   /* u_0 .. u_K */
    double *bs = malloc(fb * (size_t)(K > 0 ? K : 1));
    double *qs = malloc(fb * (size_t)(K > 0 ? K : 1));
    double *rs = malloc(fb * (size_t)(K > 0 ? K : 1));
    double *gu = malloc(fb), *qb = malloc(fb), *rb = malloc(fb), *bb = malloc(fb), *tmp = malloc(fb);
    double *gd = calloc((size_t)V, sizeof(double));
    cplx *G = calloc((size_t)V, sizeof(cplx));     /* spectrum of dL/dh0 */
    cplx *w1 = malloc(sizeof(cplx) * (size_t)V), *w2 = malloc(sizeof(cplx) * (size_t)V);
    int rc = -2;
    if (!Hs || !us || !bs || !qs || !rs || !gu || !qb || !rb || !bb || !tmp || !gd || !G || !w1 || !w2)
        goto done;
    rc = orc_psf_spectrum(psf, Hs, nz, ny, nx);
    if (rc) goto done;
    const cplx *H = (const cplx *)Hs;
    double u0 = orc_initial_value(d, V, eps);
    for (int64_t i = 0; i < V; ++i) us[i] = u0;
    for (int k = 0; k < K && !rc; ++k)
        rc = orc_rl_iterate(Hs, d, us + (size_t)k * V, eps, nz, ny, nx,
                            us + (size_t)(k + 1) * V, bs + (size_t)k * V, rs + (size_t)k * V,
                            qs + (size_t)k * V);
    if (rc) goto done;

    memcpy(gu, g_out, fb);
    for (int k = K - 1; k >= 0 && !rc; --k) {
        const double *u = us + (size_t)k * V, *b = bs + (size_t)k * V;
        const double *r = rs + (size_t)k * V, *q = qs + (size_t)k * V;
        /* u_{k+1} = u * q */
        for (int64_t i = 0; i < V; ++i) { qb[i] = gu[i] * u[i]; gu[i] = gu[i] * q[i]; }
        /* q = corr(h, r): adjoint is convolution with h */
        rc = spectral_filter(H, qb, rb, w1, nz, ny, nx, 0);
        if (rc) break;
        /* r = d / c, c = max(b, eps) */
        for (int64_t i = 0; i < V; ++i) {
            double c = b[i] > eps ? b[i] : eps;
            gd[i] += rb[i] / c;
            double cb = -rb[i] * d[i] / (c * c);
            bb[i] = b[i] > eps ? cb : 0.0;
        }
        /* b = conv(h, u): adjoint is correlation with h */
        rc = spectral_filter(H, bb, tmp, w1, nz, ny, nx, 1);
        if (rc) break;
        for (int64_t i = 0; i < V; ++i) gu[i] += tmp[i];
        /* PSF: dL/dh0 += corr(bbar, u) + corr(r, qbar)
         *   F[sum_y bb(y) u(y-x)] = BB conj(U);  F[sum_y qb(y) r(y+x)] = conj(QB) R */
        for (int64_t i = 0; i < V; ++i) { w1[i] = bb[i]; w2[i] = u[i]; }
        if ((rc = fft3(w1, nz, ny, nx, 0)) || (rc = fft3(w2, nz, ny, nx, 0))) break;
        for (int64_t i = 0; i < V; ++i) G[i] += w1[i] * conj(w2[i]);
        for (int64_t i = 0; i < V; ++i) { w1[i] = qb[i]; w2[i] = r[i]; }
        if ((rc = fft3(w1, nz, ny, nx, 0)) || (rc = fft3(w2, nz, ny, nx, 0))) break;
        for (int64_t i = 0; i < V; ++i) G[i] += conj(w1[i]) * w2[i];
    }
    if (rc) goto done;
    /* u0 = max(mean(d), eps) */
    {
        double s = 0.0, sd = 0.0;
        for (int64_t i = 0; i < V; ++i) { s += gu[i]; sd += d[i]; }
        if (sd / (double)V > eps)
            for (int64_t i = 0; i < V; ++i) gd[i] += s / (double)V;
    }
    if (grad_d) memcpy(grad_d, gd, fb);
    if (grad_psf) {
        rc = fft3(G, nz, ny, nx, 1);
        if (rc) goto done;
        for (int64_t i = 0; i < V; ++i) tmp[i] = creal(G[i]);
        origin_to_center(tmp, grad_psf, nz, ny, nx);
    }
done:
    free(Hs); free(us); free(bs); free(qs); free(rs);
    free(gu); free(qb); free(rb); free(bb); free(tmp); free(gd); free(G); free(w1); free(w2);
    return rc;
}

/* ------------------------------------------------------- Gaussian PSF */

static double gauss_g(int64_t z, int64_t y, int64_t x, int64_t nz, int64_t ny, int64_t nx,
                      double sxy, double sz, double *rxy2, double *rz2)
{
    double dz = (double)(z - nz / 2), dy = (double)(y - ny / 2), dx = (double)(x - nx / 2);
    double a = dx * dx + dy * dy, c = dz * dz;
    if (rxy2) *rxy2 = a;
    if (rz2) *rz2 = c;
    return exp(-a / (2.0 * sxy * sxy) - c / (2.0 * sz * sz));
}

/* psf = A * g / sum(g) */
int orc_psf_gaussian(int64_t nz, int64_t ny, int64_t nx, double sxy, double sz, double amp, double *psf)
{
    if (!psf || nz < 1 || ny < 1 || nx < 1 || !(sxy > 0) || !(sz > 0)) return -1;
    double s = 0.0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double g = gauss_g(z, y, x, nz, ny, nx, sxy, sz, NULL, NULL);
                psf[(z * ny + y) * nx + x] = g;
                s += g;
            }
    for (int64_t i = 0; i < nz * ny * nx; ++i) psf[i] *= amp / s;
    return 0;
}

/* Chain rule through psf = A g / S, S = sum g:
 *   dL/dA   = sum(gp * g) / S
 *   dL/dsig = A/S * [sum(gp * dg) - sum(gp * g) * sum(dg) / S],
 *   dg/dsxy = g (dx^2+dy^2) / sxy^3,  dg/dsz = g dz^2 / sz^3.
 * out3 = {dL/dsxy, dL/dsz, dL/dA}. */
int orc_psf_gaussian_grad(int64_t nz, int64_t ny, int64_t nx, double sxy, double sz, double amp,
                          const double *grad_psf, double *out3)
{
    if (!grad_psf || !out3 || nz < 1 || ny < 1 || nx < 1 || !(sxy > 0) || !(sz > 0)) return -1;
    double S = 0, Sxy = 0, Sz = 0, Pg = 0, Pxy = 0, Pz = 0;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                double a, c;
                double g = gauss_g(z, y, x, nz, ny, nx, sxy, sz, &a, &c);
                double gxy = g * a / (sxy * sxy * sxy);
                double gz = g * c / (sz * sz * sz);
                double p = grad_psf[(z * ny + y) * nx + x];
                S += g; Sxy += gxy; Sz += gz;
                Pg += p * g; Pxy += p * gxy; Pz += p * gz;
            }
    out3[0] = amp / S * (Pxy - Pg * Sxy / S);
    out3[1] = amp / S * (Pz - Pg * Sz / S);
    out3[2] = Pg / S;
    return 0;
}
