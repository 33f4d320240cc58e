/*
 * Oracle forward model: an exponential (Sersic n = 1) galaxy, sheared in the
 * reduced-shear convention (Sec. 2, Eq. ellip-phi-transform; Sec. 3.2,
 * Eq. shear-transform), convolved with a known PSF (Sec. 2: Gaussian; Moffat
 * as a per-galaxy PSF of the graphical model, Fig. pgm) and the pixel
 * response, evaluated analytically in k-space and drawn on the stamp's
 * periodic grid by an inverse DFT (Sec. 3.3 forward model).
 *
 * TEST INFRASTRUCTURE ONLY (see bs_oracle.h).
 */
#include "bs_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_LN10 2.30258509299404568402

/* Half-light radius of the exponential in units of its scale length: the
 * enclosed flux fraction of exp(-r/r0) within R is 1 - (1 + R/r0) e^{-R/r0};
 * solve for one half by Newton's method. */
double or_hlr_over_r0(void)
{
    double x = 1.7;
    for (int it = 0; it < 60; ++it) {
        double f = (1.0 + x) * exp(-x) - 0.5;
        double fp = -x * exp(-x);
        double dx = f / fp;
        x -= dx;
        if (fabs(dx) < 1e-16 * x) break;
    }
    return x;
}

/* Modified Bessel function of the second kind from its integral
 * representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (x > 0),
 * by the trapezoidal rule, which converges geometrically for this analytic,
 * double-exponentially decaying integrand. */
double or_bessel_k(double nu, double x)
{
    const double h = 0.02;
    double sum = 0.5 * exp(-x);
    double anu = fabs(nu);
    for (int j = 1; j < 2000000; ++j) {
        double t = j * h;
        double term = exp(-x * cosh(t) + anu * t) * 0.5 * (1.0 + exp(-2.0 * anu * t));
        sum += term;
        if (x * cosh(t) > anu * t + 60.0 && term < 1e-22 * sum) break;
    }
    return sum * h;
}

/* Transform of the unit-flux PSF at radial wavenumber k (1/arcsec). */
double or_psf_ft(const or_psf *psf, double k)
{
    if (psf == NULL || psf->kind == OR_PSF_NONE) return 1.0;
    if (psf->kind == OR_PSF_GAUSSIAN) {
        double sigma = psf->fwhm / (2.0 * sqrt(2.0 * log(2.0)));
        return exp(-0.5 * k * k * sigma * sigma);
    }
    /* Moffat (1 + r^2/rd^2)^-beta, FWHM = 2 rd sqrt(2^{1/beta} - 1).
     * Its Hankel transform is (2/Gamma(beta-1)) (x/2)^{beta-1} K_{beta-1}(x),
     * x = k rd, which tends to 1 as x -> 0. */
    double beta = psf->beta;
    double rd = psf->fwhm / (2.0 * sqrt(pow(2.0, 1.0 / beta) - 1.0));
    double x = k * rd;
    if (x == 0.0) return 1.0;
    double nu = beta - 1.0;
    return 2.0 / tgamma(nu) * pow(0.5 * x, nu) * or_bessel_k(nu, x);
}

/* Transform of the unit-flux exponential exp(-|S^-1 x|/r0)/(2 pi r0^2) with
 * the area-preserving shear S = (1-|e|^2)^{-1/2} [[1+e1, e2], [e2, 1-e1]]:
 * (1 + r0^2 k^T S^2 k)^{-3/2}. */
double or_exp_profile_ft(double kx, double ky, double r0, double e1, double e2)
{
    double E = e1 * e1 + e2 * e2;
    double k2 = kx * kx + ky * ky;
    double q = ((1.0 + E) * k2 + 2.0 * e1 * (kx * kx - ky * ky) + 4.0 * e2 * kx * ky) / (1.0 - E);
    return pow(1.0 + r0 * r0 * q, -1.5);
}

/* Appendix B profiles: Spergel (index nu; nu = 1/2 is the exponential) and
 * Gaussian.  Transform of the unit-flux profile as a function of
 * t = r0^2 q(k): (1 + t)^-3/2, (1 + t)^-(1+nu), exp(-t/2). */
double or_profile_ft(int profile, double nu, double t)
{
    if (profile == OR_PROFILE_SPERGEL) return pow(1.0 + t, -(1.0 + nu));
    if (profile == OR_PROFILE_GAUSSIAN) return exp(-0.5 * t);
    return pow(1.0 + t, -1.5);
}

/* hlr / r0: for the Spergel profile I(r) ~ (r/r0)^nu K_nu(r/r0), whose
 * enclosed flux is 1 - x^(1+nu) K_(1+nu)(x) / (2^nu Gamma(1+nu)) at x = r/r0,
 * the root of that flux = 1/2 by bisection; sqrt(2 ln 2) for the Gaussian
 * exp(-r^2 / (2 r0^2)). */
double or_hlr_over_r0_p(int profile, double nu)
{
    if (profile == OR_PROFILE_GAUSSIAN) return sqrt(2.0 * log(2.0));
    if (profile != OR_PROFILE_SPERGEL) return or_hlr_over_r0();
    double norm = pow(2.0, nu) * tgamma(1.0 + nu);
    double lo = 1e-8, hi = 60.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double enclosed = 1.0 - pow(mid, 1.0 + nu) * or_bessel_k(1.0 + nu, mid) / norm;
        if (enclosed < 0.5) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* PSF-and-pixel transfer T(u,v) = PSF(|k|) sinc(kx p/2) sinc(ky p/2) on the
 * full grid, row-major [v+c][u+c]; it depends only on the stamp, so the
 * likelihood computes it once per galaxy. */
void or_transfer_table(int N, double p, const or_psf *psf, double *T)
{
    int c = (N - 1) / 2;
    double dk = 2.0 * OR_PI / (N * p);
    for (int v = -c; v <= c; ++v)
        for (int u = -c; u <= c; ++u) {
            double kx = u * dk, ky = v * dk;
            T[(size_t)(v + c) * N + (u + c)] =
                or_psf_ft(psf, sqrt(kx * kx + ky * ky)) * sinc(0.5 * kx * p) * sinc(0.5 * ky * p);
        }
}

/* M(u,v) = F * I_exp(k; r0, e) * T(u,v) * exp(-i p (kx dx + ky dy)) */
void or_model_spectrum_t(int N, double p, const double *T, const double theta[6],
                         double *M_reim)
{
    int c = (N - 1) / 2;
    double F = pow(10.0, theta[0]);
    double r0 = pow(10.0, theta[1]) / or_hlr_over_r0();
    double e1 = theta[2], e2 = theta[3], dx = theta[4], dy = theta[5];
    double dk = 2.0 * OR_PI / (N * p);
    for (int v = -c; v <= c; ++v) {
        for (int u = -c; u <= c; ++u) {
            double kx = u * dk, ky = v * dk;
            size_t idx = (size_t)(v + c) * N + (u + c);
            double amp = F * or_exp_profile_ft(kx, ky, r0, e1, e2) * T[idx];
            double complex Mk = amp * cexp(-I * p * (kx * dx + ky * dy));
            M_reim[2 * idx] = creal(Mk);
            M_reim[2 * idx + 1] = cimag(Mk);
        }
    }
}

/* The same with the profile of Appendix B (profile 0 is the exponential). */
void or_model_spectrum_tp(int N, double p, const double *T, int profile, double nu, const double theta[6],
                          double *M_reim)
{
    if (profile == OR_PROFILE_EXPONENTIAL) {
        or_model_spectrum_t(N, p, T, theta, M_reim);
        return;
    }
    int c = (N - 1) / 2;
    double F = pow(10.0, theta[0]);
    double r0 = pow(10.0, theta[1]) / or_hlr_over_r0_p(profile, nu);
    double e1 = theta[2], e2 = theta[3], dx = theta[4], dy = theta[5];
    double E = e1 * e1 + e2 * e2;
    double dk = 2.0 * OR_PI / (N * p);
    for (int v = -c; v <= c; ++v) {
        for (int u = -c; u <= c; ++u) {
            double kx = u * dk, ky = v * dk, k2 = kx * kx + ky * ky;
            double q = ((1.0 + E) * k2 + 2.0 * e1 * (kx * kx - ky * ky) + 4.0 * e2 * kx * ky) / (1.0 - E);
            size_t idx = (size_t)(v + c) * N + (u + c);
            double amp = F * or_profile_ft(profile, nu, r0 * r0 * q) * T[idx];
            double complex Mk = amp * cexp(-I * p * (kx * dx + ky * dy));
            M_reim[2 * idx] = creal(Mk);
            M_reim[2 * idx + 1] = cimag(Mk);
        }
    }
}

void or_model_spectrum(int N, double p, const or_psf *psf, const double theta[6],
                       double *M_reim)
{
    double *T = malloc(sizeof(double) * (size_t)N * N);
    or_transfer_table(N, p, psf, T);
    or_model_spectrum_t(N, p, T, theta, M_reim);
    free(T);
}

/* Table of exp(+2 pi i r / N), r = 0..N-1; a phase exp(2 pi i m / N) for any
 * integer m is the entry at m reduced mod N (exact argument reduction). */
void or_twiddles(int N, double complex *tab)
{
    for (int r = 0; r < N; ++r) tab[r] = cexp(I * (2.0 * OR_PI * (double)r / (double)N));
}

static inline double complex twiddle(const double complex *tab, long m, int N)
{
    long r = m % N;
    if (r < 0) r += N;
    return tab[r];
}

void or_idft_image(int N, const double *M_reim, double *img, int method)
{
    int c = (N - 1) / 2;
    double inv = 1.0 / ((double)N * (double)N);
    double complex *tab = malloc(sizeof(double complex) * (size_t)N);
    or_twiddles(N, tab);
    if (method == 1) {
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                double complex acc = 0;
                for (int v = -c; v <= c; ++v)
                    for (int u = -c; u <= c; ++u) {
                        size_t idx = (size_t)(v + c) * N + (u + c);
                        double complex Mk = M_reim[2 * idx] + I * M_reim[2 * idx + 1];
                        acc += Mk * twiddle(tab, (long)u * (ix - c) + (long)v * (iy - c), N);
                    }
                img[iy * N + ix] = creal(acc) * inv;
            }
        free(tab);
        return;
    }
    /* separable: first over u for each (v, ix), then over v */
    double complex *A = malloc(sizeof(double complex) * (size_t)N * N);
    for (int v = -c; v <= c; ++v)
        for (int ix = 0; ix < N; ++ix) {
            double complex acc = 0;
            for (int u = -c; u <= c; ++u) {
                size_t idx = (size_t)(v + c) * N + (u + c);
                acc += (M_reim[2 * idx] + I * M_reim[2 * idx + 1]) * twiddle(tab, (long)u * (ix - c), N);
            }
            A[(size_t)(v + c) * N + ix] = acc;
        }
    for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix) {
            double complex acc = 0;
            for (int v = -c; v <= c; ++v)
                acc += A[(size_t)(v + c) * N + ix] * twiddle(tab, (long)v * (iy - c), N);
            img[iy * N + ix] = creal(acc) * inv;
        }
    free(A);
    free(tab);
}

void or_render(int N, double p, const or_psf *psf, const double theta[6],
               double *img, int method)
{
    double *M = malloc(sizeof(double) * 2 * (size_t)N * N);
    or_model_spectrum(N, p, psf, theta, M);
    or_idft_image(N, M, img, method);
    free(M);
}

/* n stamps of one side N, OpenMP-parallel over stamps; psf[n_psf] with
 * n_psf = 1 or n; theta [n][6]; img [n][N*N]. */
void or_render_many(int n, int N, double p, const or_psf *psf, int n_psf, const double *theta,
                    double *img)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int i = 0; i < n; ++i)
        or_render(N, p, psf + (n_psf == 1 ? 0 : i), theta + 6 * (size_t)i, img + (size_t)i * N * N, 0);
}

/* Real-space reference.  Pixel value = integral over the pixel of the
 * periodically summed (galaxy * PSF).  Writing the PSF-and-pixel kernel of
 * pixel j as K_j(y) = int_pixel G(x - y) dx, which for a Gaussian PSF and a
 * square pixel is a product of erf differences, the value is
 * int_box Iper(y) Kper_j(y) dy over one period box; the integral is taken by
 * the midpoint rule on nsub x nsub points per pixel. */
void or_render_realspace_gauss(int N, double p, double psf_fwhm,
                               const double theta[6], int nsub, int nimg,
                               double *img)
{
    int c = (N - 1) / 2;
    double L = N * p;
    double F = pow(10.0, theta[0]);
    double r0 = pow(10.0, theta[1]) / or_hlr_over_r0();
    double e1 = theta[2], e2 = theta[3];
    double cx = theta[4] * p, cy = theta[5] * p;
    double E = e1 * e1 + e2 * e2;
    double s = 1.0 / sqrt(1.0 - E);
    /* S^{-1} = (1-E)^{-1/2} [[1-e1, -e2], [-e2, 1+e1]] */
    double a11 = s * (1.0 - e1), a12 = -s * e2, a22 = s * (1.0 + e1);
    double sig = psf_fwhm / (2.0 * sqrt(2.0 * log(2.0)));
    int ns = N * nsub;
    double h = p / nsub;
    double *pos = malloc(sizeof(double) * ns);
    for (int i = 0; i < ns; ++i) pos[i] = -0.5 * L + (i + 0.5) * h;
    /* 1-D periodic PSF-and-pixel kernel K[j][i] for pixel j, sample i */
    double *K = malloc(sizeof(double) * (size_t)N * ns);
    for (int j = 0; j < N; ++j) {
        double xc = (j - c) * p;
        for (int i = 0; i < ns; ++i) {
            double acc = 0.0;
            for (int m = -nimg; m <= nimg; ++m) {
                double y = pos[i] + m * L;
                double hi = (xc + 0.5 * p - y) / (sqrt(2.0) * sig);
                double lo = (xc - 0.5 * p - y) / (sqrt(2.0) * sig);
                acc += 0.5 * (erf(hi) - erf(lo));
            }
            K[(size_t)j * ns + i] = acc;
        }
    }
    /* periodic galaxy on the sample grid */
    double *G = malloc(sizeof(double) * (size_t)ns * ns);
    for (int iy = 0; iy < ns; ++iy)
        for (int ix = 0; ix < ns; ++ix) {
            double acc = 0.0;
            for (int my = -nimg; my <= nimg; ++my)
                for (int mx = -nimg; mx <= nimg; ++mx) {
                    double x = pos[ix] + mx * L - cx, y = pos[iy] + my * L - cy;
                    double ux = a11 * x + a12 * y, uy = a12 * x + a22 * y;
                    acc += exp(-sqrt(ux * ux + uy * uy) / r0);
                }
            G[(size_t)iy * ns + ix] = acc * F / (2.0 * OR_PI * r0 * r0) * h * h;
        }
    /* img = K_y G K_x^T */
    double *T = malloc(sizeof(double) * (size_t)ns * N);
    for (int iy = 0; iy < ns; ++iy)
        for (int jx = 0; jx < N; ++jx) {
            double acc = 0.0;
            for (int ix = 0; ix < ns; ++ix) acc += G[(size_t)iy * ns + ix] * K[(size_t)jx * ns + ix];
            T[(size_t)iy * N + jx] = acc;
        }
    for (int jy = 0; jy < N; ++jy)
        for (int jx = 0; jx < N; ++jx) {
            double acc = 0.0;
            for (int iy = 0; iy < ns; ++iy) acc += K[(size_t)jy * ns + iy] * T[(size_t)iy * N + jx];
            img[jy * N + jx] = acc;
        }
    free(pos); free(K); free(G); free(T);
}
