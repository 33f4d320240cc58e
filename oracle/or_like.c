/*
 * Oracle likelihood and interim prior.
 *
 *   log P(d | theta) = -1/2 sum_p (d_p - m_p(theta))^2 / b      Eq. likelihood-pixels
 *   interim prior: log10 f ~ U(-1, 9), log10 s ~ U(-2, 1),
 *                  dx, dy ~ N(0, 0.5), (e1, e2) density
 *                  ~ (1-|e|^2)^2 exp(-|e|^2 / (2 * 0.3^2))      Eq. interim-prior
 *                                                               and the (e1,e2)
 *                                                               density after it
 *
 * The gradient follows the chain rule through the pixel sum:
 *   d logL / d theta_i = sum_p r_p dm_p/dtheta_i,  r = (d - m)/b,
 * and since m = IDFT(M), sum_p r_p dm_p/dtheta_i = (1/N^2) sum_k
 * Re[dM_k/dtheta_i conj(R_k)] with R = DFT(r) (the adjoint of the inverse DFT).
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

void or_prior_default(or_prior *pr)
{
    pr->lf_lo = -1.0; pr->lf_hi = 9.0;
    pr->ls_lo = -2.0; pr->ls_hi = 1.0;
    pr->sigma_xy = 0.5;
    pr->sigma_e = 0.3;
}

/* Normaliser of (1-|e|^2)^2 exp(-|e|^2/(2 alpha^2)) over the unit disk:
 * Z = pi int_0^1 (1-t)^2 exp(-a t) dt, a = 1/(2 alpha^2)
 *   = pi [1/a - 2/a^2 + 2 (1 - e^-a)/a^3]  (series in a for small a). */
static double z_ba14_of_a(double a)
{
    if (a < 1.0) {
        double s = 0.0, term = 1.0;          /* (-a)^n / n! */
        for (int n = 0; n < 40; ++n) {
            s += term * 2.0 / ((n + 1.0) * (n + 2.0) * (n + 3.0));
            term *= -a / (n + 1.0);
        }
        return OR_PI * s;
    }
    return OR_PI * (1.0 / a - 2.0 / (a * a) + 2.0 * (1.0 - exp(-a)) / (a * a * a));
}

double or_log_z_ba14(double alpha)
{
    return log(z_ba14_of_a(1.0 / (2.0 * alpha * alpha)));
}

double or_log_prior(const or_prior *pr, const double theta[6], double grad[6])
{
    double lf = theta[0], ls = theta[1], e1 = theta[2], e2 = theta[3];
    double dx = theta[4], dy = theta[5];
    double E = e1 * e1 + e2 * e2;
    if (!(lf > pr->lf_lo && lf < pr->lf_hi && ls > pr->ls_lo && ls < pr->ls_hi && E < 1.0))
        return -INFINITY;
    double sxy2 = pr->sigma_xy * pr->sigma_xy;
    double se2 = pr->sigma_e * pr->sigma_e;
    double lp = -log(pr->lf_hi - pr->lf_lo) - log(pr->ls_hi - pr->ls_lo)
                - log(2.0 * OR_PI * sxy2) - 0.5 * (dx * dx + dy * dy) / sxy2
                + 2.0 * log(1.0 - E) - 0.5 * E / se2 - or_log_z_ba14(pr->sigma_e);
    if (grad) {
        grad[0] = 0.0;
        grad[1] = 0.0;
        grad[2] = -4.0 * e1 / (1.0 - E) - e1 / se2;
        grad[3] = -4.0 * e2 / (1.0 - E) - e2 / se2;
        grad[4] = -dx / sxy2;
        grad[5] = -dy / sxy2;
    }
    return lp;
}

void or_twiddles(int N, double complex *tab);

static inline double complex tw(const double complex *tab, long m, int N)   /* exp(+2 pi i m / N) */
{
    long r = m % N;
    if (r < 0) r += N;
    return tab[r];
}

void or_idft_image(int N, const double *M_reim, double *img, int method);

/* Gradient of sum_x r(x) m(x) with respect to theta, r fixed: by Parseval
 * sum_k Re[dM_k/dtheta conj(R_k)] / N^2 with R the DFT of r (the adjoint DFT of
 * the residual), dM from the derivatives of the model spectrum M.  For the
 * profiles of Appendix B, M = F f(t) T phase with t = r0^2 q: d log f / dt is
 * -3/2 / (1 + t), -(1 + nu) / (1 + t) or -1/2, and d t / d log10 hlr = 2 ln10 t. */
static void adjoint_grad_p(int N, double p, const double *M, const double *r, const double theta[6],
                           int profile, double nu, double grad[6])
{
    int c = (N - 1) / 2;
    size_t NN = (size_t)N * N;
    /* R(u,v) = sum_{iy,ix} r exp(-2 pi i (u (ix-c) + v (iy-c)) / N), separable */
    double complex *B = malloc(sizeof(double complex) * NN);   /* [iy][u+c] */
    double complex *tab = malloc(sizeof(double complex) * (size_t)N);
    or_twiddles(N, tab);
    for (int iy = 0; iy < N; ++iy)
        for (int u = -c; u <= c; ++u) {
            double complex acc = 0;
            for (int ix = 0; ix < N; ++ix) acc += r[(size_t)iy * N + ix] * tw(tab, -(long)u * (ix - c), N);
            B[(size_t)iy * N + (u + c)] = acc;
        }
    double r0 = pow(10.0, theta[1]) / or_hlr_over_r0_p(profile, nu);
    double e1 = theta[2], e2 = theta[3];
    double E = e1 * e1 + e2 * e2;
    double dk = 2.0 * OR_PI / (N * p);
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int v = -c; v <= c; ++v)
        for (int u = -c; u <= c; ++u) {
            double complex R = 0;
            for (int iy = 0; iy < N; ++iy) R += B[(size_t)iy * N + (u + c)] * tw(tab, -(long)v * (iy - c), N);
            size_t idx = (size_t)(v + c) * N + (u + c);
            double complex Mk = M[2 * idx] + I * M[2 * idx + 1];
            double kx = u * dk, ky = v * dk, k2 = kx * kx + ky * ky;
            double A = (1.0 + E) * k2 + 2.0 * e1 * (kx * kx - ky * ky) + 4.0 * e2 * kx * ky;
            double q = A / (1.0 - E);
            double s = 1.0 + r0 * r0 * q;
            double dq1 = (2.0 * e1 * k2 + 2.0 * (kx * kx - ky * ky)) / (1.0 - E)
                         + 2.0 * e1 * A / ((1.0 - E) * (1.0 - E));
            double dq2 = (2.0 * e2 * k2 + 4.0 * kx * ky) / (1.0 - E)
                         + 2.0 * e2 * A / ((1.0 - E) * (1.0 - E));
            double complex dM[6];
            dM[0] = OR_LN10 * Mk;
            if (profile == OR_PROFILE_EXPONENTIAL) {
                dM[1] = -3.0 * OR_LN10 * (r0 * r0 * q / s) * Mk;
                dM[2] = -1.5 * r0 * r0 * dq1 / s * Mk;
                dM[3] = -1.5 * r0 * r0 * dq2 / s * Mk;
            } else {
                double dlogf = profile == OR_PROFILE_SPERGEL ? -(1.0 + nu) / s : -0.5;   /* d log f / dt */
                dM[1] = dlogf * 2.0 * OR_LN10 * r0 * r0 * q * Mk;
                dM[2] = dlogf * r0 * r0 * dq1 * Mk;
                dM[3] = dlogf * r0 * r0 * dq2 * Mk;
            }
            dM[4] = -I * p * kx * Mk;
            dM[5] = -I * p * ky * Mk;
            for (int i = 0; i < 6; ++i) g[i] += creal(dM[i] * conj(R));
        }
    for (int i = 0; i < 6; ++i) grad[i] = g[i] / (double)NN;
    free(B);
    free(tab);
}

double or_loglike_t(int N, double p, const double *T, const double *data,
                    const double *w, double sigma, const double theta[6],
                    double grad[6])
{
    size_t NN = (size_t)N * N;
    double *M = malloc(sizeof(double) * 2 * NN);
    double *m = malloc(sizeof(double) * NN);
    or_model_spectrum_t(N, p, T, theta, M);
    or_idft_image(N, M, m, 0);

    double b = sigma * sigma;
    double chi2 = 0.0;
    double *r = malloc(sizeof(double) * NN);
    for (size_t j = 0; j < NN; ++j) {
        double wj = w ? w[j] : 1.0;
        double res = data[j] - m[j];
        chi2 += wj * res * res;
        r[j] = wj * res / b;
    }
    double logl = -0.5 * chi2 / b;

    if (grad) adjoint_grad_p(N, p, M, r, theta, OR_PROFILE_EXPONENTIAL, 0.0, grad);
    free(M); free(m); free(r);
    return logl;
}

double or_loglike(int N, double p, const or_psf *psf, const double *data,
                  const double *w, double sigma, const double theta[6],
                  double grad[6])
{
    double *T = malloc(sizeof(double) * (size_t)N * N);
    or_transfer_table(N, p, psf, T);
    double v = or_loglike_t(N, p, T, data, w, sigma, theta, grad);
    free(T);
    return v;
}

double or_loglike_p(int profile, double nu, int N, double p, const or_psf *psf, const double *data,
                    double sigma, const double theta[6], double grad[6])
{
    size_t NN = (size_t)N * N;
    double *T = malloc(sizeof(double) * NN);
    double *M = malloc(sizeof(double) * 2 * NN);
    double *m = malloc(sizeof(double) * NN);
    double *r = malloc(sizeof(double) * NN);
    or_transfer_table(N, p, psf, T);
    or_model_spectrum_tp(N, p, T, profile, nu, theta, M);
    or_idft_image(N, M, m, 0);
    double b = sigma * sigma, chi2 = 0.0;
    for (size_t j = 0; j < NN; ++j) {
        double res = data[j] - m[j];
        chi2 += res * res;
        r[j] = res / b;
    }
    if (grad) adjoint_grad_p(N, p, M, r, theta, profile, nu, grad);
    free(T); free(M); free(m); free(r);
    return -0.5 * chi2 / b;
}

/* Lower Cholesky factor of the n x n symmetric matrix A (row-major) in place;
 * returns 0 if A is not positive definite. */
static int cholesky(double *A, int n)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return 0;
        d = sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / d;
        }
    }
    return 1;
}

double or_loglike_cov(int J, int N, double p, const or_psf *psf, const double *data, const double *sigma,
                      const double *corr, const double theta[6], double grad[6])
{
    int c = (N - 1) / 2, n = N * N;
    size_t NN = (size_t)n;
    double *M = malloc(sizeof(double) * 2 * NN);
    double *m = malloc(sizeof(double) * NN);
    double *T = malloc(sizeof(double) * NN);
    double *S = malloc(sizeof(double) * NN * NN);
    double *z = malloc(sizeof(double) * NN);
    double logl = 0.0, gj[6];
    if (grad)
        for (int i = 0; i < 6; ++i) grad[i] = 0.0;
    for (int j = 0; j < J && isfinite(logl); ++j) {
        or_transfer_table(N, p, &psf[j], T);
        or_model_spectrum_t(N, p, T, theta, M);
        or_idft_image(N, M, m, 0);
        const double *d = data + (size_t)j * NN;
        /* Sigma_j[a][b] = sigma_j^2 corr_j(x_a - x_b), lags wrapped to -c..c */
        double s2 = sigma[j] * sigma[j];
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                int dy = a / N - b / N, dx = a % N - b % N;
                dy = ((dy + c) % N + N) % N - c;
                dx = ((dx + c) % N + N) % N - c;
                double cv = corr ? corr[(size_t)j * NN + (size_t)(dy + c) * N + (dx + c)] : (dy == 0 && dx == 0);
                S[(size_t)a * n + b] = s2 * cv;
            }
        if (!cholesky(S, n)) {
            logl = NAN;
            break;
        }
        /* z = Sigma^-1 (d - m): forward then back substitution */
        for (int a = 0; a < n; ++a) {
            double t = d[a] - m[a];
            for (int k = 0; k < a; ++k) t -= S[(size_t)a * n + k] * z[k];
            z[a] = t / S[(size_t)a * n + a];
        }
        for (int a = n - 1; a >= 0; --a) {
            double t = z[a];
            for (int k = a + 1; k < n; ++k) t -= S[(size_t)k * n + a] * z[k];
            z[a] = t / S[(size_t)a * n + a];
        }
        double q = 0.0;
        for (int a = 0; a < n; ++a) q += (d[a] - m[a]) * z[a];
        logl -= 0.5 * q;
        if (grad) {
            adjoint_grad_p(N, p, M, z, theta, OR_PROFILE_EXPONENTIAL, 0.0, gj);
            for (int i = 0; i < 6; ++i) grad[i] += gj[i];
        }
    }
    free(M); free(m); free(T); free(S); free(z);
    return logl;
}

double or_loglike_dense(int N, double p, const or_psf *psf, const double *data, const double *Sigma,
                        const double theta[6], double grad[6])
{
    size_t n = (size_t)N * N;
    double *M = malloc(sizeof(double) * 2 * n);
    double *m = malloc(sizeof(double) * n);
    double *T = malloc(sizeof(double) * n);
    double *L = malloc(sizeof(double) * n * n);
    double *z = malloc(sizeof(double) * n);
    double logl = NAN;
    or_transfer_table(N, p, psf, T);
    or_model_spectrum_t(N, p, T, theta, M);
    or_idft_image(N, M, m, 0);
    memcpy(L, Sigma, sizeof(double) * n * n);
    if (cholesky(L, (int)n)) {
        /* z = Sigma^-1 (d - m): L y = r, then L^T z = y */
        for (size_t a = 0; a < n; ++a) {
            double t = data[a] - m[a];
            for (size_t k = 0; k < a; ++k) t -= L[a * n + k] * z[k];
            z[a] = t / L[a * n + a];
        }
        for (size_t a = n; a-- > 0;) {
            double t = z[a];
            for (size_t k = a + 1; k < n; ++k) t -= L[k * n + a] * z[k];
            z[a] = t / L[a * n + a];
        }
        double q = 0.0;
        for (size_t a = 0; a < n; ++a) q += (data[a] - m[a]) * z[a];
        logl = -0.5 * q;
        if (grad) adjoint_grad_p(N, p, M, z, theta, OR_PROFILE_EXPONENTIAL, 0.0, grad);
    }
    free(M); free(m); free(T); free(L); free(z);
    return logl;
}

double or_logpost(int N, double p, const or_psf *psf, const double *data,
                  const double *w, double sigma, const or_prior *pr,
                  const double theta[6], double grad[6])
{
    double gp[6];
    double lp = or_log_prior(pr, theta, grad ? gp : NULL);
    if (!isfinite(lp)) return -INFINITY;
    double ll = or_loglike(N, p, psf, data, w, sigma, theta, grad);
    if (grad)
        for (int i = 0; i < 6; ++i) grad[i] += gp[i];
    return ll + lp;
}
