/*
 * Oracle shear sampling phase.
 *
 *   eps' = (eps + g) / (1 + g* eps)                          Eq. shear-transform
 *   P(d | g, alpha) ~ prod_n (Z_n / K) sum_k
 *        P(omega'_nk | alpha, g) / P0(omega'_nk)             Eq. likelihood-shear
 *   P(omega' | alpha, g) = P(omega | alpha) |d eps / d eps'| Eq. true-prior-
 *                                                            jacobian-shear
 * with eps = (eps' - g) / (1 - g* eps') and the ellipticity densities over
 * (e1, e2) of Sec. 3.3 (the BA14 family (1-|e|^2)^2 exp(-|e|^2/2 alpha^2)
 * of Eq. ellip-mag-prior divided by |e|), or a Gaussian of per-component
 * width alpha truncated to |e| < R.  Centroid terms cancel sample by sample
 * (Sec. 3.3) and any other fixed prior ratio enters as a per-sample offset b.
 * The constant Z_n are dropped.
 *
 * The gradient is written with complex derivatives of the inverse map:
 *   d eps / d g1 = (-D + eps' (eps' - g)) / D^2,
 *   d eps / d g2 = -i (D + eps' (eps' - g)) / D^2,   D = 1 - g* eps'.
 *
 * Shear estimate (Sec. 3.4): posterior mean of g (and alpha) under a uniform
 * prior on the unit disk (alpha ~ U(lo, hi)), m and c from +-g pairs.
 *
 * TEST INFRASTRUCTURE ONLY (see bs_oracle.h).
 */
#include "bs_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

void or_shear_apply(double e1, double e2, double g1, double g2, double *o1, double *o2)
{
    double complex e = e1 + I * e2, g = g1 + I * g2;
    double complex r = (e + g) / (1.0 + conj(g) * e);
    *o1 = creal(r);
    *o2 = cimag(r);
}

void or_shear_invert(double e1p, double e2p, double g1, double g2, double *o1, double *o2)
{
    double complex ep = e1p + I * e2p, g = g1 + I * g2;
    double complex r = (ep - g) / (1.0 - conj(g) * ep);
    *o1 = creal(r);
    *o2 = cimag(r);
}

double or_shear_jacobian(double e1p, double e2p, double g1, double g2)
{
    double complex ep = e1p + I * e2p, g = g1 + I * g2;
    double g2abs = creal(g * conj(g));
    double D = cabs(1.0 - conj(g) * ep);
    return (1.0 - g2abs) * (1.0 - g2abs) / (D * D * D * D);
}

double or_log_z_ba14(double alpha);

/* d/da of pi int_0^1 (1-t)^2 e^{-a t} dt */
static double dz_ba14_da(double a)
{
    if (a < 1.0) {
        /* Z = pi sum_n (-a)^n/n! 2/((n+1)(n+2)(n+3)) */
        double s = 0.0, term = -1.0;      /* n (-a)^{n-1} (-1) / n!  at n = 1 */
        for (int n = 1; n < 40; ++n) {
            s += term * 2.0 / ((n + 1.0) * (n + 2.0) * (n + 3.0));
            term *= -a / n;
        }
        return OR_PI * s;
    }
    double ea = exp(-a);
    return OR_PI * (-1.0 / (a * a) + 4.0 / (a * a * a) - 6.0 * (1.0 - ea) / (a * a * a * a)
                    + 2.0 * ea / (a * a * a));
}

double or_log_z_eprior(int family, double alpha, double trunc_r)
{
    if (family == OR_EPRIOR_BA14) return or_log_z_ba14(alpha);
    double A = 1.0 / (2.0 * alpha * alpha);
    return log(2.0 * OR_PI * alpha * alpha * (1.0 - exp(-trunc_r * trunc_r * A)));
}

static double dlogz_dalpha(int family, double alpha, double trunc_r)
{
    if (family == OR_EPRIOR_BA14) {
        double a = 1.0 / (2.0 * alpha * alpha);
        double Z = exp(or_log_z_ba14(alpha));
        return dz_ba14_da(a) * (-1.0 / (alpha * alpha * alpha)) / Z;
    }
    double x = trunc_r * trunc_r / (2.0 * alpha * alpha);
    return 2.0 / alpha - (trunc_r * trunc_r / (alpha * alpha * alpha)) * exp(-x) / (1.0 - exp(-x));
}

double or_log_eprior(int family, double alpha, double trunc_r, double e1, double e2)
{
    double E = e1 * e1 + e2 * e2;
    if (family == OR_EPRIOR_BA14) {
        if (!(E < 1.0)) return -INFINITY;
        return 2.0 * log(1.0 - E) - E / (2.0 * alpha * alpha) - or_log_z_ba14(alpha);
    }
    if (!(E < trunc_r * trunc_r)) return -INFINITY;
    return -E / (2.0 * alpha * alpha) - or_log_z_eprior(family, alpha, trunc_r);
}

/* Log weight of one sample from its ellipticity: log p_e(eps | alpha)
 * + log|d eps / d eps'| - log P0_e(eps'), and (if dl) its derivatives with
 * respect to (g1, g2, alpha). */
static double eps_log_weight(double e1p, double e2p, int family, double trunc_r, double sigma_e0,
                             double g1, double g2, double alpha, double dlz, double dl[3])
{
    double complex g = g1 + I * g2;
    double gg = g1 * g1 + g2 * g2;
    double complex ep = e1p + I * e2p;
    double complex D = 1.0 - conj(g) * ep;
    double complex eps = (ep - g) / D;
    double E = creal(eps * conj(eps));
    double lpt = or_log_eprior(family, alpha, trunc_r, creal(eps), cimag(eps));
    double lJ = log(or_shear_jacobian(e1p, e2p, g1, g2));
    double lp0 = or_log_eprior(OR_EPRIOR_BA14, sigma_e0, 0.0, e1p, e2p);
    double lw = lpt + lJ - lp0;
    if (dl && isfinite(lw)) {
        double complex de1 = (-D + ep * (ep - g)) / (D * D);
        double complex de2 = -I * (D + ep * (ep - g)) / (D * D);
        double dE1 = 2.0 * creal(conj(eps) * de1);
        double dE2 = 2.0 * creal(conj(eps) * de2);
        double dlpt_dE = -1.0 / (2.0 * alpha * alpha);
        if (family == OR_EPRIOR_BA14) dlpt_dE += -2.0 / (1.0 - E);
        double absD2 = creal(D * conj(D));
        double dlJ1 = -4.0 * g1 / (1.0 - gg) - 4.0 * creal(conj(D) * (-ep)) / absD2;
        double dlJ2 = -4.0 * g2 / (1.0 - gg) - 4.0 * creal(conj(D) * (I * ep)) / absD2;
        dl[0] = dlpt_dE * dE1 + dlJ1;
        dl[1] = dlpt_dE * dE2 + dlJ2;
        dl[2] = E / (alpha * alpha * alpha) - dlz;
    }
    return lw;
}

double or_shear_loglike(const float *e1p, const float *e2p, const float *b,
                        int64_t n_gal, int K, int family, double trunc_r,
                        double sigma_e0, double g1, double g2, double alpha,
                        double grad[3])
{
    return or_shear_loglike_w(e1p, e2p, b, NULL, n_gal, K, family, trunc_r, sigma_e0, g1, g2, alpha, grad);
}

double or_shear_loglike_w(const float *e1p, const float *e2p, const float *b, const float *w,
                          int64_t n_gal, int K, int family, double trunc_r,
                          double sigma_e0, double g1, double g2, double alpha,
                          double grad[3])
{
    double dlz = dlogz_dalpha(family, alpha, trunc_r);
    double *lw = malloc(sizeof(double) * K);
    double (*dl)[3] = malloc(sizeof(double[3]) * K);
    double total = 0.0, G[3] = {0, 0, 0};
    for (int64_t n = 0; n < n_gal; ++n) {
        double mx = -INFINITY;
        for (int k = 0; k < K; ++k) {
            size_t j = (size_t)n * K + k;
            lw[k] = eps_log_weight((double)e1p[j], (double)e2p[j], family, trunc_r, sigma_e0, g1, g2, alpha,
                                   dlz, grad ? dl[k] : NULL) +
                    (b ? (double)b[j] : 0.0);
            if (lw[k] > mx) mx = lw[k];
        }
        double wn = w ? (double)w[n] : 1.0;
        if (wn == 0.0) continue;
        if (!isfinite(mx)) {
            total = -INFINITY;
            continue;
        }
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += exp(lw[k] - mx);
        total += wn * (mx + log(s) - log((double)K));
        if (grad)
            for (int k = 0; k < K; ++k) {
                double pk = exp(lw[k] - mx) / s;
                if (pk == 0.0) continue;
                for (int i = 0; i < 3; ++i) G[i] += wn * pk * dl[k][i];
            }
    }
    free(lw);
    free(dl);
    if (grad) memcpy(grad, G, sizeof G);
    return total;
}

/* ---- all properties free (Sec. 3.3 hyperpriors; Eq. lflux-lsize-dist) ---- */

double or_log_ndtr(double t)
{
    if (t > 5.0) return log1p(-0.5 * erfc(t / sqrt(2.0)));
    if (t >= -20.0) return log(0.5 * erfc(-t / sqrt(2.0)));
    /* Phi(t) = phi(t) / |t| (1 - 1/t^2 + 3/t^4 - 15/t^6 + 105/t^8 - ...) */
    double u = 1.0 / (t * t);
    double series = 1.0 - u * (1.0 - u * (3.0 - u * (15.0 - u * 105.0)));
    return -0.5 * t * t - log(-t) - 0.5 * log(2.0 * OR_PI) + log(series);
}

double or_log_skewnorm(double x, double mu, double sigma, double a)
{
    double z = (x - mu) / sigma;
    return log(2.0) - log(sigma) - 0.5 * z * z - 0.5 * log(2.0 * OR_PI) + or_log_ndtr(a * z);
}

/* Per-sample log prior ratio of log-flux and log-size, true over interim,
 * and its derivatives with respect to (mu_f, sigma_f, a_f, mu_s, sigma_s). */
static double flux_size_log_weight(double lf, double ls, const double hyp[5], const double interim[4],
                                   double dh[5])
{
    double mu_f = hyp[0], sig_f = hyp[1], a_f = hyp[2], mu_s = hyp[3], sig_s = hyp[4];
    double z = (lf - mu_f) / sig_f;
    double az = a_f * z;
    double lnorm = -0.5 * log(2.0 * OR_PI);
    double r = exp(lnorm - 0.5 * az * az - or_log_ndtr(az));   /* phi(az) / Phi(az) */
    double y = (ls - mu_s) / sig_s;
    double lw = or_log_skewnorm(lf, mu_f, sig_f, a_f) + (-log(sig_s) + lnorm - 0.5 * y * y) +
                log(interim[1] - interim[0]) + log(interim[3] - interim[2]);
    if (dh) {
        dh[0] = (z - a_f * r) / sig_f;
        dh[1] = (-1.0 + z * z - a_f * z * r) / sig_f;
        dh[2] = r * z;
        dh[3] = y / sig_s;
        dh[4] = (-1.0 + y * y) / sig_s;
    }
    return lw;
}

double or_shear_loglike_full_w(const float *e1p, const float *e2p, const float *lfp, const float *lsp,
                               const float *w, int64_t n_gal, int K, int family, double trunc_r, double sigma_e0,
                               const double interim[4], const double theta[8], double grad[8])
{
    const double g1 = theta[0], g2 = theta[1], alpha = theta[2];
    const double *hyp = theta + 3;
    double dlz = dlogz_dalpha(family, alpha, trunc_r);
    double *lw = malloc(sizeof(double) * K);
    double (*dl)[8] = malloc(sizeof(double[8]) * K);
    double total = 0.0, G[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t n = 0; n < n_gal; ++n) {
        double wn = w ? (double)w[n] : 1.0, mx = -INFINITY;
        if (wn == 0.0) continue;
        for (int k = 0; k < K; ++k) {
            size_t j = (size_t)n * K + k;
            lw[k] = eps_log_weight((double)e1p[j], (double)e2p[j], family, trunc_r, sigma_e0, g1, g2, alpha, dlz,
                                   grad ? dl[k] : NULL) +
                    flux_size_log_weight((double)lfp[j], (double)lsp[j], hyp, interim, grad ? dl[k] + 3 : NULL);
            if (lw[k] > mx) mx = lw[k];
        }
        if (!isfinite(mx)) {
            total = -INFINITY;
            continue;
        }
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += exp(lw[k] - mx);
        total += wn * (mx + log(s) - log((double)K));
        if (grad)
            for (int k = 0; k < K; ++k) {
                double pk = exp(lw[k] - mx) / s;
                if (pk == 0.0) continue;
                for (int i = 0; i < 8; ++i) G[i] += wn * pk * dl[k][i];
            }
    }
    free(lw);
    free(dl);
    if (grad) memcpy(grad, G, sizeof G);
    return total;
}

double or_shear_loglike_full(const float *e1p, const float *e2p, const float *lfp, const float *lsp,
                             int64_t n_gal, int K, int family, double trunc_r, double sigma_e0,
                             const double interim[4], const double theta[8], double grad[8])
{
    return or_shear_loglike_full_w(e1p, e2p, lfp, lsp, NULL, n_gal, K, family, trunc_r, sigma_e0, interim, theta,
                                   grad);
}

/* ---- Gauss-Hermite by Golub-Welsch: nodes are the eigenvalues of the
 *      Jacobi matrix of the Hermite recurrence (off-diagonal sqrt(k/2)),
 *      weights sqrt(pi) times the squared first eigenvector components. ---- */
int or_gauss_hermite(int n, double *x, double *w)
{
    if (n < 1 || n > 64) return -1;
    double *A = calloc((size_t)n * n, sizeof(double));
    double *V = calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int i = 0; i + 1 < n; ++i) A[i * n + i + 1] = A[(i + 1) * n + i] = sqrt((i + 1) / 2.0);
    for (int sweep = 0; sweep < 100; ++sweep) {          /* cyclic Jacobi rotations */
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (fabs(apq) < 1e-300) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < n; ++k) {          /* A <- A J */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = cs * akp - sn * akq;
                    A[k * n + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < n; ++k) {          /* A <- J^T A */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = cs * apk - sn * aqk;
                    A[q * n + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < n; ++k) {          /* V <- V J */
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = cs * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + cs * vkq;
                }
            }
    }
    /* sort ascending */
    int *idx = malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (A[idx[j] * n + idx[j]] < A[idx[i] * n + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    for (int i = 0; i < n; ++i) {
        int k = idx[i];
        x[i] = A[k * n + k];
        w[i] = sqrt(OR_PI) * V[0 * n + k] * V[0 * n + k];
    }
    free(idx); free(A); free(V);
    return 0;
}

typedef struct {
    const float *e1p, *e2p, *b, *w;
    int64_t n_gal;
    int K, family;
    double trunc_r, sigma_e0;
    int free_alpha;
    double alpha_fixed, alpha_lo, alpha_hi;
} sdat_t;

static int in_prior(const sdat_t *d, const double *x)
{
    if (!(x[0] * x[0] + x[1] * x[1] < 1.0)) return 0;
    if (d->free_alpha && !(x[2] > d->alpha_lo && x[2] < d->alpha_hi)) return 0;
    return 1;
}

static double sfun(const sdat_t *d, const double *x, double *gr)
{
    double a = d->free_alpha ? x[2] : d->alpha_fixed;
    double g3[3];
    double v = or_shear_loglike_w(d->e1p, d->e2p, d->b, d->w, d->n_gal, d->K, d->family, d->trunc_r,
                                d->sigma_e0, x[0], x[1], a, gr ? g3 : NULL);
    if (gr) {
        gr[0] = g3[0]; gr[1] = g3[1];
        if (d->free_alpha) gr[2] = g3[2];
    }
    return v;
}

/* Cholesky of a symmetric positive-definite n x n matrix (lower, in place) */
static int cholesky(double *A, int n)
{
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return -1;
        A[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / A[j * n + j];
        }
        for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
    }
    return 0;
}

/* Hessian by central differences of the analytic gradient */
static void hessian(const sdat_t *d, const double *x, int n, double *H)
{
    for (int j = 0; j < n; ++j) {
        double h = 1e-5;
        double xp[3], xm[3], gp[3], gm[3];
        memcpy(xp, x, sizeof(double) * n);
        memcpy(xm, x, sizeof(double) * n);
        xp[j] += h;
        xm[j] -= h;
        sfun(d, xp, gp);
        sfun(d, xm, gm);
        for (int i = 0; i < n; ++i) H[i * n + j] = (gp[i] - gm[i]) / (2.0 * h);
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double s = 0.5 * (H[i * n + j] + H[j * n + i]);
            H[i * n + j] = H[j * n + i] = s;
        }
}

int or_shear_estimate(const float *e1p, const float *e2p, const float *b,
                      int64_t n_gal, int K, int family, double trunc_r,
                      double sigma_e0, int free_alpha, double alpha_fixed,
                      double alpha_lo, double alpha_hi, int n_gh,
                      double *mean, double *cov)
{
    return or_shear_estimate_w(e1p, e2p, b, NULL, n_gal, K, family, trunc_r, sigma_e0, free_alpha, alpha_fixed,
                               alpha_lo, alpha_hi, n_gh, mean, cov);
}

int or_shear_estimate_w(const float *e1p, const float *e2p, const float *b, const float *w,
                        int64_t n_gal, int K, int family, double trunc_r,
                        double sigma_e0, int free_alpha, double alpha_fixed,
                        double alpha_lo, double alpha_hi, int n_gh,
                        double *mean, double *cov)
{
    sdat_t d = {e1p, e2p, b, w, n_gal, K, family, trunc_r, sigma_e0,
                free_alpha, alpha_fixed, alpha_lo, alpha_hi};
    int n = free_alpha ? 3 : 2;
    double x[3] = {0.0, 0.0, alpha_fixed};
    double gr[3], H[9], L[9];
    double f = sfun(&d, x, gr);
    /* Newton with step halving inside the prior support */
    for (int it = 0; it < 100; ++it) {
        hessian(&d, x, n, H);
        for (int i = 0; i < n * n; ++i) L[i] = -H[i];
        double step[3];
        if (cholesky(L, n) == 0) {
            double y[3];
            for (int i = 0; i < n; ++i) {           /* L y = grad */
                double s = gr[i];
                for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
                y[i] = s / L[i * n + i];
            }
            for (int i = n - 1; i >= 0; --i) {      /* L^T step = y */
                double s = y[i];
                for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * step[k];
                step[i] = s / L[i * n + i];
            }
        } else {
            for (int i = 0; i < n; ++i) step[i] = 1e-6 * gr[i];
        }
        double t = 1.0, xn[3], fn = -INFINITY, gn[3];
        for (int ls = 0; ls < 60; ++ls) {
            for (int i = 0; i < n; ++i) xn[i] = x[i] + t * step[i];
            if (in_prior(&d, xn)) {
                fn = sfun(&d, xn, gn);
                if (fn >= f - 1e-10 * fabs(f)) break;
            }
            t *= 0.5;
        }
        double dmax = 0.0;
        for (int i = 0; i < n; ++i) dmax = fmax(dmax, fabs(t * step[i]));
        memcpy(x, xn, sizeof(double) * n);
        memcpy(gr, gn, sizeof(double) * n);
        f = fn;
        if (dmax < 1e-12) break;
    }
    /* Laplace scaling: Sigma = (-H)^-1, node theta = xhat + sqrt(2) Lc z */
    hessian(&d, x, n, H);
    double Sg[9], Lc[9];
    {
        /* invert -H via Cholesky */
        for (int i = 0; i < n * n; ++i) L[i] = -H[i];
        if (cholesky(L, n) != 0) return -1;
        double Li[9] = {0};
        for (int j = 0; j < n; ++j) {               /* L^-1 column by column */
            for (int i = 0; i < n; ++i) {
                double s = (i == j) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) s -= L[i * n + k] * Li[k * n + j];
                Li[i * n + j] = s / L[i * n + i];
            }
        }
        for (int i = 0; i < n; ++i)                 /* Sigma = L^-T L^-1 */
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += Li[k * n + i] * Li[k * n + j];
                Sg[i * n + j] = s;
            }
        memcpy(Lc, Sg, sizeof(double) * n * n);
        if (cholesky(Lc, n) != 0) return -1;
    }
    double gx[64], gw[64];
    if (or_gauss_hermite(n_gh, gx, gw) != 0) return -1;
    int total = 1;
    for (int i = 0; i < n; ++i) total *= n_gh;
    double *lw = malloc(sizeof(double) * total);
    double (*th)[3] = malloc(sizeof(double[3]) * total);
    double lmax = -INFINITY;
    for (int j = 0; j < total; ++j) {
        int r = j;
        double z[3], logw = 0.0, zz = 0.0;
        for (int i = 0; i < n; ++i) {
            int a = r % n_gh;
            r /= n_gh;
            z[i] = gx[a];
            logw += log(gw[a]);
            zz += z[i] * z[i];
        }
        for (int i = 0; i < n; ++i) {
            double s = x[i];
            for (int k = 0; k <= i; ++k) s += sqrt(2.0) * Lc[i * n + k] * z[k];
            th[j][i] = s;
        }
        if (!in_prior(&d, th[j])) { lw[j] = -INFINITY; continue; }
        lw[j] = logw + sfun(&d, th[j], NULL) - f + zz;
        if (lw[j] > lmax) lmax = lw[j];
    }
    double wsum = 0.0, m[3] = {0, 0, 0};
    for (int j = 0; j < total; ++j) {
        double wj = exp(lw[j] - lmax);
        wsum += wj;
        for (int i = 0; i < n; ++i) m[i] += wj * th[j][i];
    }
    for (int i = 0; i < n; ++i) mean[i] = m[i] / wsum;
    if (cov) {
        for (int i = 0; i < 9; ++i) cov[i] = 0.0;
        for (int j = 0; j < total; ++j) {
            double wj = exp(lw[j] - lmax) / wsum;
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < n; ++c)
                    cov[a * 3 + c] += wj * (th[j][a] - mean[a]) * (th[j][c] - mean[c]);
        }
    }
    free(lw);
    free(th);
    return 0;
}
