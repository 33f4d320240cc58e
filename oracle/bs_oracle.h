/*
 * bs_oracle.h -- plain FP64 CPU oracle for Bayesian shear inference with a
 * known PSF and sky background (Mendoza et al., "Differentiable Forward
 * Modeling for Efficient and Accurate Shear Inference").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  Only
 * the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA path, and the CUDA path never calls it.
 *
 * Every function is a slow, direct restatement of the paper's definitions in
 * double precision, in the paper's order:
 *   - exponential galaxy sheared by the reduced-shear ellipticity (Sec. 2,
 *     Eq. ellip-phi-transform; Sec. 3.2, Eq. shear-transform), convolved with
 *     a known PSF and the pixel response, drawn on the stamp's periodic grid
 *     by an inverse DFT (Sec. 3.3, forward model);
 *   - Gaussian pixel likelihood (Eq. likelihood-pixels) times the interim
 *     prior (Eq. interim-prior and the (e1,e2) density that follows it);
 *   - gradient-based MCMC with dual-averaging step size (Sec. 3.3), run as
 *     fixed-length HMC, initialised as in Eq. initialize (caller-supplied);
 *   - MC shear likelihood (Eq. likelihood-shear) with the Jacobian of
 *     Eq. true-prior-jacobian-shear;
 *   - posterior-mean shear estimate and the m / c estimators of Sec. 3.4;
 *   - ESS and R-hat diagnostics of Sec. 4.1.
 *
 * Parameter vector theta = (lF, ls, e1, e2, dx, dy):
 *   lF = log10 flux, ls = log10 half-light radius in arcsec (of the circular
 *   profile before the area-preserving shear), (e1, e2) = sheared ellipticity
 *   in the reduced-shear ("epsilon") convention, (dx, dy) = centroid offset
 *   in pixels.
 *
 * Grid conventions (N odd, c = (N-1)/2, pixel scale p):
 *   pixel (iy, ix) has centre x = (ix - c) p, y = (iy - c) p;
 *   k-point (u, v), u, v in [-c, c], has kx = 2 pi u / (N p), ky = 2 pi v / (N p);
 *   image m[iy*N + ix] = (1/N^2) sum_{u,v} M(u,v) exp(+i (kx x + ky y)).
 */
#ifndef BS_ORACLE_H
#define BS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- constants ------------------------------------------------------- */

enum { OR_PSF_NONE = 0, OR_PSF_GAUSSIAN = 1, OR_PSF_MOFFAT = 2 };
enum { OR_EPRIOR_BA14 = 0, OR_EPRIOR_TRUNC_GAUSS = 1 };

typedef struct {
    int kind;          /* OR_PSF_* */
    double fwhm;       /* arcsec */
    double beta;       /* Moffat index (ignored for the Gaussian) */
} or_psf;

/* Interim prior of Eq. interim-prior. */
typedef struct {
    double lf_lo, lf_hi;   /* log10 flux ~ U(lf_lo, lf_hi)            (-1, 9) */
    double ls_lo, ls_hi;   /* log10 hlr  ~ U(ls_lo, ls_hi)            (-2, 1) */
    double sigma_xy;       /* dx, dy ~ N(0, sigma_xy) in pixels       0.5     */
    double sigma_e;        /* ellipticity shape-noise parameter        0.3     */
} or_prior;

typedef struct {
    int n_chains, n_warmup, n_samples, n_leapfrog;
    double target_accept;  /* dual-averaging target delta */
    double jitter;         /* step jitter fraction: eps * U(1-j, 1+j) */
    int adapt_mass;        /* 1: windowed diagonal metric adaptation */
    uint64_t seed;
    int random_steps;      /* 1: L_i = 1 + floor(u7 L) leapfrog steps per
                              iteration (u7 then no longer jitters eps) */
} or_hmc_cfg;

/* ---- counter-based generator (Philox4x64-10, Salmon et al. 2011) ------ */

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* Eight 24-bit uniforms in (0,1) from one Philox block with
 * key = (seed, chain_key), counter = (c0, c1, c2, 0). */
void or_uniforms8(uint64_t seed, uint64_t chain_key, uint64_t c0, uint64_t c1,
                  uint64_t c2, double u[8]);

/* ---- forward model ---------------------------------------------------- */

double or_hlr_over_r0(void);                       /* root of 1-(1+x)e^-x = 1/2 */
double or_bessel_k(double nu, double x);           /* K_nu(x), x > 0 */
double or_psf_ft(const or_psf *psf, double k);     /* PSF transform, PSF(0) = 1 */
double or_exp_profile_ft(double kx, double ky, double r0, double e1, double e2);
/* Appendix B profiles */
enum { OR_PROFILE_EXPONENTIAL = 0, OR_PROFILE_SPERGEL = 1, OR_PROFILE_GAUSSIAN = 2 };
double or_profile_ft(int profile, double nu, double t);      /* unit-flux transform at t = r0^2 q */
double or_hlr_over_r0_p(int profile, double nu);
/* Full model spectrum M(u,v) on the N x N grid, row-major [v+c][u+c],
 * complex values as interleaved (re, im) pairs. */
void or_model_spectrum(int N, double p, const or_psf *psf, const double theta[6],
                       double *M_reim);
/* The same split in two: the PSF-and-pixel transfer table T(u,v) (full grid,
 * [v+c][u+c]) and the spectrum from that table. */
void or_transfer_table(int N, double p, const or_psf *psf, double *T);
void or_model_spectrum_t(int N, double p, const double *T, const double theta[6],
                         double *M_reim);
void or_model_spectrum_tp(int N, double p, const double *T, int profile, double nu, const double theta[6],
                          double *M_reim);
/* Inverse DFT of a full Hermitian spectrum to a real N x N image.
 * method 0: separable O(N^3); method 1: direct O(N^4) double sum. */
void or_idft_image(int N, const double *M_reim, double *img, int method);
void or_render(int N, double p, const or_psf *psf, const double theta[6],
               double *img, int method);
/* n stamps of side N (separable method), OpenMP-parallel over stamps. */
void or_render_many(int n, int N, double p, const or_psf *psf, int n_psf, const double *theta,
                    double *img);
/* Brute-force real-space reference: periodic pixel integrals of the
 * exponential convolved with a Gaussian PSF, by midpoint quadrature with
 * nsub x nsub points per pixel and +-nimg periodic images. */
void or_render_realspace_gauss(int N, double p, double psf_fwhm,
                               const double theta[6], int nsub, int nimg,
                               double *img);

/* ---- likelihood and prior --------------------------------------------- */

void or_prior_default(or_prior *pr);
/* Normalised log interim prior density and its gradient (grad may be NULL).
 * Returns -INFINITY outside the support. */
double or_log_prior(const or_prior *pr, const double theta[6], double grad[6]);
double or_log_z_ba14(double alpha);
/* Gaussian pixel log-likelihood -chi^2/(2 sigma^2) (Eq. likelihood-pixels,
 * constant dropped); optional weights w (NULL = uniform) give
 * -1/2 sum w (d-m)^2 / sigma^2. Gradient by the adjoint DFT of the residual. */
double or_loglike(int N, double p, const or_psf *psf, const double *data,
                  const double *w, double sigma, const double theta[6],
                  double grad[6]);
double or_loglike_t(int N, double p, const double *T, const double *data,
                    const double *w, double sigma, const double theta[6],
                    double grad[6]);
/* Appendix C (Eq. covar-pixel-likelihood summed over exposures): J exposures
 * d_j [J][N][N] of one galaxy on one grid, exposure j with PSF psf[j] and
 * pixel covariance Sigma_j = sigma_j^2 C_j, C_j[a][b] = corr_j(x_a - x_b) with
 * the lag wrapped periodically to -c..c (corr [J][N][N], lag (dy, dx) at
 * [dy + c][dx + c], symmetric; NULL: white).  Returns
 *   -1/2 sum_j (d_j - m_j)^T Sigma_j^-1 (d_j - m_j)
 * with Sigma_j built densely in pixel space and solved by Cholesky, and the
 * gradient sum_j (Sigma_j^-1 (d_j - m_j))^T dm_j/dtheta by the adjoint DFT;
 * NAN when some Sigma_j is not positive definite. */
/* Appendix C with a general pixel covariance: -1/2 (d - m)^T Sigma^-1 (d - m)
 * for one exposure, Sigma [N*N][N*N] (row-major over pixels iy*N + ix,
 * symmetric positive definite), solved by Cholesky, and its gradient
 * (Sigma^-1 (d - m))^T dm/dtheta by the adjoint DFT; NAN when Sigma is not
 * positive definite. */
double or_loglike_dense(int N, double p, const or_psf *psf, const double *data, const double *Sigma,
                        const double theta[6], double grad[6]);
double or_loglike_cov(int J, int N, double p, const or_psf *psf, const double *data, const double *sigma,
                      const double *corr, const double theta[6], double grad[6]);
/* Eq. likelihood-pixels with the galaxy profile of Appendix B (profile, nu),
 * gradient by the adjoint DFT of the residual. */
double or_loglike_p(int profile, double nu, int N, double p, const or_psf *psf, const double *data,
                    double sigma, const double theta[6], double grad[6]);
double or_logpost(int N, double p, const or_psf *psf, const double *data,
                  const double *w, double sigma, const or_prior *pr,
                  const double theta[6], double grad[6]);

/* ---- HMC fit (image sampling phase) ------------------------------------ */

/* Warmup window schedule: writes window [start, end) pairs, returns count. */
int or_window_schedule(int n_warmup, int adapt_mass, int *starts, int *ends, int cap);

/* Fit one galaxy with cfg->n_chains chains.
 *   data: N*N, init: [n_chains][6], galaxy_id keys the generator.
 *   samples: [6][n_chains][n_samples] (parameter-major), logp: [n_chains][n_samples],
 *   accept: [n_chains][n_samples] (0/1), accept_rate, step_size, n_div: [n_chains],
 *   inv_mass: [n_chains][6], n_grad: [n_chains] gradient evaluations inside
 *   the prior support.  Any output pointer may be NULL.
 *   init_eps [n_chains] / init_im [n_chains][6] (may be NULL): resume with
 *   this step size (no initial search) and inverse metric.
 *   warm_accept / warm_stat / warm_step [n_chains][n_warmup] (each may be
 *   NULL): accept flags, accept statistics and starting step sizes (before
 *   jitter) of the warmup transitions. */
int or_fit_galaxy(int N, double p, const or_psf *psf, const double *data,
                  const double *w, double sigma, const or_prior *pr,
                  const or_hmc_cfg *cfg, uint64_t galaxy_id, const double *init,
                  double *samples, double *logp, uint8_t *accept,
                  double *accept_rate, double *step_size, int32_t *n_div,
                  double *inv_mass, int32_t *n_grad, const double *init_eps,
                  const double *init_im, uint8_t *warm_accept, double *warm_stat,
                  double *warm_step);

/* Many galaxies of one stamp size, OpenMP-parallel over galaxies (n_threads
 * <= 0: all).  data: [n_gal][N*N], sigma: [n_gal], init: [n_gal][n_chains][6],
 * ids: [n_gal] (NULL: index).  samples: [6][n_gal][n_chains][n_samples],
 * logp/accept: [n_gal][n_chains][n_samples], per-chain outputs [n_gal][n_chains]. */
int or_fit_galaxies(int n_gal, int N, double p, const or_psf *psf, int psf_per_gal,
                    const double *data, const double *sigma, const or_prior *pr,
                    const or_hmc_cfg *cfg, const uint64_t *ids, const double *init,
                    double *samples, double *logp, uint8_t *accept,
                    double *accept_rate, double *step_size, int32_t *n_div,
                    double *inv_mass, int32_t *n_grad, const double *init_eps,
                    const double *init_im, uint8_t *warm_accept, double *warm_stat,
                    double *warm_step, int n_threads);

/* The same sampler (search, dual averaging, windowed metric, transitions) on
 * the Gaussian N(mu, diag(s^2)) over all of R^6: the textbook target on which
 * its adaptation has closed-form expectations.  Chain c is keyed
 * chain_key0 + c; samples [6][n_chains][n_samples], accept_rate, step_size
 * [n_chains], inv_mass [n_chains][6], warm_stat [n_chains][n_warmup] (the
 * accept statistic min(1, e^-dH) of each warmup transition). */
int or_hmc_gauss(const double mu[6], const double s[6], const or_hmc_cfg *cfg,
                 uint64_t chain_key0, const double *init, double *samples,
                 double *accept_rate, double *step_size, double *inv_mass,
                 double *warm_stat);
/* The step-size search (index `search`, from eps0) at position x with
 * inverse metric im on that Gaussian target. */
double or_step_search_gauss(const double mu[6], const double s[6], const double x[6],
                            const double im[6], uint64_t seed, uint64_t key, int search,
                            double eps0);
/* Dual averaging fed the accept statistics a[0..n): log eps and log eps-bar
 * after each update, from a restart at eps0. */
void or_dual_averaging(int n, const double *accept_stat, double delta, double eps0,
                       double *le, double *lebar);

/* ---- diagnostics -------------------------------------------------------- */

/* x: [n_chains][n_samples] for one parameter. Multi-chain ESS with Geyer's
 * initial monotone positive sequence, and classic (non-split) R-hat. */
double or_ess(const double *x, int n_chains, int n_samples);
double or_rhat(const double *x, int n_chains, int n_samples);

/* ---- shear sampling phase ------------------------------------------------ */

/* log of the normaliser of the ellipticity density of each family */
double or_log_z_eprior(int family, double alpha, double trunc_r);
/* log of the (e1, e2) density of the family at |e|^2 = E (-inf off support) */
double or_log_eprior(int family, double alpha, double trunc_r, double e1, double e2);

/* Eq. likelihood-shear (MC estimate, Z_n dropped) with the Jacobian of
 * Eq. true-prior-jacobian-shear.  e1p/e2p: sheared samples [n_gal][K],
 * b: optional per-sample log-weight offsets (NULL = 0), alpha = sigma_e of
 * the true ellipticity density.  Returns the log-likelihood; grad (may be
 * NULL) gets d/d(g1, g2, alpha).  Interim ellipticity prior: BA14 at sigma_e0. */
double or_shear_loglike(const float *e1p, const float *e2p, const float *b,
                        int64_t n_gal, int K, int family, double trunc_r,
                        double sigma_e0, double g1, double g2, double alpha,
                        double grad[3]);

/* The same with per-galaxy weights w[n_gal] (NULL = 1): value and gradient
 * are sum_n w_n [log sum_k w_nk - log K] and its derivatives -- with integer
 * weights, the likelihood of the sample in which galaxy n appears w_n times
 * (the bootstrap of Sec. 3.4's m and c). */
double or_shear_loglike_w(const float *e1p, const float *e2p, const float *b, const float *w,
                          int64_t n_gal, int K, int family, double trunc_r,
                          double sigma_e0, double g1, double g2, double alpha,
                          double grad[3]);
int or_shear_estimate_w(const float *e1p, const float *e2p, const float *b, const float *w,
                        int64_t n_gal, int K, int family, double trunc_r,
                        double sigma_e0, int free_alpha, double alpha_fixed,
                        double alpha_lo, double alpha_hi, int n_gh,
                        double *mean, double *cov);

/* Standard normal log CDF, log Phi(t), stable in both tails. */
double or_log_ndtr(double t);
/* Log density of the skew normal of Eq. lflux-lsize-dist: location mu,
 * scale sigma, shape a: log[2 phi(z) Phi(a z) / sigma], z = (x - mu)/sigma. */
double or_log_skewnorm(double x, double mu, double sigma, double a);

/* Eq. likelihood-shear with every property's true prior (Sec. 3.2 setting
 * with all hyperparameters free): the ellipticity part as or_shear_loglike,
 * times, per sample, SkewNormal(log10 f; mu_f, sigma_f, a_f) N(log10 s; mu_s,
 * sigma_s) over the interim uniforms U(lf_lo, lf_hi) U(ls_lo, ls_hi)
 * (interim = {lf_lo, lf_hi, ls_lo, ls_hi}).  lfp, lsp: log10 flux and log10
 * hlr samples [n_gal][K].  theta = (g1, g2, sigma_e, mu_f, sigma_f, a_f, mu_s,
 * sigma_s); grad (may be NULL) gets the 8 derivatives. */
double or_shear_loglike_full(const float *e1p, const float *e2p, const float *lfp, const float *lsp,
                             int64_t n_gal, int K, int family, double trunc_r, double sigma_e0,
                             const double interim[4], const double theta[8], double grad[8]);
/* The same with per-galaxy weights w[n] (NULL: all 1) on each galaxy's term,
 * as or_shear_loglike_w. */
double or_shear_loglike_full_w(const float *e1p, const float *e2p, const float *lfp, const float *lsp,
                               const float *w, int64_t n_gal, int K, int family, double trunc_r, double sigma_e0,
                               const double interim[4], const double theta[8], double grad[8]);

/* Posterior mean of (g1, g2[, alpha]) under a uniform prior on the unit disk
 * (and alpha ~ U(alpha_lo, alpha_hi) when free_alpha): Newton to the mode on
 * the analytic gradient, then n_gh-point Gauss-Hermite quadrature on the
 * Laplace-scaled grid.  mean: 2 or 3 values; cov (may be NULL): 9 values. */
int or_shear_estimate(const float *e1p, const float *e2p, const float *b,
                      int64_t n_gal, int K, int family, double trunc_r,
                      double sigma_e0, int free_alpha, double alpha_fixed,
                      double alpha_lo, double alpha_hi, int n_gh,
                      double *mean, double *cov);

/* Gauss-Hermite nodes/weights for weight exp(-x^2). */
int or_gauss_hermite(int n, double *x, double *w);

/* Shear transform (Eq. shear-transform) and its inverse; complex in/out. */
void or_shear_apply(double e1, double e2, double g1, double g2, double *o1, double *o2);
void or_shear_invert(double e1p, double e2p, double g1, double g2, double *o1, double *o2);
/* |d eps / d eps'| in closed form. */
double or_shear_jacobian(double e1p, double e2p, double g1, double g2);

#ifdef __cplusplus
}
#endif
#endif
