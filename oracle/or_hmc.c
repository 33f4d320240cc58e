/*
 * Oracle image-sampling phase (Sec. 3.3): gradient-based MCMC on the interim
 * posterior of Eq. interim-post, one chain per galaxy image and chain index,
 * warmed up by dual averaging of the step size (Nesterov 2009; Hoffman &
 * Gelman 2014 Alg. 5 with the Stan defaults gamma = 0.05, t0 = 10,
 * kappa = 0.75, mu = log(10 eps)).  The sampler is HMC with a fixed number of
 * leapfrog steps L.  Chains start at caller-supplied points (Eq. initialize
 * needs the true parameters, which only the caller has).
 *
 * Algorithm (identical on the CUDA side, which is written independently):
 *   random numbers: Philox4x64-10, key (seed, galaxy_id * n_chains + chain),
 *     counter (i, 0, 0) for the transition at iteration i, counter
 *     (s, 1, t) for trial t of step-size search s; eight 24-bit uniforms per
 *     block; normals by Box-Muller on the pairs (u0,u1), (u2,u3), (u4,u5):
 *     z = sqrt(-2 ln ua) (cos 2 pi ub, sin 2 pi ub).
 *   transition: p = z / sqrt(m), eps_i = eps (1 + jitter (2 u7 - 1)) and
 *     L leapfrog steps, or with random_steps eps_i = eps and
 *     L_i = 1 + floor(u7 L) steps (a randomised integration time that breaks
 *     the resonance of fixed-length trajectories); each step is half kick,
 *     drift, half kick; a position that leaves
 *     the prior support ends the trajectory as divergent; dH = H1 - H0,
 *     H = -log pi + 1/2 sum m p^2; divergent also if dH is not finite or
 *     exceeds 1000; accept statistic a = min(1, e^-dH) (0 if divergent);
 *     accept iff not divergent and ln u6 < -dH.
 *   step-size search: one leapfrog from the current point with a fresh
 *     momentum; if its log acceptance exceeds ln 0.8 double eps until it no
 *     longer does, else halve it until it does; return the last eps tried.
 *   warmup: search (s = 0, eps = 1), dual averaging throughout; with metric
 *     adaptation, in each slow window [start, end) the post-transition
 *     positions feed a Welford variance; at the end of the window the inverse
 *     metric becomes (n/(n+5)) var + 1e-3 (5/(n+5)), a search (s = w + 1)
 *     follows, and dual averaging restarts.  After warmup eps = exp(log eps
 *     bar).  Windows: initial fast buffer 75, first slow window 25 doubling,
 *     final fast buffer 50 (15% / 75% / 10% of the warmup when it is shorter
 *     than 150); the last slow window stretches to the final buffer.
 *
 * TEST INFRASTRUCTURE ONLY (see bs_oracle.h).
 */
#include "bs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846


int or_window_schedule(int n_warmup, int adapt_mass, int *starts, int *ends, int cap)
{
    if (!adapt_mass || n_warmup < 20) return 0;
    int init_buf = 75, term_buf = 50, base = 25;
    if (n_warmup < init_buf + term_buf + base) {
        init_buf = (int)(0.15 * n_warmup);
        term_buf = (int)(0.10 * n_warmup);
        base = n_warmup - init_buf - term_buf;
    }
    int last_end = n_warmup - term_buf;
    int start = init_buf, size = base, n = 0;
    while (n < cap) {
        int end = start + size;
        if (end + 2 * size > last_end) end = last_end;
        starts[n] = start;
        ends[n] = end;
        ++n;
        if (end >= last_end) break;
        start = end;
        size *= 2;
    }
    return n;
}

typedef struct {
    int N;
    double p;
    const double *T;
    const double *data;
    const double *w;
    double sigma;
    const or_prior *pr;
    int *n_eval;            /* evaluations inside the support */
    /* Gaussian test target N(gmu, diag(gs^2)) on all of R^6 instead of the
     * galaxy posterior when gmu != NULL (the textbook case the sampler's
     * adaptation is checked on) */
    const double *gmu, *gs;
} target_t;

/* log posterior and gradient; -inf outside the prior support */
static double target_eval(const target_t *tg, const double th[6], double g[6])
{
    if (tg->gmu) {
        double lp = 0.0;
        for (int i = 0; i < 6; ++i) {
            double z = (th[i] - tg->gmu[i]) / tg->gs[i];
            lp -= 0.5 * z * z;
            g[i] = -z / tg->gs[i];
        }
        ++*tg->n_eval;
        return lp;
    }
    double gp[6];
    double lp = or_log_prior(tg->pr, th, gp);
    if (!isfinite(lp)) return -INFINITY;
    ++*tg->n_eval;
    double ll = or_loglike_t(tg->N, tg->p, tg->T, tg->data, tg->w, tg->sigma, th, g);
    for (int i = 0; i < 6; ++i) g[i] += gp[i];
    return ll + lp;
}

static int in_support(const target_t *tg, const double th[6])
{
    if (tg->gmu) return 1;
    const or_prior *pr = tg->pr;
    double E = th[2] * th[2] + th[3] * th[3];
    return th[0] > pr->lf_lo && th[0] < pr->lf_hi && th[1] > pr->ls_lo && th[1] < pr->ls_hi && E < 1.0;
}

static void normals6(const double u[8], double z[6])
{
    for (int j = 0; j < 3; ++j) {
        double r = sqrt(-2.0 * log(u[2 * j]));
        double a = 2.0 * OR_PI * u[2 * j + 1];
        z[2 * j] = r * cos(a);
        z[2 * j + 1] = r * sin(a);
    }
}

typedef struct {
    double th[6], g[6], lp;
    double im[6];           /* inverse metric (diagonal) */
    double eps;
    /* dual averaging */
    double mu, hbar, lebar;
    int m_da;
} chain_t;

static void da_restart(chain_t *ch)
{
    ch->mu = log(10.0 * ch->eps);
    ch->hbar = 0.0;
    ch->lebar = 0.0;
    ch->m_da = 0;
}

static void da_update(chain_t *ch, double accept_stat, double delta)
{
    const double gamma = 0.05, t0 = 10.0, kappa = 0.75;
    ch->m_da += 1;
    double m = (double)ch->m_da;
    double eta = 1.0 / (m + t0);
    ch->hbar = (1.0 - eta) * ch->hbar + eta * (delta - accept_stat);
    double le = ch->mu - sqrt(m) / gamma * ch->hbar;
    double xe = pow(m, -kappa);
    ch->lebar = xe * le + (1.0 - xe) * ch->lebar;
    ch->eps = exp(le);
}

static double kinetic(const double pm[6], const double im[6])
{
    double k = 0.0;
    for (int i = 0; i < 6; ++i) k += im[i] * pm[i] * pm[i];
    return 0.5 * k;
}

/* One leapfrog trajectory of n steps from (th, g, lp) with momentum pm
 * (updated in place).  Returns 1 if it stayed in the support and finite. */
static int trajectory(const target_t *tg, const chain_t *ch, double eps, int n,
                      double pm[6], double th[6], double g[6], double *lp)
{
    for (int l = 0; l < n; ++l) {
        for (int i = 0; i < 6; ++i) pm[i] += 0.5 * eps * g[i];
        for (int i = 0; i < 6; ++i) th[i] += eps * ch->im[i] * pm[i];
        if (!in_support(tg, th)) return 0;
        *lp = target_eval(tg, th, g);
        if (!isfinite(*lp)) return 0;
        for (int i = 0; i < 6; ++i) pm[i] += 0.5 * eps * g[i];
    }
    return 1;
}

static double search_logacc(const target_t *tg, const chain_t *ch, uint64_t seed,
                            uint64_t key, int s, int t, double eps)
{
    double u[8], z[6], pm[6], th[6], g[6], lp = ch->lp;
    or_uniforms8(seed, key, (uint64_t)s, 1, (uint64_t)t, u);
    normals6(u, z);
    for (int i = 0; i < 6; ++i) pm[i] = z[i] / sqrt(ch->im[i]);
    double H0 = -ch->lp + kinetic(pm, ch->im);
    memcpy(th, ch->th, sizeof th);
    memcpy(g, ch->g, sizeof g);
    if (!trajectory(tg, ch, eps, 1, pm, th, g, &lp)) return -INFINITY;
    double H1 = -lp + kinetic(pm, ch->im);
    double a = H0 - H1;
    return isfinite(a) ? a : -INFINITY;
}

static double step_search(const target_t *tg, const chain_t *ch, uint64_t seed,
                          uint64_t key, int s, double eps)
{
    const double thr = log(0.8);
    double a = search_logacc(tg, ch, seed, key, s, 0, eps);
    int dir = a > thr ? 1 : -1;
    for (int t = 1; t <= 60; ++t) {
        eps = dir > 0 ? 2.0 * eps : 0.5 * eps;
        a = search_logacc(tg, ch, seed, key, s, t, eps);
        if (dir > 0 && !(a > thr)) break;
        if (dir < 0 && a > thr) break;
    }
    return eps;
}

/* HMC transition at iteration i; returns the accept statistic, sets *acc and
 * *div. */
static double transition(const target_t *tg, chain_t *ch, const or_hmc_cfg *cfg,
                         uint64_t key, int i, int *acc, int *div)
{
    double u[8], z[6], pm[6], th[6], g[6];
    or_uniforms8(cfg->seed, key, (uint64_t)i, 0, 0, u);
    normals6(u, z);
    for (int k = 0; k < 6; ++k) pm[k] = z[k] / sqrt(ch->im[k]);
    double eps = ch->eps;
    int nsteps = cfg->n_leapfrog;
    if (cfg->random_steps)
        nsteps = 1 + (int)floor(u[7] * cfg->n_leapfrog);
    else
        eps *= 1.0 + cfg->jitter * (2.0 * u[7] - 1.0);
    double H0 = -ch->lp + kinetic(pm, ch->im);
    memcpy(th, ch->th, sizeof th);
    memcpy(g, ch->g, sizeof g);
    double lp = ch->lp;
    int ok = trajectory(tg, ch, eps, nsteps, pm, th, g, &lp);
    double dH = INFINITY;
    if (ok) {
        dH = (-lp + kinetic(pm, ch->im)) - H0;
        if (!isfinite(dH) || dH > 1000.0) ok = 0;
    }
    *div = !ok;
    if (!ok) { *acc = 0; return 0.0; }
    double a = dH < 0.0 ? 1.0 : exp(-dH);
    *acc = log(u[6]) < -dH;
    if (*acc) {
        memcpy(ch->th, th, sizeof th);
        memcpy(ch->g, g, sizeof g);
        ch->lp = lp;
    }
    return a;
}

/* Outputs of one chain; any pointer may be NULL.  samples: parameter i of
 * draw s at samples[i * sstride + s]; logp, accept: [n_samples];
 * warm_accept / warm_stat / warm_step: [n_warmup] accept flags, accept
 * statistics and starting step sizes (before jitter) of the warmup
 * transitions. */
typedef struct {
    double *samples;
    size_t sstride;
    double *logp;
    uint8_t *accept, *warm_accept;
    double *warm_stat, *warm_step;
    double *accept_rate, *step_size, *inv_mass;
    int32_t *n_div, *n_grad;
} chain_out_t;

/* One chain: initial search, warmup (dual averaging, windowed metric),
 * sampling.  Returns 1 if the start has no finite log density. */
static int run_chain(const target_t *tg, const or_hmc_cfg *cfg, const int *starts,
                     const int *ends, int nw, uint64_t key, const double init[6],
                     const double *init_eps, const double *init_im, const chain_out_t *o)
{
    int S = cfg->n_samples, W = cfg->n_warmup;
    chain_t ch;
    int status = 0;
    *tg->n_eval = 0;
    memcpy(ch.th, init, sizeof ch.th);
    for (int i = 0; i < 6; ++i) ch.im[i] = init_im ? init_im[i] : 1.0;
    ch.lp = target_eval(tg, ch.th, ch.g);
    if (!isfinite(ch.lp)) status = 1;
    if (init_eps)       /* resume an adapted chain: no search */
        ch.eps = *init_eps;
    else
        ch.eps = step_search(tg, &ch, cfg->seed, key, 0, 1.0);
    da_restart(&ch);

    int wi = 0, wn = 0;
    double wmean[6] = {0}, wm2[6] = {0};
    for (int it = 0; it < W; ++it) {
        int acc, div;
        if (o->warm_step) o->warm_step[it] = ch.eps;
        double a = transition(tg, &ch, cfg, key, it, &acc, &div);
        if (o->warm_accept) o->warm_accept[it] = (uint8_t)acc;
        if (o->warm_stat) o->warm_stat[it] = a;
        da_update(&ch, a, cfg->target_accept);
        if (wi < nw && it >= starts[wi] && it < ends[wi]) {
            ++wn;
            for (int i = 0; i < 6; ++i) {
                double d = ch.th[i] - wmean[i];
                wmean[i] += d / wn;
                wm2[i] += d * (ch.th[i] - wmean[i]);
            }
        }
        if (wi < nw && it == ends[wi] - 1) {
            double n = (double)wn;
            for (int i = 0; i < 6; ++i) {
                double var = wm2[i] / (n - 1.0);
                ch.im[i] = (n / (n + 5.0)) * var + 1e-3 * (5.0 / (n + 5.0));
                wmean[i] = 0.0;
                wm2[i] = 0.0;
            }
            wn = 0;
            ch.eps = step_search(tg, &ch, cfg->seed, key, wi + 1, ch.eps);
            da_restart(&ch);
            ++wi;
        }
    }
    if (W > 0) ch.eps = exp(ch.lebar);

    double asum = 0.0;
    int ndiv = 0;
    for (int s = 0; s < S; ++s) {
        int acc, div;
        double a = transition(tg, &ch, cfg, key, W + s, &acc, &div);
        asum += a;
        ndiv += div;
        if (o->samples)
            for (int i = 0; i < 6; ++i) o->samples[(size_t)i * o->sstride + s] = ch.th[i];
        if (o->logp) o->logp[s] = ch.lp;
        if (o->accept) o->accept[s] = (uint8_t)acc;
    }
    if (o->accept_rate) *o->accept_rate = S > 0 ? asum / S : 0.0;
    if (o->step_size) *o->step_size = ch.eps;
    if (o->n_div) *o->n_div = ndiv;
    if (o->inv_mass) memcpy(o->inv_mass, ch.im, sizeof ch.im);
    if (o->n_grad) *o->n_grad = *tg->n_eval;
    return status;
}

int or_fit_galaxy(int N, double p, const or_psf *psf, const double *data,
                  const double *w, double sigma, const or_prior *pr,
                  const or_hmc_cfg *cfg, uint64_t galaxy_id, const double *init,
                  double *samples, double *logp, uint8_t *accept,
                  double *accept_rate, double *step_size, int32_t *n_div,
                  double *inv_mass, int32_t *n_grad, const double *init_eps,
                  const double *init_im, uint8_t *warm_accept, double *warm_stat,
                  double *warm_step)
{
    int C = cfg->n_chains, S = cfg->n_samples, W = cfg->n_warmup;
    double *T = malloc(sizeof(double) * (size_t)N * N);
    or_transfer_table(N, p, psf, T);
    int n_eval = 0;
    target_t tg = {N, p, T, data, w, sigma, pr, &n_eval, NULL, NULL};
    int starts[64], ends[64];
    int nw = or_window_schedule(W, cfg->adapt_mass, starts, ends, 64);
    int status = 0;

    for (int c = 0; c < C; ++c) {
        uint64_t key = galaxy_id * (uint64_t)C + (uint64_t)c;
        chain_out_t o = {
            samples ? samples + (size_t)c * S : NULL, (size_t)C * S,
            logp ? logp + (size_t)c * S : NULL,
            accept ? accept + (size_t)c * S : NULL,
            warm_accept ? warm_accept + (size_t)c * W : NULL,
            warm_stat ? warm_stat + (size_t)c * W : NULL,
            warm_step ? warm_step + (size_t)c * W : NULL,
            accept_rate ? accept_rate + c : NULL,
            step_size ? step_size + c : NULL,
            inv_mass ? inv_mass + 6 * c : NULL,
            n_div ? n_div + c : NULL,
            n_grad ? n_grad + c : NULL};
        if (run_chain(&tg, cfg, starts, ends, nw, key, init + 6 * c,
                      init_eps ? init_eps + c : NULL, init_im ? init_im + 6 * c : NULL, &o))
            status = 1;
    }
    free(T);
    return status;
}

int or_hmc_gauss(const double mu[6], const double s[6], const or_hmc_cfg *cfg,
                 uint64_t chain_key0, const double *init, double *samples,
                 double *accept_rate, double *step_size, double *inv_mass,
                 double *warm_stat)
{
    int C = cfg->n_chains, S = cfg->n_samples, W = cfg->n_warmup;
    int starts[64], ends[64];
    int nw = or_window_schedule(W, cfg->adapt_mass, starts, ends, 64);
    int status = 0;
    for (int c = 0; c < C; ++c) {
        int n_eval = 0;
        target_t tg = {0, 0.0, NULL, NULL, NULL, 0.0, NULL, &n_eval, mu, s};
        chain_out_t o = {
            samples ? samples + (size_t)c * S : NULL, (size_t)C * S, NULL, NULL, NULL,
            warm_stat ? warm_stat + (size_t)c * W : NULL, NULL,
            accept_rate ? accept_rate + c : NULL,
            step_size ? step_size + c : NULL,
            inv_mass ? inv_mass + 6 * c : NULL, NULL, NULL};
        status |= run_chain(&tg, cfg, starts, ends, nw, chain_key0 + (uint64_t)c, init + 6 * c,
                            NULL, NULL, &o);
    }
    return status;
}

double or_step_search_gauss(const double mu[6], const double s[6], const double x[6],
                            const double im[6], uint64_t seed, uint64_t key, int search,
                            double eps0)
{
    int n_eval = 0;
    target_t tg = {0, 0.0, NULL, NULL, NULL, 0.0, NULL, &n_eval, mu, s};
    chain_t ch;
    memcpy(ch.th, x, sizeof ch.th);
    memcpy(ch.im, im, sizeof ch.im);
    ch.lp = target_eval(&tg, ch.th, ch.g);
    return step_search(&tg, &ch, seed, key, search, eps0);
}

void or_dual_averaging(int n, const double *accept_stat, double delta, double eps0,
                       double *le, double *lebar)
{
    chain_t ch;
    ch.eps = eps0;
    da_restart(&ch);
    for (int m = 0; m < n; ++m) {
        da_update(&ch, accept_stat[m], delta);
        le[m] = log(ch.eps);
        lebar[m] = ch.lebar;
    }
}

int or_fit_galaxies(int n_gal, int N, double p, const or_psf *psf, int psf_per_gal,
                    const double *data, const double *sigma, const or_prior *pr,
                    const or_hmc_cfg *cfg, const uint64_t *ids, const double *init,
                    double *samples, double *logp, uint8_t *accept,
                    double *accept_rate, double *step_size, int32_t *n_div,
                    double *inv_mass, int32_t *n_grad, const double *init_eps,
                    const double *init_im, uint8_t *warm_accept, double *warm_stat,
                    double *warm_step, int n_threads)
{
    int C = cfg->n_chains, S = cfg->n_samples, W = cfg->n_warmup;
    size_t NN = (size_t)N * N;
    int bad = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(+ : bad)
#endif
    for (int n = 0; n < n_gal; ++n) {
        double *smp = samples ? malloc(sizeof(double) * 6 * (size_t)C * S) : NULL;
        const or_psf *ps = psf_per_gal ? psf + n : psf;
        uint64_t id = ids ? ids[n] : (uint64_t)n;
        int st = or_fit_galaxy(N, p, ps, data + NN * n, NULL, sigma[n], pr, cfg, id,
                               init + (size_t)n * C * 6, smp,
                               logp ? logp + (size_t)n * C * S : NULL,
                               accept ? accept + (size_t)n * C * S : NULL,
                               accept_rate ? accept_rate + (size_t)n * C : NULL,
                               step_size ? step_size + (size_t)n * C : NULL,
                               n_div ? n_div + (size_t)n * C : NULL,
                               inv_mass ? inv_mass + (size_t)n * C * 6 : NULL,
                               n_grad ? n_grad + (size_t)n * C : NULL,
                               init_eps ? init_eps + (size_t)n * C : NULL,
                               init_im ? init_im + (size_t)n * C * 6 : NULL,
                               warm_accept ? warm_accept + (size_t)n * C * W : NULL,
                               warm_stat ? warm_stat + (size_t)n * C * W : NULL,
                               warm_step ? warm_step + (size_t)n * C * W : NULL);
        bad += st != 0;
        if (smp) {
            /* [6][C][S] -> [6][n_gal][C][S] */
            for (int i = 0; i < 6; ++i)
                memcpy(samples + (((size_t)i * n_gal + n) * C) * S, smp + (size_t)i * C * S,
                       sizeof(double) * (size_t)C * S);
            free(smp);
        }
    }
    return bad;
}
