/*
 * Oracle chain diagnostics (Sec. 4.1): R-hat of Gelman & Rubin (1992), the
 * classic (non-split) potential scale reduction, and the multi-chain effective
 * sample size with Geyer's initial monotone positive sequence as described in
 * Gelman et al., Bayesian Data Analysis (3rd ed.), Sec. 11.5:
 *   W = mean within-chain variance, B/n = variance of chain means,
 *   var+ = (n-1)/n W + B/n,
 *   rho_t = 1 - (W - mean_c acov_c(t)) / var+   (t >= 1; rho_0 = 1),
 *   acov_c(t) = (1/n) sum_{s < n-t} (x_s - xbar_c)(x_{s+t} - xbar_c),
 *   P_k = rho_{2k} + rho_{2k+1} summed while positive and made monotone,
 *   tau = -1 + 2 sum_k P_k,  ESS = m n / tau,
 * with tau floored at 1/log10(m n) (ESS at most m n log10(m n)) so that
 * antithetic chains, whose first pair sum can be near zero, stay finite.
 *
 * TEST INFRASTRUCTURE ONLY (see bs_oracle.h).
 */
#include "bs_oracle.h"

#include <math.h>
#include <stdlib.h>

static void chain_moments(const double *x, int C, int S, double *mean_c,
                          double *W, double *varplus)
{
    double wsum = 0.0, mbar = 0.0;
    for (int c = 0; c < C; ++c) {
        double m = 0.0;
        for (int s = 0; s < S; ++s) m += x[(size_t)c * S + s];
        m /= S;
        double v = 0.0;
        for (int s = 0; s < S; ++s) {
            double d = x[(size_t)c * S + s] - m;
            v += d * d;
        }
        v /= (S - 1);
        mean_c[c] = m;
        wsum += v;
        mbar += m;
    }
    *W = wsum / C;
    mbar /= C;
    double b_over_n = 0.0;
    if (C > 1) {
        for (int c = 0; c < C; ++c) b_over_n += (mean_c[c] - mbar) * (mean_c[c] - mbar);
        b_over_n /= (C - 1);
    }
    *varplus = (S - 1.0) / S * (*W) + b_over_n;
}

double or_rhat(const double *x, int C, int S)
{
    double *mc = malloc(sizeof(double) * C), W, vp;
    chain_moments(x, C, S, mc, &W, &vp);
    free(mc);
    return sqrt(vp / W);
}

double or_ess(const double *x, int C, int S)
{
    double *mc = malloc(sizeof(double) * C), W, vp;
    chain_moments(x, C, S, mc, &W, &vp);
    double *rho = malloc(sizeof(double) * (S + 1));
    rho[0] = 1.0;
    for (int t = 1; t < S; ++t) {
        double acov = 0.0;
        for (int c = 0; c < C; ++c) {
            const double *xc = x + (size_t)c * S;
            double a = 0.0;
            for (int s = 0; s + t < S; ++s) a += (xc[s] - mc[c]) * (xc[s + t] - mc[c]);
            acov += a / S;
        }
        acov /= C;
        rho[t] = 1.0 - (W - acov) / vp;
    }
    rho[S] = 0.0;
    double sum = 0.0, prev = INFINITY;
    for (int k = 0; 2 * k + 1 < S; ++k) {
        double P = rho[2 * k] + rho[2 * k + 1];
        if (!(P > 0.0)) break;
        if (P > prev) P = prev;
        sum += P;
        prev = P;
    }
    double tau = -1.0 + 2.0 * sum;
    double tau_min = 1.0 / log10((double)C * S);
    if (tau < tau_min) tau = tau_min;
    free(mc);
    free(rho);
    return (double)C * S / tau;
}
