// Shear sampling phase as MCMC (Sec. 3.2, "Shear Sampling Phase"): HMC on the
// shear g and any chosen hyperparameters of the true galaxy prior, with the
// likelihood of Eq. likelihood-shear evaluated on the GPU at every leapfrog
// step (bs_shear_loglike, or bs_shear_loglike_full when log-flux and log-size
// samples are given), a uniform prior on the unit disk for g and uniform
// hyperpriors (Sec. 3.3).
//
// The chain runs on the host in FP64: one GPU likelihood-and-gradient pass per
// leapfrog step (plus an optional all-reduce of its 9 doubles over ranks).
// Sampler: HMC with a diagonal metric; dual averaging of the step size
// (Hoffman & Gelman 2014, gamma 0.05, t0 10, kappa 0.75, target delta);
// Stan-style metric windows; a doubling/halving step-size search at the start
// and after each window; random trajectory lengths L_i ~ U{1..L} or a fixed L;
// proposals outside the prior support are rejected as divergent.  Random
// numbers: Philox4x64-10 keyed by (seed, 0), counter (iteration, block, 0).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bs_device.cuh"
#include "bs_internal.h"

namespace {

constexpr int kP = 8;   // g1, g2, sigma_e, mu_f, sigma_f, a_f, mu_s, sigma_s

struct ShearTarget {
    const bs_shear_data *d;
    const bs_shear_sample_cfg *cfg;
    bool full;
    int nf;
    int idx[kP];          // free parameter i -> theta index
    void *ws;
    size_t wsb;
    cudaStream_t stream;
    int n_evals = 0;

    // log posterior at the free coordinates q and its gradient; -inf outside
    // the prior support
    bs_status eval(const double *q, double &lp, double *grad)
    {
        double th[kP];
        std::memcpy(th, cfg->theta0, sizeof th);
        for (int i = 0; i < nf; ++i) th[idx[i]] = q[i];
        lp = -INFINITY;
        if (!(th[0] * th[0] + th[1] * th[1] < 1.0)) return BS_OK;
        for (int i = 2; i < nf; ++i) {
            const int k = idx[i];
            if (!(th[k] > cfg->lo[k] && th[k] < cfg->hi[k])) return BS_OK;
        }
        double out[bs::kShearFullOut];
        bs_status st;
        if (full) {
            st = bs_shear_loglike_full(d, cfg->lf, cfg->ls, cfg->interim, th, out, 1, ws, wsb, stream);
        } else {
            st = bs_shear_loglike(d, th[0], th[1], th[2], out, 1, ws, wsb, stream);
            for (int k = 4; k < bs::kShearFullOut; ++k) out[k] = 0.0;
        }
        if (st != BS_OK) return st;
        ++n_evals;
        if (cfg->allreduce) {
            // ranks sum value and gradient: 4 doubles per call of the hook
            cfg->allreduce(out, cfg->allreduce_user);
            if (full) {
                cfg->allreduce(out + 4, cfg->allreduce_user);
                double tail[4] = {out[8], 0.0, 0.0, 0.0};
                cfg->allreduce(tail, cfg->allreduce_user);
                out[8] = tail[0];
            }
        }
        lp = out[0];
        for (int i = 0; i < nf; ++i) grad[i] = out[1 + idx[i]];
        return BS_OK;
    }
};

// Uniforms in (0, 1) (53-bit) from one Philox block.
void uniforms4(uint64_t seed, uint64_t it, uint64_t blk, double u[4])
{
    const bs::Philox4x64 r = bs::philox4x64_10(it, blk, 0, 0, seed, 0);
    for (int j = 0; j < 4; ++j) u[j] = ((double)(r.w[j] >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// nf standard normals (Box-Muller) for iteration it, stream slot blk0.. .
void normals(uint64_t seed, uint64_t it, uint64_t blk0, int nf, double *z)
{
    const double kTwoPi = 6.283185307179586;
    for (int i = 0; i < nf; i += 4) {
        double u[4];
        uniforms4(seed, it, blk0 + (uint64_t)(i / 4), u);
        for (int j = 0; j < 4 && i + j < nf; j += 2) {
            const double r = std::sqrt(-2.0 * std::log(u[j]));
            z[i + j] = r * std::cos(kTwoPi * u[j + 1]);
            if (i + j + 1 < nf) z[i + j + 1] = r * std::sin(kTwoPi * u[j + 1]);
        }
    }
}

struct Hmc {
    ShearTarget &T;
    int nf;
    std::vector<double> q, g, im;
    double lp = -INFINITY;

    explicit Hmc(ShearTarget &t) : T(t), nf(t.nf), q(t.nf), g(t.nf), im(t.nf, 1.0) {}

    // One trajectory from (q, p) with step eps and nst steps; returns the
    // proposal's (q, g, lp) and whether it stayed finite inside the support.
    bs_status trajectory(std::vector<double> &qp, std::vector<double> &gp, double &lpp, std::vector<double> &p,
                         double eps, int nst, bool &ok)
    {
        qp = q;
        gp = g;
        lpp = lp;
        ok = true;
        for (int l = 0; l < nst; ++l) {
            for (int i = 0; i < nf; ++i) p[i] += 0.5 * eps * gp[i];
            for (int i = 0; i < nf; ++i) qp[i] += eps * im[i] * p[i];
            bs_status st = T.eval(qp.data(), lpp, gp.data());
            if (st != BS_OK) return st;
            if (!std::isfinite(lpp)) {
                ok = false;
                return BS_OK;
            }
            for (int i = 0; i < nf; ++i) p[i] += 0.5 * eps * gp[i];
        }
        return BS_OK;
    }

    double kinetic(const std::vector<double> &p) const
    {
        double k = 0.0;
        for (int i = 0; i < nf; ++i) k += im[i] * p[i] * p[i];
        return 0.5 * k;
    }
};

}  // namespace

extern "C" {

void bs_shear_hyperprior_default(double lo[8], double hi[8])
{
    // Sec. 3.3: sigma_e ~ U(1e-4, 1), mu_f ~ U(-2, 6), sigma_f ~ U(0, 2),
    // a_f ~ U(-100, 100), mu_s ~ U(-2, 2), sigma_s ~ U(0, 0.5); g on the unit disk
    const double l[8] = {-1.0, -1.0, 1e-4, -2.0, 0.0, -100.0, -2.0, 0.0};
    const double h[8] = {1.0, 1.0, 1.0, 6.0, 2.0, 100.0, 2.0, 0.5};
    if (lo) std::memcpy(lo, l, sizeof l);
    if (hi) std::memcpy(hi, h, sizeof h);
}

}  // extern "C"

namespace {

bs_status shear_sample_impl(const bs_shear_data *d, const bs_shear_sample_cfg *cfg, double *samples,
                            double *accept_rate, double *step_size, int32_t *n_evals, void *workspace,
                            size_t workspace_bytes, void *stream)
{
    const char *who = "bs_shear_sample";
    if (!d || !cfg || !samples) return bs::set_error(BS_ERR_INVALID_ARG, "%s: NULL argument", who);
    if ((cfg->free_mask & 3u) != 3u || (cfg->free_mask >> kP) != 0u)
        return bs::set_error(BS_ERR_INVALID_ARG, "%s: free_mask must contain g1, g2 (bits 0, 1) and no bit >= 8", who);
    const bool full = cfg->lf != nullptr || cfg->ls != nullptr;
    if (!full && (cfg->free_mask & ~7u))
        return bs::set_error(BS_ERR_INVALID_ARG, "%s: flux/size hyperparameters need lf and ls", who);
    if (full && (!cfg->lf || !cfg->ls)) return bs::set_error(BS_ERR_INVALID_ARG, "%s: lf and ls go together", who);
    if (cfg->n_warmup < 0 || cfg->n_samples < 1 || cfg->n_leapfrog < 1)
        return bs::set_error(BS_ERR_INVALID_ARG, "%s: n_warmup / n_samples / n_leapfrog", who);
    if (!(cfg->target_accept > 0.f && cfg->target_accept < 1.f))
        return bs::set_error(BS_ERR_INVALID_ARG, "%s: target_accept", who);
    ShearTarget T;
    T.d = d;
    T.cfg = cfg;
    T.full = full;
    T.nf = 0;
    for (int k = 0; k < kP; ++k)
        if (cfg->free_mask & (1u << k)) T.idx[T.nf++] = k;
    T.ws = workspace;
    T.wsb = workspace_bytes;
    T.stream = static_cast<cudaStream_t>(stream);
    Hmc H(T);
    for (int i = 0; i < T.nf; ++i) H.q[i] = cfg->theta0[T.idx[i]];
    bs_status st = T.eval(H.q.data(), H.lp, H.g.data());
    if (st != BS_OK) return st;
    if (!std::isfinite(H.lp)) return bs::set_error(BS_ERR_INVALID_ARG, "%s: theta0 outside the prior support", who);

    const int W = cfg->n_warmup, S = cfg->n_samples, L = cfg->n_leapfrog, nf = T.nf;
    int ws_[bs::kMaxWindows], we_[bs::kMaxWindows];
    const int n_win = bs::warmup_windows(W, true, ws_, we_, bs::kMaxWindows);
    const double delta = cfg->target_accept, thr_search = std::log(0.8);
    std::vector<double> p(nf), qp(nf), gp(nf), wmean(nf, 0.0), wm2(nf, 0.0);
    double lpp = 0.0, eps = 1.0, da_mu = 0.0, da_hbar = 0.0, da_lebar = 0.0, asum = 0.0;
    int da_m = 0, wn = 0, wi = 0;
    uint64_t search_id = 0;

    // step-size search from eps (Stan's heuristic: double or halve until the
    // one-step acceptance crosses 0.8)
    auto search = [&](double e0) -> bs_status {
        double e = e0;
        int dir = 0;
        for (int t = 0; t <= 60; ++t) {
            normals(cfg->seed, search_id, 1000 + (uint64_t)t * 4, nf, p.data());
            for (int i = 0; i < nf; ++i) p[i] /= std::sqrt(H.im[i]);
            const double h0 = -H.lp + H.kinetic(p);
            bool ok;
            bs_status s2 = H.trajectory(qp, gp, lpp, p, e, 1, ok);
            if (s2 != BS_OK) return s2;
            const double la = ok ? -((-lpp + H.kinetic(p)) - h0) : -INFINITY;
            const bool good = la > thr_search;
            if (t == 0)
                dir = good ? 1 : -1;
            else if ((dir > 0 && !good) || (dir < 0 && good))
                break;
            e = dir > 0 ? 2.0 * e : 0.5 * e;
        }
        ++search_id;
        eps = e;
        da_mu = std::log(10.0 * eps);
        da_hbar = 0.0;
        da_lebar = 0.0;
        da_m = 0;
        return BS_OK;
    };
    st = search(0.1);
    if (st != BS_OK) return st;

    for (int it = 0; it < W + S; ++it) {
        double u[4];
        uniforms4(cfg->seed, (uint64_t)it, 0, u);
        normals(cfg->seed, (uint64_t)it, 1, nf, p.data());
        for (int i = 0; i < nf; ++i) p[i] /= std::sqrt(H.im[i]);
        int nst = L;
        double e_use = eps;
        if (cfg->random_steps)
            nst = 1 + (int)(u[1] * L);
        const double h0 = -H.lp + H.kinetic(p);
        bool ok;
        st = H.trajectory(qp, gp, lpp, p, e_use, nst, ok);
        if (st != BS_OK) return st;
        double dH = INFINITY;
        if (ok) {
            dH = (-lpp + H.kinetic(p)) - h0;
            if (!std::isfinite(dH) || dH > 1000.0) ok = false;
        }
        const double a = ok ? (dH < 0.0 ? 1.0 : std::exp(-dH)) : 0.0;
        if (ok && std::log(u[0]) < -dH) {
            H.q = qp;
            H.g = gp;
            H.lp = lpp;
        }
        if (it < W) {
            da_m += 1;
            const double m = (double)da_m, eta = 1.0 / (m + 10.0);
            da_hbar = (1.0 - eta) * da_hbar + eta * (delta - a);
            const double le = da_mu - std::sqrt(m) / 0.05 * da_hbar;
            const double xe = std::pow(m, -0.75);
            da_lebar = xe * le + (1.0 - xe) * da_lebar;
            eps = std::exp(le);
            if (wi < n_win && it >= ws_[wi] && it < we_[wi]) {
                ++wn;
                for (int i = 0; i < nf; ++i) {
                    const double dd = H.q[i] - wmean[i];
                    wmean[i] += dd / wn;
                    wm2[i] += dd * (H.q[i] - wmean[i]);
                }
            }
            if (wi < n_win && it == we_[wi] - 1) {
                const double n = (double)wn;
                for (int i = 0; i < nf; ++i) {
                    H.im[i] = (n / (n + 5.0)) * (wm2[i] / (n - 1.0)) + 1e-3 * (5.0 / (n + 5.0));
                    wmean[i] = wm2[i] = 0.0;
                }
                wn = 0;
                ++wi;
                st = search(eps);
                if (st != BS_OK) return st;
            }
            if (it == W - 1) eps = std::exp(da_lebar);
        } else {
            asum += a;
            double *row = samples + (size_t)(it - W) * kP;
            std::memcpy(row, cfg->theta0, sizeof(double) * kP);
            for (int i = 0; i < nf; ++i) row[T.idx[i]] = H.q[i];
        }
    }
    if (accept_rate) *accept_rate = asum / S;
    if (step_size) *step_size = eps;
    if (n_evals) *n_evals = T.n_evals;
    return BS_OK;
}

}  // namespace

extern "C" {

bs_status bs_shear_sample(const bs_shear_data *d, const bs_shear_sample_cfg *cfg, double *samples,
                          double *accept_rate, double *step_size, int32_t *n_evals, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    // no C++ exception crosses the C ABI: a failed host allocation is reported
    try {
        return shear_sample_impl(d, cfg, samples, accept_rate, step_size, n_evals, workspace, workspace_bytes,
                                 stream);
    } catch (const std::bad_alloc &) {
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_shear_sample: host allocation failed");
    }
}

}  // extern "C"
