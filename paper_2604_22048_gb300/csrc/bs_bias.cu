// Multiplicative and additive shear bias by shape-noise cancellation
// (Sec. 3.4).  Two datasets share their galaxies and noise and differ only in
// the applied shear, +g = (|g|, 0) and -g; with their shear estimates g+ and
// g-, the intrinsic shapes cancel in
//     m = (g+_1 - g-_1) / (2 |g|) - 1,   c = (g+_2 + g-_2) / 2.
// The errors are bootstrap standard deviations: a resample draws the n_gal
// galaxies with replacement and applies the same counts to both datasets (the
// image-phase samples are kept, so a resample is the same likelihood with an
// integer weight on each galaxy's term); m and c themselves come from the
// original sample.
//
// Host code only: the estimators are the library's GPU shear estimate
// (bs_shear_estimate) or the mean of the shear sampler's draws
// (bs_shear_sample), or the caller's own (bs_shear_bias_custom).
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bs_device.cuh"
#include "bs_internal.h"

namespace {

// One evaluation source: weights first, then the estimate of either dataset.
struct Estimators {
    virtual ~Estimators() = default;
    virtual bs_status set_weights(const float *w, double wsum) = 0;
    virtual bs_status estimate(int which, double g[2]) = 0;   // 0: +g, 1: -g
};

// Counts of resample r: draw j picks galaxy floor(n x / 2^64), x = word
// (j mod 4) of the Philox4x64-10 block with key (seed, r) and counter
// (floor(j / 4), 0, 1, 0).
void resample_counts(int64_t n, uint64_t seed, uint64_t r, const float *base, std::vector<float> &w)
{
    std::fill(w.begin(), w.end(), 0.0f);
    for (int64_t b = 0; 4 * b < n; ++b) {
        const bs::Philox4x64 x = bs::philox4x64_10((uint64_t)b, 0ull, 1ull, 0ull, seed, r);
        const uint64_t *words = x.w;
        for (int k = 0; k < 4 && 4 * b + k < n; ++k) {
            const uint64_t i = (uint64_t)(((unsigned __int128)words[k] * (uint64_t)n) >> 64);
            w[i] += 1.0f;
        }
    }
    if (base)
        for (int64_t i = 0; i < n; ++i) w[i] *= base[i];
}

bs_status bias_core(int64_t n, Estimators &E, const bs_bias_cfg *cfg, double *out)
{
    const double two_g = 2.0 * cfg->g_abs;
    auto mc = [&](double &m, double &c) -> bs_status {
        double gp[2], gm[2];
        bs_status st = E.estimate(0, gp);
        if (st != BS_OK) return st;
        st = E.estimate(1, gm);
        if (st != BS_OK) return st;
        m = (gp[0] - gm[0]) / two_g - 1.0;
        c = 0.5 * (gp[1] + gm[1]);
        return BS_OK;
    };
    std::vector<float> w;
    try {
        w.resize((size_t)n);
    } catch (const std::bad_alloc &) {
        return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_shear_bias: out of host memory");
    }
    // the original sample (with the base weights, if any)
    double wsum = (double)n;
    if (cfg->base_weight) {
        wsum = 0.0;
        for (int64_t i = 0; i < n; ++i) wsum += cfg->base_weight[i];
    }
    bs_status st = E.set_weights(cfg->base_weight, wsum);
    if (st != BS_OK) return st;
    double m0, c0;
    st = mc(m0, c0);
    if (st != BS_OK) return st;
    // resamples: running means and sums of squared deviations (Welford)
    double mm = 0.0, mc2 = 0.0, cm = 0.0, cc2 = 0.0;
    for (int32_t r = 0; r < cfg->n_boot; ++r) {
        resample_counts(n, cfg->seed, (uint64_t)r, cfg->base_weight, w);
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += w[i];
        st = E.set_weights(w.data(), s);
        if (st != BS_OK) return st;
        double m, c;
        st = mc(m, c);
        if (st != BS_OK) return st;
        if (cfg->m_boot) cfg->m_boot[r] = m;
        if (cfg->c_boot) cfg->c_boot[r] = c;
        const double k = (double)(r + 1);
        const double dm = m - mm, dc = c - cm;
        mm += dm / k;
        cm += dc / k;
        mc2 += dm * (m - mm);
        cc2 += dc * (c - cm);
    }
    out[0] = m0;
    out[1] = c0;
    out[2] = cfg->n_boot > 1 ? std::sqrt(mc2 / (cfg->n_boot - 1)) : NAN;
    out[3] = cfg->n_boot > 1 ? std::sqrt(cc2 / (cfg->n_boot - 1)) : NAN;
    return BS_OK;
}

bs_status check_cfg(int64_t n, const bs_bias_cfg *cfg, const double *out, const char *who)
{
    if (!cfg || !out) return bs::set_error(BS_ERR_INVALID_ARG, "%s: NULL cfg or out", who);
    if (n <= 0) return bs::set_error(BS_ERR_INVALID_ARG, "%s: n_gal must be positive", who);
    if (!(cfg->g_abs > 0.0) || !std::isfinite(cfg->g_abs))
        return bs::set_error(BS_ERR_INVALID_ARG, "%s: g_abs must be positive", who);
    if (cfg->n_boot < 0) return bs::set_error(BS_ERR_INVALID_ARG, "%s: n_boot must be >= 0", who);
    if (cfg->base_weight)
        for (int64_t i = 0; i < n; ++i)
            if (!(cfg->base_weight[i] >= 0.0f) || !std::isfinite(cfg->base_weight[i]))
                return bs::set_error(BS_ERR_INVALID_ARG, "%s: base_weight[%lld] must be finite and >= 0", who,
                                     (long long)i);
    return BS_OK;
}

struct CustomEstimators final : Estimators {
    bs_g_estimator_fn f[2];
    void *user[2];
    const float *w = nullptr;
    double wsum = 0.0;
    bs_status set_weights(const float *ww, double s) override
    {
        w = ww;
        wsum = s;
        return BS_OK;
    }
    bs_status estimate(int which, double g[2]) override
    {
        const int32_t rc = f[which](w, wsum, g, user[which]);
        if (rc != 0)
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias_custom: the %s estimator returned %d",
                                 which ? "-g" : "+g", (int)rc);
        if (!std::isfinite(g[0]) || !std::isfinite(g[1]))
            return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias_custom: the %s estimate is not finite",
                                 which ? "-g" : "+g");
        return BS_OK;
    }
};

struct DeviceEstimators final : Estimators {
    bs_shear_data d[2];
    int32_t method;
    const bs_estimate_cfg *est;
    const bs_shear_sample_cfg *smp;
    float *wdev;
    void *ws;
    size_t wsb;
    void *stream;
    std::vector<double> draws;
    bs_status set_weights(const float *w, double s) override
    {
        for (int k = 0; k < 2; ++k) {
            d[k].gal_weight = w ? wdev : nullptr;
            d[k].gal_weight_sum = w ? s : 0.0;
        }
        if (!w) return BS_OK;
        const cudaError_t e = cudaMemcpyAsync(wdev, w, sizeof(float) * (size_t)d[0].n_gal, cudaMemcpyHostToDevice,
                                              (cudaStream_t)stream);
        if (e != cudaSuccess) return bs::set_error(BS_ERR_CUDA, "bs_shear_bias: weights: %s", cudaGetErrorString(e));
        return BS_OK;
    }
    bs_status estimate(int which, double g[2]) override
    {
        if (method == BS_BIAS_QUADRATURE) {
            double mean[3];
            const bs_status st = bs_shear_estimate(&d[which], est, mean, nullptr, nullptr, ws, wsb, stream);
            if (st != BS_OK) return st;
            g[0] = mean[0];
            g[1] = mean[1];
            return BS_OK;
        }
        const bs_status st = bs_shear_sample(&d[which], smp, draws.data(), nullptr, nullptr, nullptr, ws, wsb, stream);
        if (st != BS_OK) return st;
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < smp->n_samples; ++i) {
            s0 += draws[(size_t)i * 8 + 0];
            s1 += draws[(size_t)i * 8 + 1];
        }
        g[0] = s0 / smp->n_samples;
        g[1] = s1 / smp->n_samples;
        return BS_OK;
    }
};

}  // namespace

extern "C" {

bs_status bs_shear_bias_custom(int64_t n_gal, bs_g_estimator_fn est_plus, void *user_plus,
                               bs_g_estimator_fn est_minus, void *user_minus, const bs_bias_cfg *cfg,
                               double *out)
{
    bs_status st = check_cfg(n_gal, cfg, out, "bs_shear_bias_custom");
    if (st != BS_OK) return st;
    if (!est_plus || !est_minus) return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias_custom: NULL estimator");
    CustomEstimators E;
    E.f[0] = est_plus;
    E.f[1] = est_minus;
    E.user[0] = user_plus;
    E.user[1] = user_minus;
    return bias_core(n_gal, E, cfg, out);
}

bs_status bs_shear_bias(const bs_shear_data *plus, const bs_shear_data *minus, int32_t method,
                        const bs_estimate_cfg *est, const bs_shear_sample_cfg *smp, const bs_bias_cfg *cfg,
                        float *weight_dev, double *out, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!plus || !minus) return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias: NULL dataset");
    bs_status st = check_cfg(plus->n_gal, cfg, out, "bs_shear_bias");
    if (st != BS_OK) return st;
    if (minus->n_gal != plus->n_gal)
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias: the +g and -g datasets must hold the same galaxies");
    if (method == BS_BIAS_QUADRATURE ? !est : (method == BS_BIAS_HMC ? !smp : true))
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias: method must be BS_BIAS_QUADRATURE with est or "
                                                 "BS_BIAS_HMC with smp");
    if (method == BS_BIAS_HMC && smp->n_samples <= 0)
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias: smp->n_samples must be positive");
    if ((cfg->n_boot > 0 || cfg->base_weight) && !weight_dev)
        return bs::set_error(BS_ERR_INVALID_ARG, "bs_shear_bias: weight_dev is required for resamples or base weights");
    DeviceEstimators E;
    E.d[0] = *plus;
    E.d[1] = *minus;
    E.method = method;
    E.est = est;
    E.smp = smp;
    E.wdev = weight_dev;
    E.ws = workspace;
    E.wsb = workspace_bytes;
    E.stream = stream;
    if (method == BS_BIAS_HMC) {
        try {
            E.draws.resize((size_t)smp->n_samples * 8);
        } catch (const std::bad_alloc &) {
            return bs::set_error(BS_ERR_OUT_OF_MEMORY, "bs_shear_bias: out of host memory");
        }
    }
    return bias_core(plus->n_gal, E, cfg, out);
}

}  // extern "C"
