// C ABI of the bpshear library: argument validation, launch configuration,
// the per-galaxy constants of the shear likelihood, and the host-driven
// shear estimate (Newton to the mode, Gauss-Hermite quadrature on the
// Laplace-scaled grid).  See include/bpshear.h for the contract of each call.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "bs_internal.h"

namespace {

thread_local char g_err[512] = "";

bs_status fail(bs_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

bs_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(BS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr double kPi = 3.14159265358979323846;

// log of pi * int_0^1 (1-t)^2 exp(-a t) dt, the normaliser of the
// (1-|e|^2)^2 exp(-|e|^2 / (2 alpha^2)) ellipticity density, a = 1/(2 alpha^2)
double log_z_ba14(double alpha)
{
    const double a = 1.0 / (2.0 * alpha * alpha);
    double z;
    if (a < 1e-2)
        z = 1.0 / 3.0 - a / 12.0 + a * a / 60.0 - a * a * a / 360.0;
    else
        z = 1.0 / a - 2.0 / (a * a) - 2.0 * std::expm1(-a) / (a * a * a);
    return std::log(kPi * z);
}

// d log Z / d alpha for the family
double dlog_z_dalpha(int family, double alpha, double trunc_r)
{
    if (family == BS_EPRIOR_BA14) {
        const double a = 1.0 / (2.0 * alpha * alpha);
        double z, dz;   // without the factor pi
        if (a < 1e-2) {
            z = 1.0 / 3.0 - a / 12.0 + a * a / 60.0;
            dz = -1.0 / 12.0 + a / 30.0 - a * a / 120.0;
        } else {
            const double em = std::expm1(-a), e = std::exp(-a);
            z = 1.0 / a - 2.0 / (a * a) - 2.0 * em / (a * a * a);
            dz = -1.0 / (a * a) + 4.0 / (a * a * a) + 6.0 * em / (a * a * a * a) + 2.0 * e / (a * a * a);
        }
        const double da = -1.0 / (alpha * alpha * alpha);
        return dz * da / z;
    }
    const double x = trunc_r * trunc_r / (2.0 * alpha * alpha);
    return 2.0 / alpha - (trunc_r * trunc_r / (alpha * alpha * alpha)) / std::expm1(x);
}

double log_z_family(int family, double alpha, double trunc_r)
{
    if (family == BS_EPRIOR_BA14) return log_z_ba14(alpha);
    const double x = trunc_r * trunc_r / (2.0 * alpha * alpha);
    return std::log(2.0 * kPi * alpha * alpha) + std::log(-std::expm1(-x));
}

}  // namespace

namespace bs {

// Warmup windows: fast buffer, doubling slow windows, final fast buffer
// (75 / 25... / 50, or 15% / rest / 10% for warmups shorter than 150); the
// last slow window runs up to the final buffer.
int warmup_windows(int W, bool adapt, int *st, int *en, int cap)
{
    if (!adapt || W < 20) return 0;
    int head = 75, tail = 50, len = 25;
    if (W < head + tail + len) {
        head = (int)(0.15 * W);
        tail = (int)(0.10 * W);
        len = W - head - tail;
    }
    const int stop = W - tail;
    int count = 0, s = head;
    while (count < cap) {
        int e = s + len;
        const bool last = e + 2 * len > stop;
        if (last) e = stop;
        st[count] = s;
        en[count] = e;
        ++count;
        if (last || e >= stop) break;
        s = e;
        len *= 2;
    }
    return count;
}

}  // namespace bs

namespace {

using bs::warmup_windows;

bool odd_side_ok(int s) { return s >= 3 && s <= BS_MAX_SIDE && (s & 1); }

}  // namespace

extern "C" {

void bs_prior_default(bs_prior *prior)
{
    if (!prior) return;
    prior->lf_lo = -1.0f;
    prior->lf_hi = 9.0f;
    prior->ls_lo = -2.0f;
    prior->ls_hi = 1.0f;
    prior->sigma_xy = 0.5f;
    prior->sigma_e = 0.3f;
}

const char *bs_last_error(void) { return g_err; }

const char *bs_version(void) { return "bpshear 0.1 (sm_103a)"; }

bs_status bs_render(int32_t n, const float *theta, const float *shear, const int64_t *offsets,
                    const int32_t *side, int32_t max_side, const bs_psf *psf, int32_t n_psf,
                    float pixel_scale, float *out, void *stream)
{
    if (n < 0) return fail(BS_ERR_INVALID_ARG, "bs_render: n < 0");
    if (n == 0) return BS_OK;
    if (!theta || !offsets || !side || !psf || !out)
        return fail(BS_ERR_INVALID_ARG, "bs_render: NULL required pointer");
    if (!odd_side_ok(max_side)) return fail(BS_ERR_INVALID_ARG, "bs_render: max_side %d", max_side);
    if (n_psf != 1 && n_psf != n) return fail(BS_ERR_INVALID_ARG, "bs_render: n_psf must be 1 or n");
    if (!(pixel_scale > 0.f)) return fail(BS_ERR_INVALID_ARG, "bs_render: pixel_scale <= 0");
    cudaError_t e = bs::launch_render(n, theta, shear, offsets, side, max_side, psf, n_psf, pixel_scale,
                                      out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BS_OK : cuda_fail(e, "bs_render");
}

size_t bs_fit_workspace_bytes(const bs_fit_args *args)
{
    (void)args;
    return 256;
}

static bs_status fill_fit_params(const bs_fit_args *a, bs::FitParams &p, const char *who)
{
    if (!a) return fail(BS_ERR_INVALID_ARG, "%s: NULL args", who);
    if (a->n_gal < 0) return fail(BS_ERR_INVALID_ARG, "%s: n_gal < 0", who);
    if (a->n_gal > 0 && (!a->data || !a->offsets || !a->side || !a->psf || !a->noise_sigma))
        return fail(BS_ERR_INVALID_ARG, "%s: NULL required input pointer", who);
    if (a->data_dtype != BS_F32 && a->data_dtype != BS_F64)
        return fail(BS_ERR_INVALID_ARG, "%s: data_dtype", who);
    if (!odd_side_ok(a->max_side)) return fail(BS_ERR_INVALID_ARG, "%s: max_side %d", who, a->max_side);
    if (a->n_exposures < 0 || a->n_exposures > BS_MAX_EXPOSURES)
        return fail(BS_ERR_INVALID_ARG, "%s: n_exposures 0..%d", who, BS_MAX_EXPOSURES);
    const int n_exp = a->n_exposures > 1 ? a->n_exposures : 1;
    if (a->n_psf != 1 && (int64_t)a->n_psf != (int64_t)a->n_gal * n_exp)
        return fail(BS_ERR_INVALID_ARG, "%s: n_psf must be 1 or n_gal x n_exposures", who);
    if (!(a->pixel_scale > 0.f)) return fail(BS_ERR_INVALID_ARG, "%s: pixel_scale", who);
    const bs_prior &pr = a->prior;
    if (!(pr.lf_hi > pr.lf_lo && pr.ls_hi > pr.ls_lo && pr.sigma_xy > 0.f && pr.sigma_e > 0.f))
        return fail(BS_ERR_INVALID_ARG, "%s: prior", who);
    std::memset(&p, 0, sizeof p);
    p.data = a->data;
    p.data_f64 = a->data_dtype == BS_F64;
    p.offsets = a->offsets;
    p.side = a->side;
    p.psf = a->psf;
    p.n_psf = a->n_psf;
    p.sigma = a->noise_sigma;
    p.n_exp = n_exp;
    p.noise_corr = a->noise_corr;
    if (a->profile != BS_PROFILE_EXPONENTIAL && a->profile != BS_PROFILE_SPERGEL && a->profile != BS_PROFILE_GAUSSIAN)
        return fail(BS_ERR_INVALID_ARG, "%s: profile", who);
    if (a->profile == BS_PROFILE_SPERGEL && !(a->spergel_nu >= -0.9f && a->spergel_nu <= 4.0f))
        return fail(BS_ERR_INVALID_ARG, "%s: spergel_nu must be in [-0.9, 4]", who);
    p.profile = a->profile;
    p.prof_c = a->profile == BS_PROFILE_SPERGEL ? 1.0f + a->spergel_nu : a->profile == BS_PROFILE_GAUSSIAN ? 0.5f : 1.5f;
    p.prof_npow = a->profile == BS_PROFILE_SPERGEL ? -(1.0f + a->spergel_nu) : -1.5f;
    p.inv_hlr_r0 = (float)(1.0 / bs::profile_hlr_over_r0(a->profile, a->spergel_nu));
    p.pix_w = a->pixel_weight;
    p.pix_prec = a->pixel_prec;
    p.prec_offs = a->prec_offsets;
    if (a->pixel_prec) {
        if (a->pixel_weight || !a->prec_offsets)
            return fail(BS_ERR_INVALID_ARG, "%s: pixel_prec needs prec_offsets and no pixel_weight", who);
        if (a->profile != BS_PROFILE_EXPONENTIAL || a->n_exposures > 1 || a->noise_corr)
            return fail(BS_ERR_INVALID_ARG,
                        "%s: pixel_prec needs the exponential profile, one exposure and no noise_corr", who);
        if (a->max_side > bs::kDenseMaxSide)
            return fail(BS_ERR_INVALID_ARG, "%s: pixel_prec needs max_side <= %d", who, bs::kDenseMaxSide);
        p.profile = 4;
    } else if (a->pixel_weight) {
        if (a->profile != BS_PROFILE_EXPONENTIAL || n_exp > 1 || a->noise_corr)
            return fail(BS_ERR_INVALID_ARG,
                        "%s: pixel_weight needs the exponential profile, one exposure and no noise_corr", who);
        if (a->max_side > 63) return fail(BS_ERR_INVALID_ARG, "%s: pixel_weight needs max_side <= 63", who);
        p.profile = 3;
    }
    p.gal_id = a->gal_id;
    p.init = a->init;
    p.init_step = a->init_step_size;
    p.init_im = a->init_inv_mass;
    p.n_gal = a->n_gal;
    p.pixel_scale = a->pixel_scale;
    p.lf_lo = pr.lf_lo;
    p.lf_hi = pr.lf_hi;
    p.ls_lo = pr.ls_lo;
    p.ls_hi = pr.ls_hi;
    p.inv_sxy2 = 1.0f / (pr.sigma_xy * pr.sigma_xy);
    p.inv_se2 = 1.0f / (pr.sigma_e * pr.sigma_e);
    const double sxy = pr.sigma_xy;
    p.prior_const = (float)(-std::log((double)pr.lf_hi - pr.lf_lo) - std::log((double)pr.ls_hi - pr.ls_lo) -
                            std::log(2.0 * kPi * sxy * sxy) - log_z_ba14(pr.sigma_e));
    p.max_side = a->max_side;
    p.h_max = (a->max_side + 1) / 2;
    p.npad = 32 * ((a->max_side + 31) / 32);
    if (a->chains_per_cta != 0) {
        if (a->chains_per_cta < 1 || a->chains_per_cta >= a->n_chains || a->n_chains % a->chains_per_cta != 0)
            return fail(BS_ERR_INVALID_ARG, "%s: chains_per_cta must be 0 or a divisor of n_chains below it", who);
        if (p.profile != 0 || n_exp > 1 || a->noise_corr)
            return fail(BS_ERR_INVALID_ARG,
                        "%s: chains_per_cta needs the exponential profile, one exposure and white noise", who);
        p.cpc = a->chains_per_cta;
    }
    if (p.profile == 3) p.cpc = 2;   // the pixel-weight path: two chains per CTA
    return BS_OK;
}

}  // extern "C"

namespace bs {

// Validate a fit request and fill every launch parameter except the
// scheduling fields (work list, counter).
bs_status fit_params_from_args(const bs_fit_args *a, const bs_fit_out *o, FitParams &p, const char *who)
{
    bs_status st = fill_fit_params(a, p, who);
    if (st != BS_OK) return st;
    if (!o) return fail(BS_ERR_INVALID_ARG, "%s: NULL outputs", who);
    if (a->n_gal > 0 && !o->samples) return fail(BS_ERR_INVALID_ARG, "%s: NULL samples output", who);
    if (a->n_gal > 0 && !a->init) return fail(BS_ERR_INVALID_ARG, "%s: NULL init", who);
    if (p.profile == 4 && a->n_chains > 4)
        return fail(BS_ERR_INVALID_ARG, "%s: pixel_prec allows at most 4 chains", who);
    if (a->n_chains < 1 || a->n_chains > bs::kMaxChains)
        return fail(BS_ERR_INVALID_ARG, "%s: n_chains must be 1..%d", who, bs::kMaxChains);
    if (a->n_warmup < 0 || a->n_samples < 0 || a->n_leapfrog < 1)
        return fail(BS_ERR_INVALID_ARG, "%s: n_warmup/n_samples/n_leapfrog", who);
    if (!(a->target_accept > 0.f && a->target_accept < 1.f))
        return fail(BS_ERR_INVALID_ARG, "%s: target_accept", who);
    if (!(a->jitter >= 0.f && a->jitter < 1.f)) return fail(BS_ERR_INVALID_ARG, "%s: jitter", who);
    if (a->registers != 0 && a->registers != 128 && a->registers != 96 && a->registers != 80)
        return fail(BS_ERR_INVALID_ARG, "%s: registers must be 0, 128, 96 or 80", who);
    p.regs = a->registers;
    p.n_chains = a->n_chains;
    p.n_warmup = a->n_warmup;
    p.n_samples = a->n_samples;
    p.n_leapfrog = a->n_leapfrog;
    p.target_accept = a->target_accept;
    p.jitter = a->jitter;
    p.random_steps = a->random_steps ? 1 : 0;
    p.seed = a->seed;
    p.n_windows = warmup_windows(a->n_warmup, a->adapt_mass != 0, p.win_start, p.win_end, bs::kMaxWindows);
    p.samples = o->samples;
    p.logp = o->logp;
    p.accepted = o->accepted;
    p.accept_rate = o->accept_rate;
    p.step_size = o->step_size;
    p.inv_mass = o->inv_mass;
    p.n_div = o->n_divergent;
    p.status = o->status;
    p.n_grad = o->n_grad;
    p.warm_accepted = o->warmup_accepted;
    p.warm_stat = o->warmup_accept_stat;
    p.warm_step = o->warmup_step_size;
    p.work = nullptr;
    p.n_work = a->n_gal;
    p.queue = nullptr;
    return BS_OK;
}

}  // namespace bs

extern "C" {

bs_status bs_fit_galaxies(const bs_fit_args *a, const bs_fit_out *o, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    bs::FitParams p;
    bs_status st = bs::fit_params_from_args(a, o, p, "bs_fit_galaxies");
    if (st != BS_OK) return st;
    if (!workspace || workspace_bytes < bs_fit_workspace_bytes(a))
        return fail(BS_ERR_OUT_OF_MEMORY, "bs_fit_galaxies: workspace of %zu bytes needed",
                    bs_fit_workspace_bytes(a));
    if (a->n_gal == 0) return BS_OK;
    p.queue = static_cast<unsigned int *>(workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (o->status) {
        e = cudaMemsetAsync(o->status, 0, sizeof(int32_t) * (size_t)a->n_gal, s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_fit_galaxies: status reset");
    }
    e = cudaMemsetAsync(workspace, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return cuda_fail(e, "bs_fit_galaxies: queue reset");
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = bs::fit_blocks_per_sm(bs::cta_chains(p), a->max_side, p.regs, p.profile);
    long long grid = (long long)sms * per_sm;
    const long long items = (long long)a->n_gal * bs::cta_groups(p);
    if (grid > items) grid = items;
    e = bs::launch_fit(p, (int)grid, s);
    return e == cudaSuccess ? BS_OK : cuda_fail(e, "bs_fit_galaxies: launch");
}

int32_t bs_fit_resident_galaxies(int32_t n_chains, int32_t max_side, int32_t registers)
{
    if (n_chains < 1 || n_chains > bs::kMaxChains || !odd_side_ok(max_side)) return 0;
    if (registers != 0 && registers != 128 && registers != 96 && registers != 80) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms * bs::fit_blocks_per_sm(n_chains, max_side, registers);
}

bs_status bs_logpost_points(const bs_fit_args *a, int32_t n_points, const int32_t *gal_index,
                            const float *theta, double *logp, float *grad, void *stream)
{
    bs::FitParams p;
    bs_status st = fill_fit_params(a, p, "bs_logpost_points");
    if (st != BS_OK) return st;
    if (n_points < 0) return fail(BS_ERR_INVALID_ARG, "bs_logpost_points: n_points < 0");
    if (n_points == 0) return BS_OK;
    if (!gal_index || !theta) return fail(BS_ERR_INVALID_ARG, "bs_logpost_points: NULL input");
    if (!logp && !grad) return fail(BS_ERR_INVALID_ARG, "bs_logpost_points: no output");
    cudaError_t e = bs::launch_logpost_points(p, n_points, gal_index, theta, logp, grad,
                                              static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BS_OK : cuda_fail(e, "bs_logpost_points");
}

bs_status bs_chain_ess(const float *samples, int32_t n_gal, int32_t n_chains, int32_t n_samples,
                       float *ess, float *rhat, void *stream)
{
    if (!samples || !ess) return fail(BS_ERR_INVALID_ARG, "bs_chain_ess: NULL pointer");
    if (n_gal < 0 || n_chains < 1 || n_chains > bs::kMaxChains || n_samples < 4)
        return fail(BS_ERR_INVALID_ARG, "bs_chain_ess: sizes (n_chains 1..%d, n_samples >= 4)",
                    bs::kMaxChains);
    cudaError_t e = bs::launch_chain_ess(samples, n_gal, n_chains, n_samples, ess, rhat,
                                         static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BS_OK : cuda_fail(e, "bs_chain_ess");
}

bs_status bs_fp32_peak(int32_t packed, double *tflops, void *stream)
{
    if (!tflops) return fail(BS_ERR_INVALID_ARG, "bs_fp32_peak: NULL tflops");
    double t = 0.0;
    const cudaError_t e = bs::measure_fma_peak(packed != 0 ? 1 : 0, t, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "bs_fp32_peak");
    *tflops = t;
    return BS_OK;
}

bs_status bs_fp64_peak(double *tflops, void *stream)
{
    if (!tflops) return fail(BS_ERR_INVALID_ARG, "bs_fp64_peak: NULL tflops");
    double t = 0.0;
    const cudaError_t e = bs::measure_fma_peak(2, t, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "bs_fp64_peak");
    *tflops = t;
    return BS_OK;
}

size_t bs_shear_workspace_bytes(int64_t n_gal, int32_t K)
{
    (void)n_gal;
    (void)K;
    // per-block partials of the 4-output kernel, of the all-free one or of the
    // several-point one, plus the device copy of the results
    const size_t a = (size_t)bs::shear_grid_blocks() * 4, b = (size_t)bs::shear_full_grid_blocks() * bs::kShearFullOut;
    const size_t c = (size_t)bs::shear_multi_grid_blocks() * bs::kMultiPoints * 4;
    size_t m = a > b ? a : b;
    m = m > c ? m : c;
    return (m + 4 * bs::kMultiPoints + bs::kShearFullOut) * sizeof(double);
}

static bs_status validate_shear(const bs_shear_data *d, const char *who)
{
    if (!d) return fail(BS_ERR_INVALID_ARG, "%s: NULL data", who);
    if (d->n_gal < 0 || d->K < 1) return fail(BS_ERR_INVALID_ARG, "%s: n_gal < 0 or K < 1", who);
    if (d->n_gal > 0 && (!d->e1 || !d->e2)) return fail(BS_ERR_INVALID_ARG, "%s: NULL e1/e2", who);
    if (d->family != BS_EPRIOR_BA14 && d->family != BS_EPRIOR_TRUNC_GAUSS)
        return fail(BS_ERR_INVALID_ARG, "%s: family", who);
    if (d->family == BS_EPRIOR_TRUNC_GAUSS && !(d->trunc_r > 0.f && d->trunc_r <= 1.f))
        return fail(BS_ERR_INVALID_ARG, "%s: trunc_r", who);
    if (!(d->sigma_e0 > 0.f)) return fail(BS_ERR_INVALID_ARG, "%s: sigma_e0", who);
    if (d->gal_weight && !(std::isfinite(d->gal_weight_sum) && d->gal_weight_sum >= 0.0))
        return fail(BS_ERR_INVALID_ARG, "%s: gal_weight_sum must be finite and >= 0", who);
    return BS_OK;
}


bs_status bs_shear_loglike(const bs_shear_data *d, double g1, double g2, double alpha, double *out,
                           int32_t out_on_host, void *workspace, size_t workspace_bytes, void *stream)
{
    bs::ShearLaunch L;
    double add[4], alpha_scale = 0.0;
    bs_status st = bs::shear_prepare(d, g1, g2, alpha, L, add, alpha_scale, "bs_shear_loglike");
    if (st != BS_OK) return st;
    if (!out) return fail(BS_ERR_INVALID_ARG, "bs_shear_loglike: NULL out");
    const int grid = bs::shear_grid_blocks();
    const size_t need = (size_t)(grid * 4 + 4) * sizeof(double);
    if (!workspace || workspace_bytes < need)
        return fail(BS_ERR_OUT_OF_MEMORY, "bs_shear_loglike: workspace of %zu bytes needed", need);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = static_cast<double *>(workspace);
    double *dev_out = out_on_host ? partials + (size_t)grid * 4 : out;
    cudaError_t e;
    if (d->n_gal > 0) {
        L.partials = partials;
        e = bs::launch_shear(L, grid, s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike: launch");
        bs::count_launches(1);
    }
    const int n_part = d->n_gal > 0 ? grid : 0;
    e = bs::launch_shear_finalize(partials, n_part, add[0], add[1], add[2], add[3], alpha_scale, dev_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike: finalize");
    bs::count_launches(1);
    if (out_on_host) {
        e = cudaMemcpyAsync(out, dev_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike: copy");
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike: sync");
    }
    return BS_OK;
}

bs_status bs_shear_loglike_multi(const bs_shear_data *d, int32_t n_points, const double *points, double *out,
                                 int32_t out_on_host, void *workspace, size_t workspace_bytes, void *stream)
{
    const char *who = "bs_shear_loglike_multi";
    bs_status st = validate_shear(d, who);
    if (st != BS_OK) return st;
    if (d->b) return fail(BS_ERR_INVALID_ARG, "%s: data->b must be NULL", who);
    if (n_points < 0) return fail(BS_ERR_INVALID_ARG, "%s: n_points < 0", who);
    if (n_points == 0) return BS_OK;
    if (!points || !out) return fail(BS_ERR_INVALID_ARG, "%s: NULL points/out", who);
    constexpr int NP = bs::kMultiPoints;
    const int grid = bs::shear_multi_grid_blocks();
    const size_t need = ((size_t)grid * NP * 4 + 4 * NP) * sizeof(double);
    if (!workspace || workspace_bytes < need)
        return fail(BS_ERR_OUT_OF_MEMORY, "%s: workspace of %zu bytes needed", who, need);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = static_cast<double *>(workspace);
    double *host_stage = partials + (size_t)grid * NP * 4;
    for (int start = 0; start < n_points; start += NP) {
        const int np = n_points - start < NP ? n_points - start : NP;
        bs::ShearMultiLaunch M;
        double add[NP][4], ascale[NP];
        for (int p = 0; p < np; ++p) {
            const double *x = points + 3 * (size_t)(start + p);
            bs::ShearLaunch L;
            st = bs::shear_prepare(d, x[0], x[1], x[2], L, add[p], ascale[p], who);
            if (st != BS_OK) return st;
            if (p == 0) M.s = L;
            M.g1[p] = L.g1;
            M.g2[p] = L.g2;
            M.a2[p] = L.a2;
        }
        for (int p = np; p < NP; ++p) M.g1[p] = M.g2[p] = M.a2[p] = 0.f;
        M.n_points = np;
        M.partials = partials;
        cudaError_t e;
        if (d->n_gal > 0) {
            e = bs::launch_shear_multi(M, grid, s);
            if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_multi: launch");
            bs::count_launches(1);
        }
        const int n_part = d->n_gal > 0 ? grid : 0;
        double *dev_out = out_on_host ? host_stage : out + 4 * (size_t)start;
        for (int p = 0; p < np; ++p) {
            e = bs::launch_shear_finalize(partials + (size_t)p * grid * 4, n_part, add[p][0], add[p][1], add[p][2],
                                          add[p][3], ascale[p], dev_out + 4 * p, s);
            if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_multi: finalize");
            bs::count_launches(1);
        }
        if (out_on_host) {
            e = cudaMemcpyAsync(out + 4 * (size_t)start, host_stage, 4 * np * sizeof(double), cudaMemcpyDeviceToHost,
                                s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_multi: copy");
        }
    }
    return BS_OK;
}

bs_status bs_shear_loglike_full(const bs_shear_data *d, const float *lf, const float *ls, const double interim[4],
                                const double theta[8], double *out, int32_t out_on_host, void *workspace,
                                size_t workspace_bytes, void *stream)
{
    const char *who = "bs_shear_loglike_full";
    if (!theta || !interim || !out) return fail(BS_ERR_INVALID_ARG, "%s: NULL theta/interim/out", who);
    bs::ShearFullLaunch F;
    double add[bs::kShearFullOut], scale[bs::kShearFullOut];
    double alpha_scale = 0.0;
    bs_status st = bs::shear_prepare(d, theta[0], theta[1], theta[2], F.s, add, alpha_scale, who);
    if (st != BS_OK) return st;
    if (d->b) return fail(BS_ERR_INVALID_ARG, "%s: b must be NULL (the flux/size terms are explicit)", who);
    if (d->n_gal > 0 && (!lf || !ls)) return fail(BS_ERR_INVALID_ARG, "%s: NULL lf/ls", who);
    const double mu_f = theta[3], sig_f = theta[4], a_f = theta[5], mu_s = theta[6], sig_s = theta[7];
    if (!(sig_f > 0.0 && sig_s > 0.0 && std::isfinite(mu_f) && std::isfinite(a_f) && std::isfinite(mu_s)))
        return fail(BS_ERR_INVALID_ARG, "%s: sigma_f, sigma_s must be > 0", who);
    if (!(interim[1] > interim[0] && interim[3] > interim[2]))
        return fail(BS_ERR_INVALID_ARG, "%s: interim bounds", who);
    const int grid = bs::shear_full_grid_blocks();
    const size_t need = (size_t)(grid + 1) * bs::kShearFullOut * sizeof(double);
    if (!workspace || workspace_bytes < need)
        return fail(BS_ERR_OUT_OF_MEMORY, "%s: workspace of %zu bytes needed", who, need);
    F.lf = lf;
    F.ls = ls;
    F.mu_f = (float)mu_f;
    F.inv_sf = (float)(1.0 / sig_f);
    F.a_f = (float)a_f;
    F.mu_s = (float)mu_s;
    F.inv_ss = (float)(1.0 / sig_s);
    // the per-galaxy terms at the widths the rounded reciprocals stand for
    // (as shear_prepare does for alpha): one set of parameters for the total
    const double sfe = 1.0 / (double)F.inv_sf, sse = 1.0 / (double)F.inv_ss;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *partials = static_cast<double *>(workspace);
    double *dev_out = out_on_host ? partials + (size_t)grid * bs::kShearFullOut : out;
    cudaError_t e;
    if (d->n_gal > 0) {
        F.s.partials = partials;
        e = bs::launch_shear_full(F, grid, s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_full: launch");
        bs::count_launches(1);
    }
    // per-galaxy constants of the flux/size ratio: log 2 - log sigma_f - log sigma_s
    // - log 2 pi + log of the interim widths (Eq. lflux-lsize-dist over the
    // interim uniforms); d/dsigma of the -log sigma terms
    const double ng = bs::shear_weight_total(d);
    const double kPiD = 3.14159265358979323846;
    add[0] += ng * (std::log(2.0) - std::log(sfe) - std::log(sse) - std::log(2.0 * kPiD) +
                    std::log(interim[1] - interim[0]) + std::log(interim[3] - interim[2]));
    for (int i = 0; i < bs::kShearFullOut; ++i) scale[i] = 1.0;
    scale[0] = 0.6931471805599453;   // log2 -> natural log
    scale[3] = alpha_scale;
    scale[4] = 1.0 / sfe;
    add[4] = 0.0;
    scale[5] = 1.0 / sfe;
    add[5] = -ng / sfe;
    add[6] = 0.0;
    scale[7] = 1.0 / sse;
    add[7] = 0.0;
    scale[8] = 1.0 / sse;
    add[8] = -ng / sse;
    const int n_part = d->n_gal > 0 ? grid : 0;
    e = bs::launch_shear_finalize_n(partials, n_part, bs::kShearFullOut, scale, add, dev_out, s);
    if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_full: finalize");
    bs::count_launches(1);
    if (out_on_host) {
        e = cudaMemcpyAsync(out, dev_out, bs::kShearFullOut * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_full: copy");
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "bs_shear_loglike_full: sync");
    }
    return BS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Shear estimate (host): posterior mean under a uniform prior on the unit disk
// (and a uniform alpha hyperprior), Sec. 3.3-3.4.
// ---------------------------------------------------------------------------
namespace {

struct ShearObjective {
    const bs_shear_data *d;
    const bs_estimate_cfg *cfg;
    void *ws;
    size_t wsb;
    void *stream;
    int n;
    bs_loglike_points_fn fn = nullptr;   // the caller's likelihood instead of the GPU pass
    void *user = nullptr;
    bs_status err = BS_OK;
    int32_t n_evals = 0;

    bool custom(const double *x, int m, double *out)
    {
        if (fn(x, m, out, user) != 0) {
            err = fail(BS_ERR_INVALID_ARG, "bs_shear_estimate_custom: the likelihood callback failed");
            return false;
        }
        return true;
    }
    // value and gradient over (g1, g2[, alpha]); false on failure
    bool eval(const double *x, double &v, double *g)
    {
        const double alpha = n == 3 ? x[2] : cfg->alpha;
        double buf[4];
        ++n_evals;
        bs_status st = BS_OK;
        if (fn) {
            const double pt[3] = {x[0], x[1], alpha};
            if (!custom(pt, 1, buf)) return false;
        } else {
            st = bs_shear_loglike(d, x[0], x[1], alpha, buf, 1, ws, wsb, stream);
        }
        if (st != BS_OK) {
            err = st;
            return false;
        }
        if (cfg->allreduce) cfg->allreduce(buf, cfg->allreduce_user);
        v = buf[0];
        if (g) {
            g[0] = buf[1];
            g[1] = buf[2];
            if (n == 3) g[2] = buf[3];
        }
        return true;
    }
    // values (and gradients, g may be NULL) at m points x[m][3] (alpha in x[.][2]
    // even when it is fixed): several points per pass over the samples, or
    // one pass each when the data carry per-sample offsets b
    bool eval_many(const double *x, int m, double *v, double *g)
    {
        if (m == 0) return true;
        std::vector<double> buf((size_t)4 * m);
        if (fn) {
            if (!custom(x, m, buf.data())) return false;
        } else if (d->b) {
            for (int i = 0; i < m; ++i) {
                bs_status st = bs_shear_loglike(d, x[3 * i], x[3 * i + 1], x[3 * i + 2], &buf[4 * (size_t)i], 1, ws,
                                                wsb, stream);
                if (st != BS_OK) {
                    err = st;
                    return false;
                }
            }
        } else {
            bs_status st = bs_shear_loglike_multi(d, m, x, buf.data(), 1, ws, wsb, stream);
            if (st != BS_OK) {
                err = st;
                return false;
            }
        }
        n_evals += m;
        for (int i = 0; i < m; ++i) {
            double *b4 = &buf[4 * (size_t)i];
            if (cfg->allreduce) cfg->allreduce(b4, cfg->allreduce_user);
            v[i] = b4[0];
            if (g)
                for (int k = 0; k < 3; ++k) g[3 * (size_t)i + k] = b4[1 + k];
        }
        return true;
    }
    bool inside(const double *x) const
    {
        if (!(x[0] * x[0] + x[1] * x[1] < 1.0)) return false;
        if (n == 3 && !(x[2] > cfg->alpha_lo && x[2] < cfg->alpha_hi)) return false;
        return true;
    }
};

// lower Cholesky factor of a symmetric positive-definite n x n matrix
bool chol(const double *A, double *Lo, int n)
{
    for (int i = 0; i < n * n; ++i) Lo[i] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= Lo[i * n + k] * Lo[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                Lo[i * n + i] = std::sqrt(s);
            } else {
                Lo[i * n + j] = s / Lo[j * n + j];
            }
        }
    return true;
}

// Gauss-Hermite rule for weight exp(-x^2): nodes are the zeros of the
// orthonormal Hermite polynomial p_n, bracketed by a sign scan and refined by
// Newton's method; weights are the Christoffel numbers 1 / sum_j p_j(x)^2.
void hermite_rule(int n, double *x, double *w)
{
    auto eval = [n](double t, double &pn, double &pnm1, double &sumsq) {
        double pm = 0.0, p = std::pow(kPi, -0.25);
        sumsq = 0.0;
        for (int j = 0; j < n; ++j) {
            sumsq += p * p;
            const double pn1 = t * std::sqrt(2.0 / (j + 1)) * p - std::sqrt((double)j / (j + 1)) * pm;
            pm = p;
            p = pn1;
        }
        pn = p;
        pnm1 = pm;
    };
    const double lim = std::sqrt(2.0 * n + 1.0) + 1.0;
    const double h = lim / (200.0 * n);
    int found = 0;
    double t0 = -lim, p0, q0, s0;
    eval(t0, p0, q0, s0);
    while (found < n && t0 < lim) {
        const double t1 = t0 + h;
        double p1, q1, s1;
        eval(t1, p1, q1, s1);
        if ((p0 < 0.0) != (p1 < 0.0) || p1 == 0.0) {
            double a = t0, b = t1, fa = p0;
            for (int it = 0; it < 200 && b - a > 1e-15 * (1.0 + std::fabs(a)); ++it) {
                const double m = 0.5 * (a + b);
                double pm_, qm_, sm_;
                eval(m, pm_, qm_, sm_);
                if ((pm_ < 0.0) == (fa < 0.0)) { a = m; fa = pm_; } else { b = m; }
            }
            double r = 0.5 * (a + b);
            for (int it = 0; it < 3; ++it) {   // Newton polish: p_n' = sqrt(2n) p_{n-1}
                double pn, pnm1, ss;
                eval(r, pn, pnm1, ss);
                const double dp = std::sqrt(2.0 * n) * pnm1;
                if (dp != 0.0) r -= pn / dp;
            }
            double pn, pnm1, ss;
            eval(r, pn, pnm1, ss);
            x[found] = r;
            w[found] = 1.0 / ss;
            ++found;
        }
        t0 = t1;
        p0 = p1;
    }
}

}  // namespace

static bs_status shear_estimate_impl(const bs_shear_data *d, const bs_estimate_cfg *cfg, double *mean,
                                     double *cov, int32_t *n_evals, void *workspace, size_t workspace_bytes,
                                     void *stream, bs_loglike_points_fn fn = nullptr, void *user = nullptr)
{
    if (!fn) {
        bs_status st = validate_shear(d, "bs_shear_estimate");
        if (st != BS_OK) return st;
    }
    if (!cfg || !mean) return fail(BS_ERR_INVALID_ARG, "bs_shear_estimate: NULL cfg/mean");
    if (cfg->n_gh < 1 || cfg->n_gh > 32) return fail(BS_ERR_INVALID_ARG, "bs_shear_estimate: n_gh 1..32");
    const int n = cfg->free_alpha ? 3 : 2;
    if (cfg->free_alpha && !(cfg->alpha_lo < cfg->alpha && cfg->alpha < cfg->alpha_hi && cfg->alpha_lo > 0.0))
        return fail(BS_ERR_INVALID_ARG, "bs_shear_estimate: alpha start outside (alpha_lo, alpha_hi)");
    if (!(cfg->alpha > 0.0)) return fail(BS_ERR_INVALID_ARG, "bs_shear_estimate: alpha <= 0");
    ShearObjective f{d, cfg, workspace, workspace_bytes, stream, n, fn, user};
    struct EvalCount {
        int32_t *dst;
        ShearObjective *f;
        ~EvalCount()
        {
            if (dst) *dst = f->n_evals;
        }
    } report{n_evals, &f};
    double x[3] = {0.0, 0.0, cfg->alpha}, g[3], v;
    if (!f.eval(x, v, g)) return f.err;

    // Hessian by central differences of the gradient, the 2n points in one batch
    auto hessian = [&](const double *xc, double *H) -> bool {
        const double h = 1e-5;
        double pts[6][3], vv[6], gg[6][3];
        for (int j = 0; j < n; ++j)
            for (int sgn = 0; sgn < 2; ++sgn) {
                double *q = pts[2 * j + sgn];
                q[0] = xc[0];
                q[1] = xc[1];
                q[2] = n == 3 ? xc[2] : cfg->alpha;
                q[j] += sgn == 0 ? h : -h;
            }
        if (!f.eval_many(&pts[0][0], 2 * n, vv, &gg[0][0])) return false;
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) H[i * n + j] = (gg[2 * j][i] - gg[2 * j + 1][i]) / (2.0 * h);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) H[i * n + j] = H[j * n + i] = 0.5 * (H[i * n + j] + H[j * n + i]);
        return true;
    };

    // Newton ascent with a backtracking line search. The objective is summed
    // from FP32 per-galaxy terms, so its value and gradient carry rounding
    // noise. The Newton decrement g.(-H)^-1 g is the squared length of the
    // step in units of the Laplace posterior width: below 1e-4 (a step under
    // 1% of a standard deviation, where the predicted gain is comparable to
    // the value's rounding noise) the step is taken whole instead of being
    // halved until that noise happens to favour it, and below 1e-10 (the mode
    // known to 1e-5 of a standard deviation, above the gradient's noise
    // floor) the iteration stops.
    double H[9], negH[9], Lo[9];
    bool hess_at_x = false;
    for (int iter = 0; iter < 100; ++iter) {
        if (!hessian(x, H)) return f.err;
        hess_at_x = true;
        for (int i = 0; i < n * n; ++i) negH[i] = -H[i];
        double step[3] = {0, 0, 0}, decrement = INFINITY;
        if (chol(negH, Lo, n)) {
            double y[3];
            for (int i = 0; i < n; ++i) {
                double s = g[i];
                for (int k = 0; k < i; ++k) s -= Lo[i * n + k] * y[k];
                y[i] = s / Lo[i * n + i];
            }
            for (int i = n - 1; i >= 0; --i) {
                double s = y[i];
                for (int k = i + 1; k < n; ++k) s -= Lo[k * n + i] * step[k];
                step[i] = s / Lo[i * n + i];
            }
            decrement = 0.0;
            for (int i = 0; i < n; ++i) decrement += g[i] * step[i];
            if (decrement < 1e-10) break;
        } else {
            for (int i = 0; i < n; ++i) step[i] = 1e-6 * g[i];
        }
        double t = 1.0, xn[3] = {x[0], x[1], x[2]}, vn = -INFINITY, gn[3] = {0, 0, 0};
        bool accepted = false;
        for (int ls = 0; ls < 60 && !accepted; ++ls) {
            for (int i = 0; i < n; ++i) xn[i] = x[i] + t * step[i];
            if (f.inside(xn)) {
                if (!f.eval(xn, vn, gn)) return f.err;
                accepted = decrement < 1e-4 ? std::isfinite(vn) : vn >= v - 1e-10 * std::fabs(v);
            }
            if (!accepted) t *= 0.5;
        }
        if (!accepted) break;   // no ascent along the step: x is the mode to working precision
        double dmax = 0.0;
        for (int i = 0; i < n; ++i) {
            dmax = std::fmax(dmax, std::fabs(t * step[i]));
            x[i] = xn[i];
            g[i] = gn[i];
        }
        v = vn;
        hess_at_x = false;
        if (dmax < 1e-12) break;
    }
    if (!std::isfinite(v))
        return fail(BS_ERR_INVALID_ARG,
                    "bs_shear_estimate: log-likelihood %g at the mode (a galaxy with no sample of non-zero weight "
                    "near it, e.g. every sample beyond the truncation radius): give it weight 0", v);
    if (!hess_at_x && !hessian(x, H)) return f.err;
    // Laplace covariance Sigma = (-H)^-1 and its Cholesky factor
    for (int i = 0; i < n * n; ++i) negH[i] = -H[i];
    if (!chol(negH, Lo, n)) return fail(BS_ERR_UNSUPPORTED, "bs_shear_estimate: posterior not log-concave at the mode");
    double Linv[9] = {0};
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; ++k) s -= Lo[i * n + k] * Linv[k * n + j];
            Linv[i * n + j] = (i < j) ? 0.0 : s / Lo[i * n + i];
        }
    double Sig[9], Lc[9];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += Linv[k * n + i] * Linv[k * n + j];
            Sig[i * n + j] = s;
        }
    if (!chol(Sig, Lc, n)) return fail(BS_ERR_UNSUPPORTED, "bs_shear_estimate: covariance");
    const int q = cfg->n_gh;
    double gx[32], gw[32];
    hermite_rule(q, gx, gw);
    int total = 1;
    for (int i = 0; i < n; ++i) total *= q;
    std::vector<double> lw(total), th((size_t)total * 3), qp, qv;
    std::vector<int> qidx;
    double lmax = -INFINITY;
    for (int j = 0; j < total; ++j) {
        int r = j;
        double z[3] = {0, 0, 0}, logw = 0.0, zz = 0.0;
        for (int i = 0; i < n; ++i) {
            const int a = r % q;
            r /= q;
            z[i] = gx[a];
            logw += std::log(gw[a]);
            zz += z[i] * z[i];
        }
        double *tj = &th[(size_t)j * 3];
        tj[2] = cfg->alpha;
        for (int i = 0; i < n; ++i) {
            double s = x[i];
            for (int k = 0; k <= i; ++k) s += std::sqrt(2.0) * Lc[i * n + k] * z[k];
            tj[i] = s;
        }
        if (!f.inside(tj)) {
            lw[j] = -INFINITY;
            continue;
        }
        lw[j] = logw + zz;      // + (value - v) once the batch is evaluated
        qidx.push_back(j);
        qp.insert(qp.end(), {tj[0], tj[1], tj[2]});
    }
    // the nodes inside the support in batches of several points per pass
    qv.resize(qidx.size());
    if (!f.eval_many(qp.data(), (int)qidx.size(), qv.data(), nullptr)) return f.err;
    for (size_t q = 0; q < qidx.size(); ++q) {
        const int j = qidx[q];
        lw[j] += qv[q] - v;
        if (lw[j] > lmax) lmax = lw[j];
    }
    double wsum = 0.0, m[3] = {0, 0, 0};
    for (int j = 0; j < total; ++j) {
        const double wj = std::exp(lw[j] - lmax);
        wsum += wj;
        for (int i = 0; i < n; ++i) m[i] += wj * th[(size_t)j * 3 + i];
    }
    for (int i = 0; i < 3; ++i) mean[i] = (i < n) ? m[i] / wsum : cfg->alpha;
    if (cov) {
        for (int i = 0; i < 9; ++i) cov[i] = 0.0;
        for (int j = 0; j < total; ++j) {
            const double wj = std::exp(lw[j] - lmax) / wsum;
            for (int a = 0; a < n; ++a)
                for (int c = 0; c < n; ++c)
                    cov[a * 3 + c] += wj * (th[(size_t)j * 3 + a] - mean[a]) * (th[(size_t)j * 3 + c] - mean[c]);
        }
    }
    return BS_OK;
}

extern "C" bs_status bs_shear_estimate(const bs_shear_data *d, const bs_estimate_cfg *cfg, double *mean,
                                       double *cov, int32_t *n_evals, void *workspace,
                                       size_t workspace_bytes, void *stream)
{
    // no C++ exception crosses the C ABI: a failed host allocation is reported
    try {
        return shear_estimate_impl(d, cfg, mean, cov, n_evals, workspace, workspace_bytes, stream);
    } catch (const std::bad_alloc &) {
        return fail(BS_ERR_OUT_OF_MEMORY, "bs_shear_estimate: host allocation failed");
    }
}

extern "C" bs_status bs_shear_estimate_custom(bs_loglike_points_fn fn, void *user, const bs_estimate_cfg *cfg,
                                              double *mean, double *cov, int32_t *n_evals)
{
    if (!fn) return fail(BS_ERR_INVALID_ARG, "bs_shear_estimate_custom: NULL likelihood");
    try {
        return shear_estimate_impl(nullptr, cfg, mean, cov, n_evals, nullptr, 0, nullptr, fn, user);
    } catch (const std::bad_alloc &) {
        return fail(BS_ERR_OUT_OF_MEMORY, "bs_shear_estimate_custom: host allocation failed");
    }
}

namespace bs {

bs_status set_error(bs_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

// Number of galaxies the per-galaxy constants count: the weight sum when
// galaxies carry weights.
namespace {
std::atomic<unsigned long long> g_kernel_launches{0};   // one process-wide count
thread_local unsigned long long *tl_capture_tally = nullptr;
}  // namespace

void count_launches(unsigned long long n)
{
    if (tl_capture_tally)
        *tl_capture_tally += n;
    else
        g_kernel_launches.fetch_add(n, std::memory_order_relaxed);
}

void capture_launches(unsigned long long *tally) { tl_capture_tally = tally; }

unsigned long long kernel_launches_total() { return g_kernel_launches.load(std::memory_order_relaxed); }

double shear_weight_total(const bs_shear_data *d)
{
    return d->gal_weight ? d->gal_weight_sum : (double)d->n_gal;
}

bs_status shear_prepare(const bs_shear_data *d, double g1, double g2, double alpha, ShearLaunch &L,
                        double add[4], double &alpha_scale, const char *who)
{
    bs_status st = validate_shear(d, who);
    if (st != BS_OK) return st;
    const double gg = g1 * g1 + g2 * g2;
    if (!(gg < 1.0)) return fail(BS_ERR_INVALID_ARG, "%s: |g| >= 1", who);
    if (!(alpha > 0.0)) return fail(BS_ERR_INVALID_ARG, "%s: alpha <= 0", who);
    L.e1 = d->e1;
    L.e2 = d->e2;
    L.b = d->b;
    L.w = d->gal_weight;
    L.n_gal = d->n_gal;
    L.K = d->K;
    L.family = d->family;
    L.g1 = (float)g1;
    L.g2 = (float)g2;
    L.a2 = (float)(1.4426950408889634 / (2.0 * alpha * alpha));
    if (!(L.a2 > 0.0f) || !std::isfinite(L.a2)) return fail(BS_ERR_INVALID_ARG, "%s: alpha %g out of range", who, alpha);
    L.kappa = d->family == BS_EPRIOR_BA14 ? 4.0f : 2.0f;
    L.c0 = (float)(1.4426950408889634 / (2.0 * (double)d->sigma_e0 * d->sigma_e0));
    L.r2 = d->trunc_r * d->trunc_r;
    L.partials = nullptr;
    // The per-sample terms see g and 1/(2 alpha^2) rounded to FP32; the
    // per-galaxy constants are taken at the same rounded values, so that the
    // total is the likelihood at one (g, alpha), a smooth function of it.
    // With alpha itself here, the constant and the samples' exponent would
    // stand for two alphas whose difference jumps with every rounding step
    // of a2: by the rounding of a2 (2^-24 relative) times the samples'
    // a2 Q, a shift of order 0.01 nat at 10^6 x 300 samples.
    const double ge1 = (double)L.g1, ge2 = (double)L.g2, gge = ge1 * ge1 + ge2 * ge2;
    if (!(gge < 1.0)) return fail(BS_ERR_INVALID_ARG, "%s: |g| >= 1 in FP32", who);
    const double ae = std::sqrt(1.4426950408889634 / (2.0 * (double)L.a2));
    const double ng = shear_weight_total(d);
    const double kap = d->family == BS_EPRIOR_BA14 ? 4.0 : 2.0;
    add[0] = ng * (kap * std::log1p(-gge) - log_z_family(d->family, ae, d->trunc_r) +
                   log_z_ba14(d->sigma_e0) - std::log((double)d->K));
    add[1] = ng * (-2.0 * kap * ge1 / (1.0 - gge));
    add[2] = ng * (-2.0 * kap * ge2 / (1.0 - gge));
    add[3] = -ng * dlog_z_dalpha(d->family, ae, d->trunc_r);
    alpha_scale = 1.0 / (ae * ae * ae);
    return BS_OK;
}

}  // namespace bs

extern "C" uint64_t bs_kernel_launches(void) { return bs::kernel_launches_total(); }
