// Host/device shared definitions of the bpshear kernels (not part of the ABI).
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/bpshear.h"

namespace bs {

constexpr int kMaxChains = 8;
constexpr int kMaxWindows = 24;
constexpr int kDenseMaxSide = 31;   // largest stamp with a general pixel covariance

// Everything one fit launch needs, filled by the C-ABI layer.
struct FitParams {
    // inputs
    const void *data;
    int data_f64;
    const int64_t *offsets;
    const int32_t *side;
    const bs_psf *psf;
    int n_psf;
    const float *sigma;
    int n_exp;                 // exposures per galaxy (>= 1)
    const float *noise_corr;   // per-exposure noise correlation (layout of data) or NULL
    int profile;               // BS_PROFILE_*
    float prof_c;              // -d log f / d s = prof_c psi(s): 1 + nu (Spergel), 1/2 (Gaussian)
    float prof_npow;           // -(1 + nu) (Spergel)
    float inv_hlr_r0;          // r0 / hlr of the profile
    const float *pix_w;        // per-pixel weights (layout of data) or NULL; profile 3 when set
    const float *pix_prec;     // per-galaxy precision Sigma^-1 [N^2][N^2] at prec_offs[gal], or NULL;
    const int64_t *prec_offs;  // profile 4 when set (the pixel-space kernel with a dense covariance)
    const uint64_t *gal_id;
    const float *init;
    const float *init_step;
    const float *init_im;
    int n_gal;
    float pixel_scale;
    // interim prior
    float lf_lo, lf_hi, ls_lo, ls_hi, inv_sxy2, inv_se2;
    float prior_const;   // log of the prior's normalising constants
    // sampler
    int n_chains, n_warmup, n_samples, n_leapfrog;
    float target_accept, jitter;
    int random_steps;
    uint64_t seed;
    int n_windows;
    int win_start[kMaxWindows], win_end[kMaxWindows];
    // outputs
    float *samples;
    float *logp;
    uint8_t *accepted;
    float *accept_rate;
    float *step_size;
    float *inv_mass;
    int32_t *n_div;
    int32_t *status;
    int32_t *n_grad;
    uint8_t *warm_accepted;
    float *warm_stat;
    float *warm_step;
    // scheduling: the CTAs take positions 0..n_work-1 of `work` (galaxy
    // indices; NULL = identity) from the atomic counter `queue`
    const int32_t *work;
    int n_work;
    unsigned int *queue;
    int max_side;
    int h_max, npad;   // shared-memory geometry for max_side
    int cpc;           // chains per CTA (0: all n_chains): a galaxy's chains may be split
                       // over n_chains / cpc CTAs, each staging the galaxy itself
    int regs;          // register cap of the kernel instance (128, 96 or 80;
                       // 0 = default)
    // serving: when `done` is set (host-mapped), each CTA copies its galaxy's
    // outputs to (address + pub_shift) -- the pinned mirror of the output
    // arrays -- then sets done[gal] = 1 with a system-scope fence before it
    uint32_t *done;
    long long pub_shift;
};

// Chains (warps) of one CTA of a fit launch.
__host__ __device__ inline int cta_chains(const FitParams &p) { return p.cpc > 0 ? p.cpc : p.n_chains; }
// CTAs a galaxy's chains are split over (the pixel-weight path: pairs of chains, the
// last one alone for an odd count).
__host__ __device__ inline int cta_groups(const FitParams &p)
{
    return p.profile == 3 ? (p.n_chains + 1) / 2 : p.n_chains / cta_chains(p);
}

// Shared memory bytes per CTA for a given max stamp side and chains per galaxy.
size_t fit_smem_bytes(int max_side, int n_chains);
// Launch helpers implemented in the .cu files.
cudaError_t launch_fit(const FitParams &p, int grid, cudaStream_t stream);
int fit_blocks_per_sm(int n_chains, int max_side, int regs = 0, int profile = 0);
// Spergel / Gaussian instances (bs_fit_prof.cu)
int fit_blocks_per_sm_profile(int profile, int n_chains, int max_side);
cudaError_t launch_fit_profile(const FitParams &p, int grid, cudaStream_t stream);
cudaError_t launch_logpost_points_profile(const FitParams &p, int n_points, const int32_t *gal_index,
                                          const float *theta, double *logp, float *grad, cudaStream_t stream);
// half-light radius over r0 of a profile (Spergel of index nu: root of its enclosed flux)
double profile_hlr_over_r0(int profile, double nu);
// Validate a fit request and fill every launch parameter except the
// scheduling fields (work list, counter) and the serving fields.
bs_status fit_params_from_args(const bs_fit_args *a, const bs_fit_out *o, FitParams &p, const char *who);
cudaError_t launch_logpost_points(const FitParams &p, int n_points, const int32_t *gal_index,
                                  const float *theta, double *logp, float *grad,
                                  cudaStream_t stream);
cudaError_t launch_render(int n, const float *theta, const float *shear, const int64_t *offsets,
                          const int32_t *side, int max_side, const bs_psf *psf, int n_psf,
                          float pixel_scale, float *out, cudaStream_t stream);

struct ShearLaunch {
    const float *e1, *e2, *b;
    const float *w;   // per-galaxy weight of the galaxy's term, or NULL (all 1)
    long long n_gal;
    int K;
    int family;
    float g1, g2;
    float a2;         // log2(e) / (2 alpha^2)
    float kappa;      // 4 (BA14) or 2 (truncated Gaussian)
    float c0;         // log2(e) / (2 sigma_e0^2)
    float r2;         // truncation radius squared
    double *partials; // [grid][4]
};
// All properties free: per sample also log10 flux and log10 hlr, with the
// skew-normal / normal true priors of their hyperparameters.
struct ShearFullLaunch {
    ShearLaunch s;         // ellipticity part (b must be NULL); partials: [grid][kShearFullOut]
    const float *lf, *ls;
    float mu_f, inv_sf, a_f, mu_s, inv_ss;
};
constexpr int kShearFullOut = 9;   // value, d/d(g1, g2, sigma_e, mu_f, sigma_f, a_f, mu_s, sigma_s)

int shear_grid_blocks();
double shear_weight_total(const bs_shear_data *d);
// Several (g1, g2, alpha) points per pass over the samples (no b).
constexpr int kMultiPoints = 4;
struct ShearMultiLaunch {
    ShearLaunch s;                  // data, K, family, kappa, c0, r2, w (g1, g2, a2 unused)
    int n_points;                   // 1..kMultiPoints
    float g1[kMultiPoints], g2[kMultiPoints], a2[kMultiPoints];
    double *partials;               // [kMultiPoints][grid][4]
};
int shear_multi_grid_blocks();
cudaError_t launch_shear_multi(const ShearMultiLaunch &m, int grid, cudaStream_t stream);
int shear_full_grid_blocks();
cudaError_t launch_shear(const ShearLaunch &s, int grid, cudaStream_t stream);
cudaError_t launch_shear_full(const ShearFullLaunch &f, int grid, cudaStream_t stream);
// out[i] = scale[i] * sum over blocks of partials[.][i] + add[i], i < n_out (<= kShearFullOut)
cudaError_t launch_shear_finalize_n(const double *partials, int n_part, int n_out, const double *scale,
                                    const double *add, double *out, cudaStream_t stream);
cudaError_t launch_shear_finalize(const double *partials, int n_part, double add_value,
                                  double add_g1, double add_g2, double add_alpha,
                                  double alpha_scale, double *out, cudaStream_t stream);

// Stan-style metric-adaptation windows of a warmup of W iterations (none when
// !adapt or W < 20): [st[i], en[i]), returns the count (<= cap).
int warmup_windows(int W, bool adapt, int *st, int *en, int cap);

// Thread-local error message of the C ABI (bs_last_error).
bs_status set_error(bs_status st, const char *fmt, ...);

// Kernel launches of the library (bs_kernel_launches): every launch site adds
// one.  While a thread captures a CUDA graph its launches go to the capture's
// own tally instead (capture_launches), which the graph's replays then add.
void count_launches(unsigned long long n);
void capture_launches(unsigned long long *tally);
unsigned long long kernel_launches_total();
// Validate a shear-likelihood request and fill the kernel arguments (except
// `partials`) and the per-galaxy constants the finalize step adds:
// add = {value, d/dg1, d/dg2, d/dalpha}, alpha_scale multiplies the sum of
// softmax-weighted |eps|^2.
bs_status shear_prepare(const bs_shear_data *d, double g1, double g2, double alpha, ShearLaunch &L,
                        double add[4], double &alpha_scale, const char *who);

cudaError_t launch_chain_ess(const float *samples, int n_gal, int n_chains, int n_samples,
                             float *ess, float *rhat, cudaStream_t stream);
// FMA throughput in TFLOP/s (an FMA counts 2): kind 0 FFMA, 1 packed FFMA2, 2 DFMA.
cudaError_t measure_fma_peak(int kind, double &tflops, cudaStream_t stream);

}  // namespace bs
