/*
 * bpshear.h -- C ABI of the GB300 (sm_103a) hot path of Bayesian shear
 * inference with a known PSF and sky background (Mendoza et al.,
 * "Differentiable Forward Modeling for Efficient and Accurate Shear
 * Inference"):
 *
 *   image sampling phase (Sec. 3.3): per-galaxy HMC on the interim posterior
 *     of Eq. interim-post, i.e. the Gaussian pixel likelihood of
 *     Eq. likelihood-pixels times the interim prior of Eq. interim-prior, for
 *     an exponential galaxy sheared in the reduced-shear convention
 *     (Eq. shear-transform) and convolved with a known PSF and the pixel;
 *   shear sampling phase (Sec. 3.2-3.4): the MC shear likelihood of
 *     Eq. likelihood-shear with the Jacobian of
 *     Eq. true-prior-jacobian-shear, its gradient, and the posterior-mean
 *     shear estimate.
 *
 * Conventions shared by every call
 *   - All array arguments are plain pointers to caller-owned memory, device
 *     memory unless stated.  The library never allocates device memory; calls
 *     that need scratch take a caller-provided workspace whose size the
 *     matching *_workspace_bytes() call reports.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; only the calls that
 *     return host results (bs_shear_estimate, and bs_shear_loglike with a host
 *     output) synchronise it.
 *   - Every call returns a bs_status.  Argument errors are detected on the
 *     host before anything is launched; CUDA launch errors are reported as
 *     BS_ERR_CUDA.  bs_last_error() returns a thread-local message describing
 *     the last failure.  No call aborts the process and no C++ exception
 *     crosses this interface.  Problems found inside a kernel (a galaxy whose
 *     starting point is outside the prior support) go to the per-galaxy
 *     status array, which the caller reads after synchronising.
 *   - Parameter vector theta = (lF, ls, e1, e2, dx, dy): lF = log10 flux,
 *     ls = log10 half-light radius [arcsec] of the circular profile before
 *     the area-preserving shear, (e1, e2) = ellipticity in the reduced-shear
 *     ("epsilon") convention (Sec. 2, Eq. ellip-phi-transform), (dx, dy) =
 *     centroid offset from the stamp centre in pixels.
 *   - A stamp of odd side N has pixel (iy, ix) centred at
 *     ((ix - c) p, (iy - c) p), c = (N-1)/2, stored row-major (iy slowest).
 *     Its model is the inverse DFT on the N x N periodic grid of the
 *     analytic spectrum M(k) = F (1 + r0^2 k^T S^2 k)^{-3/2} PSF(|k|)
 *     sinc(kx p/2) sinc(ky p/2) exp(-i p (kx dx + ky dy)), with
 *     r0 = hlr / 1.678347 and S the shear matrix of (e1, e2).
 */
#ifndef BPSHEAR_H
#define BPSHEAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BS_OK = 0,
    BS_ERR_INVALID_ARG = -1,   /* bad pointer, size, layout or option */
    BS_ERR_CUDA = -2,          /* a CUDA runtime call or launch failed */
    BS_ERR_OUT_OF_MEMORY = -3, /* workspace smaller than *_workspace_bytes() */
    BS_ERR_TIMEOUT = -4,       /* a bounded device wait gave up */
    BS_ERR_UNSUPPORTED = -5    /* valid request this build does not serve */
} bs_status;

enum { BS_F32 = 0, BS_F64 = 1 };
enum { BS_PSF_GAUSSIAN = 1, BS_PSF_MOFFAT = 2 };
enum { BS_EPRIOR_BA14 = 0, BS_EPRIOR_TRUNC_GAUSS = 1 };

/* Largest stamp side the kernels accept. */
#define BS_MAX_SIDE 127

/* Known PSF of one galaxy (Sec. 2: Gaussian, FWHM 0.8"; the graphical model
 * of Fig. pgm allows a different known PSF per galaxy).
 * Gaussian: exp(-r^2 / 2 s^2), s = fwhm / 2.35482.
 * Moffat:   (1 + r^2/rd^2)^-beta, fwhm = 2 rd sqrt(2^(1/beta) - 1), beta > 1. */
typedef struct {
    int32_t kind;   /* BS_PSF_* */
    float fwhm;     /* arcsec */
    float beta;     /* Moffat only */
} bs_psf;

/* Interim prior of Eq. interim-prior: log10 f ~ U(lf_lo, lf_hi),
 * log10 s ~ U(ls_lo, ls_hi), dx, dy ~ N(0, sigma_xy) [px], (e1, e2) density
 * proportional to (1-|e|^2)^2 exp(-|e|^2 / (2 sigma_e^2)). */
typedef struct {
    float lf_lo, lf_hi, ls_lo, ls_hi, sigma_xy, sigma_e;
} bs_prior;

/* Paper values: U(-1, 9), U(-2, 1), sigma_xy = 0.5, sigma_e = 0.3. */
void bs_prior_default(bs_prior *prior);

const char *bs_last_error(void);
const char *bs_version(void);

/* Number of kernels this library has launched in this process, over all
 * threads and devices: each direct launch counts one when it is issued, and
 * each replay of a fit plan's CUDA graph counts the kernels the graph holds
 * (kernels recorded while the graph is captured are not launches).  Read it
 * before and after a region to count that region's launches.  Never fails;
 * instrumentation, not a step of the method (the paper has no counterpart). */
uint64_t bs_kernel_launches(void);

/* ------------------------------------------------------------------------ */
/* Rendering (forward model, Sec. 3.3)                                       */
/* ------------------------------------------------------------------------ */

/* Draw n noiseless model stamps.
 *   theta   device float [n][6]; with `shear` non-NULL, (e1, e2) is the
 *           intrinsic ellipticity and is sheared by g = shear[i] with
 *           Eq. shear-transform before drawing.
 *   shear   device float [n][2] or NULL.
 *   offsets device int64 [n]: element offset of stamp i in `out`.
 *   side    device int32 [n]: odd side, 3 <= side <= max_side.
 *   max_side host bound on side[] (<= BS_MAX_SIDE).
 *   psf     device bs_psf [n_psf], n_psf = 1 (shared) or n.
 *   out     device float, written at out[offsets[i] + iy*N + ix].
 * Errors: BS_ERR_INVALID_ARG for NULL required pointers, n < 0, n_psf not
 * in {1, n}, max_side out of range or pixel_scale <= 0. */
bs_status bs_render(int32_t n, const float *theta, const float *shear,
                    const int64_t *offsets, const int32_t *side, int32_t max_side,
                    const bs_psf *psf, int32_t n_psf, float pixel_scale,
                    float *out, void *stream);

/* ------------------------------------------------------------------------ */
/* Image sampling phase: fit_galaxies (Sec. 3.3)                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n_gal;
    int32_t data_dtype;         /* BS_F32 or BS_F64 */
    const void *data;           /* device: packed noisy stamps */
    const int64_t *offsets;     /* device [n_gal]: element offset of each stamp */
    const int32_t *side;        /* device [n_gal]: odd side, 3..max_side */
    int32_t max_side;           /* host bound on side[], <= BS_MAX_SIDE */
    const bs_psf *psf;          /* device [n_psf] */
    int32_t n_psf;              /* 1 (shared) or n_gal */
    const float *noise_sigma;   /* device [n_gal]: pixel noise sd, b = sigma^2 */
    const uint64_t *gal_id;     /* device [n_gal] or NULL (= index): keys the
                                   random stream, so a galaxy's chains do not
                                   depend on its batch or position */
    const float *init;          /* device [n_gal][n_chains][6]: chain starts
                                   (Eq. initialize needs the truth; the caller
                                   supplies them) */
    float pixel_scale;          /* arcsec */
    bs_prior prior;
    int32_t n_chains;           /* 1..8 chains per galaxy */
    int32_t n_warmup;           /* dual-averaging / metric warmup iterations */
    int32_t n_samples;          /* kept iterations per chain */
    int32_t n_leapfrog;         /* L (fixed) or L_max (random_steps) */
    float target_accept;        /* dual-averaging target, 0 < delta < 1 */
    float jitter;               /* eps * U(1-j, 1+j) when !random_steps */
    int32_t adapt_mass;         /* windowed diagonal metric adaptation */
    int32_t random_steps;       /* L_i uniform on 1..n_leapfrog */
    uint64_t seed;
    const float *init_step_size;  /* device [n_gal][n_chains] or NULL: start
                                     from this step size instead of searching
                                     (resuming an adapted chain) */
    const float *init_inv_mass;   /* device [n_gal][n_chains][6] or NULL
                                     (= identity metric) */
    int32_t registers;            /* register cap of the fit kernel: 128, 96
                                     (up to 4 chains) or 80; 0 = 128.  The
                                     library is built without implicit
                                     multiply-add contraction, so all three
                                     round every operation alike and give the
                                     same chains bit for bit: the cap changes
                                     only the speed. */
    /* Pixel-likelihood extensions of Appendix C (zero-initialised: one
     * exposure, white noise, the likelihood of Eq. likelihood-pixels). */
    int32_t n_exposures;          /* J, 0 or 1..BS_MAX_EXPOSURES: exposures of
                                     each galaxy on one pixel grid, stored one
                                     after another from offsets[n] (J side^2
                                     pixels); psf holds n_gal * J entries
                                     (exposure j of galaxy n at n J + j)
                                     unless n_psf == 1, noise_sigma n_gal * J.
                                     The likelihood is the sum over exposures
                                     of Eq. covar-pixel-likelihood with the same
                                     galaxy parameters and each exposure's PSF. */
    const float *noise_corr;      /* NULL (white noise) or device float with the
                                     layout of data (J stamps of side^2 per
                                     galaxy, from offsets[n]): the noise
                                     correlation of exposure j at pixel lag
                                     (dy, dx) in element (dy + c) side + (dx + c),
                                     c = (side - 1)/2; the pixel covariance is
                                     noise_sigma^2 corr(x_a - x_b), stationary
                                     and periodic on the stamp (a circulant
                                     Sigma), corr(0) = 1 for a noise_sigma that
                                     is the pixel sd.  Its spectrum must be
                                     positive (status 3 otherwise). */
    /* Galaxy profile of the forward model (Appendix B; zero: exponential). */
    int32_t profile;              /* BS_PROFILE_EXPONENTIAL, BS_PROFILE_SPERGEL
                                     or BS_PROFILE_GAUSSIAN: transform
                                     (1 + r0^2 q)^-3/2, (1 + r0^2 q)^-(1+nu) or
                                     exp(-r0^2 q / 2) with the same sheared
                                     quadratic form q and log10 hlr parameter;
                                     hlr / r0 = 1.678347 (exponential), the
                                     root of the Spergel enclosed flux
                                     1 - x^(1+nu) K_(1+nu)(x) / (2^nu
                                     Gamma(1+nu)) = 1/2, or sqrt(2 ln 2).  The
                                     register cap applies to the exponential
                                     only (the others run at 128). */
    float spergel_nu;             /* Spergel index nu in [-0.9, 4] (0.5 is the
                                     exponential; -0.6 is close to de
                                     Vaucouleurs) */
    const float *pixel_weight;    /* NULL, or device float with the layout of
                                     data: spatially variable noise (Appendix C),
                                     log L = -1/2 sum_x w(x) (d - m)^2 / sigma^2,
                                     w >= 0 (0 masks a pixel).  Each evaluation
                                     then renders the model image and transforms
                                     the weighted residual back (four dense
                                     DFT-matrix products on the tensor cores,
                                     3xTF32, two chains per CTA).  Requires the
                                     exponential profile, one exposure, no
                                     noise_corr and max_side <= 63. */
    const float *pixel_prec;      /* NULL, or device float: a general pixel
                                     covariance Sigma (Appendix C,
                                     Eq. covar-pixel-likelihood: spatially
                                     variable and correlated at once) given as
                                     its precision P = Sigma^-1, which
                                     bs_dense_precision computes: galaxy n's
                                     block [N^2][N^2] (pixels iy N + ix,
                                     symmetric) starts at prec_offsets[n];
                                     log L = -1/2 (d - m)^T P (d - m) and
                                     noise_sigma is not used.  Each evaluation
                                     renders the model image, multiplies the
                                     residual by P (N^4 multiply-adds, P read
                                     from L2) and transforms the product back.
                                     Requires the exponential profile, one
                                     exposure, no noise_corr or pixel_weight,
                                     max_side <= 31 and at most 4 chains. */
    const int64_t *prec_offsets;  /* device [n_gal]: float offset of each
                                     galaxy's block (with pixel_prec) */
    int32_t chains_per_cta;       /* launch layout: 0 (all of a galaxy's chains
                                     in one CTA) or a divisor of n_chains below
                                     it (the chains split over several CTAs,
                                     each staging the galaxy); the same results
                                     either way.  Nonzero only for the
                                     exponential profile with one exposure and
                                     white noise.  The ragged plan's autotuner
                                     chooses it itself. */
} bs_fit_args;

enum { BS_PROFILE_EXPONENTIAL = 0, BS_PROFILE_SPERGEL = 1, BS_PROFILE_GAUSSIAN = 2 };

#define BS_MAX_EXPOSURES 64

/* Outputs, caller-allocated device buffers (NULL = not wanted, except
 * samples).  Samples are parameter-major so that each parameter plane, e.g.
 * the (e1, e2) planes the shear phase reads, is contiguous. */
typedef struct {
    float *samples;        /* [6][n_gal][n_chains][n_samples] (required) */
    float *logp;           /* [n_gal][n_chains][n_samples]: log posterior
                              (log-likelihood without its constant plus the
                              normalised log interim prior) */
    uint8_t *accepted;     /* [n_gal][n_chains][n_samples]: 1 if accepted */
    float *accept_rate;    /* [n_gal][n_chains]: mean accept statistic */
    float *step_size;      /* [n_gal][n_chains]: adapted step size */
    float *inv_mass;       /* [n_gal][n_chains][6]: adapted inverse metric */
    int32_t *n_divergent;  /* [n_gal][n_chains]: divergent transitions */
    int32_t *status;       /* [n_gal]: 0 ok, 1 a chain started off-support,
                              2 side[] invalid for max_side (galaxy skipped),
                              3 noise_corr of an exposure has a spectrum that is
                              not positive, i.e. no covariance (galaxy skipped),
                              4 (pixel_weight) a tensor-core transform did not
                              complete within its time limit: the galaxy's
                              draws are not valid */
    int32_t *n_grad;       /* [n_gal][n_chains]: log-posterior gradient
                              evaluations the chain made (warmup, searches and
                              sampling) */
    /* Warmup trace (diagnostics; each may be NULL), [n_gal][n_chains][n_warmup]:
     * per warmup transition its accept flag, its accept statistic
     * min(1, e^-dH) (0 when divergent) and the step size it started from
     * (before any jitter); with them the step-size adaptation can be replayed
     * exactly. */
    uint8_t *warmup_accepted;
    float *warmup_accept_stat;
    float *warmup_step_size;
} bs_fit_out;

/* The precision matrices P = Sigma^-1 of general pixel covariances (Appendix
 * C, Eq. covar-pixel-likelihood), once per galaxy, for bs_fit_args.pixel_prec:
 * in FP64 on the device, by the Cholesky factor L of Sigma, W = L^-1 and
 * P = W^T W, stored as FP32.
 *   side    device int32 [n_gal] (odd, 3..max_side);
 *   cov     device float: galaxy n's Sigma, [N^2][N^2] row-major over pixels
 *           iy N + ix, at cov_offsets[n] (device int64 [n_gal]);
 *   prec    device float, the same layout (may not alias cov);
 *   status  device int32 [n_gal] or NULL: set to 3 where Sigma is not
 *           positive definite (that block of prec is zeroed), to 2 where the
 *           side is not odd in 3..max_side (that block is not written);
 *           other entries are left unchanged.
 * max_side <= 31.  Workspace: bs_dense_precision_workspace_bytes(max_side)
 * (an FP64 scratch of 2 max_side^4 doubles per SM).  About N^6 / 2 FP64
 * multiply-adds per galaxy.  Asynchronous on `stream`. */
size_t bs_dense_precision_workspace_bytes(int32_t max_side);
bs_status bs_dense_precision(int32_t n_gal, const int32_t *side, int32_t max_side, const float *cov,
                             const int64_t *cov_offsets, float *prec, int32_t *status, void *workspace,
                             size_t workspace_bytes, void *stream);

/* Bytes of device workspace bs_fit_galaxies needs (a work-queue counter). */
size_t bs_fit_workspace_bytes(const bs_fit_args *args);

/* Run warmup + sampling for every chain of every galaxy in one persistent
 * launch: for each galaxy, the stamp's DFT and the PSF/pixel transfer are
 * staged in shared memory once, then each chain (one warp) runs its whole
 * Markov chain; the per-evaluation log posterior and gradient are evaluated
 * on the spectrum, which for white noise equals the pixel-space chi^2 of
 * Eq. likelihood-pixels (Parseval on the stamp's periodic grid).
 * Errors: BS_ERR_INVALID_ARG (bad sizes, NULL required pointers, n_chains
 * outside 1..8, max_side out of range), BS_ERR_OUT_OF_MEMORY (workspace too
 * small), BS_ERR_CUDA (launch failure).  An empty batch (n_gal == 0) needs no
 * input or output array and returns BS_OK without a launch. */
bs_status bs_fit_galaxies(const bs_fit_args *args, const bs_fit_out *out,
                          void *workspace, size_t workspace_bytes, void *stream);

/* Ragged batches: a launch plan over galaxies of mixed stamp sizes and
 * per-galaxy PSFs (the graphical model of Fig. pgm allows a known PSF per
 * galaxy).  Galaxies are split by the 32-column slots their side needs
 * (<= 31, <= 63, <= 95, <= 127 px) and ordered largest first inside each
 * class; each class gets its own persistent launch sized for its largest
 * stamp.  flags (bitwise or):
 *   BS_PLAN_CAPTURE:  the class launches are recorded once as parallel
 *                     branches of a CUDA graph that bs_fit_plan_launch
 *                     replays (one graph launch per batch); otherwise they
 *                     are issued one after another;
 *   BS_PLAN_AUTOTUNE: per class, the kernel's register cap (128: 4 CTAs =
 *                     16 warps of 4-chain galaxies per SM; 96: 5 CTAs, for
 *                     up to 4 chains; 80: 6 CTAs; the smaller caps spill a
 *                     little; as far as shared memory allows) and layout (all
 *                     or half of a galaxy's chains per CTA) are chosen by
 *                     timing them on the class's first galaxies at creation
 *                     (their outputs are overwritten by every later launch);
 *                     the results are the same whichever is chosen (see
 *                     bs_fit_args.registers).
 *   side_host: host copy of args->side (n_gal).
 *   workspace: bs_fit_plan_workspace_bytes(args) bytes of device memory
 *              (work lists and per-class counters), owned by the caller.
 * The plan keeps the device pointers of args and out: those arrays must stay
 * allocated at the same addresses while the plan is used; their contents may
 * change between launches.  Creation synchronises `stream`.
 * Errors: as bs_fit_galaxies, plus BS_ERR_INVALID_ARG for a side_host entry
 * that is even or outside 3..max_side. */
#define BS_PLAN_CAPTURE 1
#define BS_PLAN_AUTOTUNE 2
typedef struct bs_fit_plan_s *bs_fit_plan;
size_t bs_fit_plan_workspace_bytes(const bs_fit_args *args);
bs_status bs_fit_plan_create(const bs_fit_args *args, const bs_fit_out *out,
                             const int32_t *side_host, int32_t flags, void *workspace,
                             size_t workspace_bytes, void *stream, bs_fit_plan *plan);
bs_status bs_fit_plan_launch(bs_fit_plan plan, void *stream);
bs_status bs_fit_plan_destroy(bs_fit_plan plan);

/* What the plan chose for its i-th class launch (0 <= i < num_launches). */
typedef struct {
    int32_t slot_class;      /* 1..4: stamps of up to 32 x slot_class - 1 px */
    int32_t max_side;        /* largest stamp of the class */
    int32_t n_gal;           /* galaxies in the class */
    int32_t grid;            /* persistent CTAs */
    int32_t registers;       /* register cap of the kernel instance: 128, 96 or 80
                                (the same results with each) */
    float trial_ms_128, trial_ms_96, trial_ms_80;  /* autotune trial times (0 if not tuned) */
    int32_t chains_per_cta;  /* layout: warps (chains) per CTA; below n_chains a
                                galaxy's chains are split over several CTAs,
                                each staging the galaxy */
    float trial_ms_128_half, trial_ms_96_half, trial_ms_80_half;  /* trial
                                times with half the chains per CTA (0 if that
                                layout was not a candidate) */
} bs_fit_plan_launch_info;
int32_t bs_fit_plan_num_launches(bs_fit_plan plan);
bs_status bs_fit_plan_info(bs_fit_plan plan, int32_t i, bs_fit_plan_launch_info *info);

/* Galaxies of side max_side (n_chains chains each) that the current device
 * holds at once in one fit launch with the given register cap (as
 * bs_fit_args.registers; 0 = 128): SMs x resident CTAs, the batch size of a
 * launch that fills the GPU exactly once.  Returns 0 for invalid arguments. */
int32_t bs_fit_resident_galaxies(int32_t n_chains, int32_t max_side, int32_t registers);

/* ------------------------------------------------------------------------ */
/* Serving: fit requests admitted while others run (continuous batching)     */
/* ------------------------------------------------------------------------ */

/* The paper fits a fixed catalogue; a survey pipeline instead receives
 * stamps as they are cut.  A server runs the same per-galaxy fit as
 * bs_fit_galaxies (same kernel, same random streams keyed by gal_id, so a
 * request's result does not depend on what else is on the GPU) for requests
 * that arrive one by one:
 *   - an engine thread admits pending requests first-in first-out, as long as
 *     the device arena has room for their inputs and outputs and fewer than
 *     max_inflight requests are on the GPU ("admission by memory");
 *   - the requests admitted together are staged with one host-to-device copy
 *     and launched, one CTA per galaxy, one launch per 32-column slot class,
 *     each on an idle stream, so the GPU's block scheduler starts them as
 *     soon as running galaxies retire and SMs free up;
 *   - chain state and step-size/metric adaptation live on the GPU for the
 *     whole fit; each CTA copies its galaxy's results into pinned host
 *     memory and raises a completion flag there, which the engine picks up.
 * Times are nanoseconds of a steady clock whose zero is the server's
 * creation (bs_serve_now_ns).  A request is one exposure with white noise
 * and the exponential profile (the Appendix B and C options of
 * bs_fit_args are batch-only). */
typedef struct {
    int32_t max_side;        /* largest stamp side accepted (odd, <= BS_MAX_SIDE) */
    float pixel_scale;       /* arcsec */
    bs_prior prior;
    int32_t n_chains;        /* 1..8 */
    int32_t n_warmup, n_samples, n_leapfrog;
    float target_accept, jitter;
    int32_t adapt_mass, random_steps;
    uint64_t seed;
    int32_t max_inflight;    /* requests on the GPU at once (0: twice the
                                galaxies of side 63 the GPU holds at once) */
    int32_t batch_us;        /* admission interval while the GPU is full
                                (0: 500 us); requests are admitted at once
                                while fewer than the GPU holds are running */
    int32_t n_streams;       /* launch streams (0: 128; 4..128) */
    int32_t registers[4];    /* register cap of the fit kernel per 32-column slot
                                class (stamps up to 31, 63, 95, 127 px): 128,
                                96 or 80, e.g. as a bs_fit_plan autotune chose
                                them; 0 = 128.  Results do not depend on it. */
} bs_serve_cfg;

typedef struct {
    uint64_t tag;            /* caller's identifier, echoed in the completion */
    uint64_t gal_id;         /* keys the random stream, as bs_fit_args.gal_id */
    int32_t side;            /* odd, 3..max_side */
    bs_psf psf;
    float noise_sigma;       /* pixel noise sd */
    const float *stamp;      /* host float [side][side], row-major */
    const float *init;       /* host float [n_chains][6]: chain starts */
    int64_t t_arrival_ns;    /* arrival time on the server clock, or < 0 for
                                the time of submission */
} bs_serve_request;

typedef struct {
    uint64_t tag;
    int32_t status;          /* as bs_fit_out.status */
    int32_t side;
    int64_t t_arrival_ns, t_submit_ns, t_admit_ns, t_done_ns;
    /* Results in the server's pinned host memory, valid until the next
     * bs_serve_poll or bs_serve_destroy call on this server.
     * samples: parameter k, chain c, draw s at
     *          samples[k * plane_stride + c * n_samples + s]. */
    const float *samples;
    int64_t plane_stride;
    const float *logp;           /* [n_chains][n_samples] */
    const uint8_t *accepted;     /* [n_chains][n_samples] */
    const float *accept_rate;    /* [n_chains] */
    const float *step_size;      /* [n_chains] */
    const float *inv_mass;       /* [n_chains][6] */
    const int32_t *n_divergent;  /* [n_chains] */
    const int32_t *n_grad;       /* [n_chains] */
} bs_serve_completion;

typedef struct {
    int64_t submitted, admitted, completed;
    int64_t launches;            /* fit launches issued */
    int64_t ticks;               /* admission rounds that launched work */
    int64_t waits_memory;        /* admission rounds cut short by the arena */
    int64_t waits_inflight;      /* ... by max_inflight */
    int64_t waits_streams;       /* ... by no idle stream */
    int64_t arena_bytes, arena_used, arena_high_water;
    int32_t pending, inflight;
} bs_serve_stats;

typedef struct bs_server_s *bs_server;

/* Arena bytes one request of this side takes while it is admitted (inputs
 * and outputs, before the per-launch alignment). */
size_t bs_serve_request_bytes(const bs_serve_cfg *cfg, int32_t side);

/* Create a server on the current device.
 *   arena: device memory owned by the caller (arena_bytes, >= 1 MiB), which
 *          the server uses for admitted requests until bs_serve_destroy.
 * The server allocates, here only, a pinned host mirror of arena_bytes and
 * its streams, and starts its engine thread.
 * Errors: BS_ERR_INVALID_ARG (bad configuration), BS_ERR_CUDA. */
bs_status bs_serve_create(const bs_serve_cfg *cfg, void *arena, size_t arena_bytes,
                          bs_server *srv);

/* Queue n requests (thread-safe).  The stamp and init arrays are read when a
 * request is admitted: they must stay valid and unchanged until its
 * completion is returned.  All n are checked first; nothing is queued if one
 * is invalid (BS_ERR_INVALID_ARG).  A request larger than the whole arena is
 * invalid. */
bs_status bs_serve_submit(bs_server srv, const bs_serve_request *req, int32_t n);

/* Return up to max completions (first the oldest), waiting up to timeout_us
 * for the first one; *n_out receives the count (0 on timeout).  Completions
 * returned by the previous call are released first, so their result
 * pointers become invalid.  BS_ERR_CUDA if the engine met a CUDA error. */
bs_status bs_serve_poll(bs_server srv, bs_serve_completion *out, int32_t max,
                        int32_t timeout_us, int32_t *n_out);

bs_status bs_serve_get_stats(bs_server srv, bs_serve_stats *stats);
int64_t bs_serve_now_ns(bs_server srv);

/* Stop the engine: requests not yet admitted are dropped, admitted ones run
 * to completion (the call waits for the GPU), then the mirror and the
 * streams are freed. */
bs_status bs_serve_destroy(bs_server srv);

/* Log posterior and gradient of single parameter points, for checking and
 * for differentiation (same arithmetic as the fit's inner loop).
 *   gal_index device int32 [n_points]: which galaxy of `args` each point uses
 *   theta     device float [n_points][6]
 *   logp      device double [n_points] (log-likelihood + log prior; -inf off
 *             the prior support) or NULL; grad device float [n_points][6] or
 *             NULL.  Only the data fields of `args` are read. */
bs_status bs_logpost_points(const bs_fit_args *args, int32_t n_points,
                            const int32_t *gal_index, const float *theta,
                            double *logp, float *grad, void *stream);

/* ------------------------------------------------------------------------ */
/* Chain diagnostics (Sec. 4.1)                                               */
/* ------------------------------------------------------------------------ */

/* Per galaxy and parameter: multi-chain ESS (Geyer initial monotone
 * sequence, ESS capped at C S log10(C S)) and classic R-hat.
 *   samples device float [6][n_gal][n_chains][n_samples]
 *   ess, rhat device float [n_gal][6] (rhat may be NULL). */
bs_status bs_chain_ess(const float *samples, int32_t n_gal, int32_t n_chains,
                       int32_t n_samples, float *ess, float *rhat, void *stream);

/* FP32 FMA throughput of the current device in TFLOP/s (an FMA counts 2),
 * measured with independent FFMA chains (packed = 0) or packed FFMA2 chains
 * (packed != 0) over SMs x 8 blocks of 256 threads: the check on the derived
 * FP32 peak that the fit kernel's roofline uses.  Allocates a scratch buffer
 * (stream-ordered) and synchronises `stream`.  Measurement helper, not a
 * step of the method. */
bs_status bs_fp32_peak(int32_t packed, double *tflops, void *stream);

/* FP64 FMA throughput of the current device in TFLOP/s (an FMA counts 2),
 * measured the same way with independent DFMA chains: the rate an FP64 path
 * (the precision of the CPU restatement) would run at on this GPU.  Same
 * allocation and synchronisation as bs_fp32_peak; measurement helper. */
bs_status bs_fp64_peak(double *tflops, void *stream);

/* ------------------------------------------------------------------------ */
/* Shear sampling phase (Sec. 3.2 - 3.4)                                     */
/* ------------------------------------------------------------------------ */

/* Interim samples of the sheared ellipticity, K per galaxy. */
typedef struct {
    const float *e1;      /* device [n_gal][K] */
    const float *e2;      /* device [n_gal][K] */
    const float *b;       /* device [n_gal][K] or NULL: per-sample log prior
                             ratio of the other properties (0 if NULL) */
    int64_t n_gal;
    int32_t K;
    int32_t family;       /* true ellipticity density: BS_EPRIOR_* */
    float trunc_r;        /* truncation radius (TRUNC_GAUSS only) */
    float sigma_e0;       /* interim ellipticity prior parameter (0.3) */
    const float *gal_weight;  /* device [n_gal] or NULL (all 1): weight w_n >= 0
                                 of galaxy n's term in the log-likelihood,
                                 sum_n w_n L_n; integer weights are a bootstrap
                                 resample (w_n copies of galaxy n), 0 drops it */
    double gal_weight_sum;    /* sum_n w_n when gal_weight != NULL (the
                                 per-galaxy constants scale with it); not read
                                 otherwise.  Must be finite and >= 0. */
} bs_shear_data;

size_t bs_shear_workspace_bytes(int64_t n_gal, int32_t K);

/* Eq. likelihood-shear, Z_n dropped:
 *   value = sum_n [ log sum_k w_nk - log K ],
 *   w = p_e(eps | alpha) |d eps / d eps'| / P0_e(eps') exp(b),
 *   eps = (eps' - g) / (1 - g* eps'),
 * and its gradient with respect to (g1, g2, alpha).  out = {value, d/dg1,
 * d/dg2, d/dalpha} (double[4]); on the device, or on the host when
 * out_on_host != 0 (the call then synchronises `stream`).  Requires
 * |g| < 1, alpha > 0.  A galaxy whose every sample has zero weight makes the
 * value -inf. */
bs_status bs_shear_loglike(const bs_shear_data *data, double g1, double g2,
                           double alpha, double *out, int32_t out_on_host,
                           void *workspace, size_t workspace_bytes, void *stream);

/* bs_shear_loglike at n_points points (g1, g2, alpha) with one read of the
 * samples per kMultiPoints (4) points: the per-sample arithmetic is repeated
 * per point, so a batch of independent points (a Hessian's central
 * differences, quadrature nodes, a grid) costs about its arithmetic instead
 * of one HBM pass per point.
 *   points  host double [n_points][3] = (g1, g2, alpha), each |g| < 1, alpha > 0.
 *   out     double [n_points][4] = {value, d/dg1, d/dg2, d/dalpha} per point,
 *           on the device, or on the host when out_on_host != 0 (the call
 *           then synchronises `stream` after each group of 4 points).
 * data->b must be NULL.  Results agree with bs_shear_loglike up to the
 * summation order (a different reduction layout).  Workspace:
 * bs_shear_workspace_bytes.  n_points == 0 returns BS_OK at once. */
bs_status bs_shear_loglike_multi(const bs_shear_data *data, int32_t n_points, const double *points, double *out,
                                 int32_t out_on_host, void *workspace, size_t workspace_bytes, void *stream);

/* Eq. likelihood-shear with every galaxy property's true prior free (the
 * paper's all-free setting, Sec. 3.3): per sample, the ellipticity weight of
 * bs_shear_loglike times the log-flux and log-size prior ratio
 *   SkewNormal(lf; mu_f, sigma_f, a_f) N(ls; mu_s, sigma_s)
 *     / [U(lf; lf_lo, lf_hi) U(ls; ls_lo, ls_hi)]       (Eq. lflux-lsize-dist
 * over the interim uniforms of Eq. interim-prior), with the skew normal
 * 2 phi(z) Phi(a z) / sigma, z = (lf - mu_f)/sigma_f.
 *   lf, ls   device float [n_gal][K]: log10 flux and log10 hlr samples.
 *   interim  host double [4]: lf_lo, lf_hi, ls_lo, ls_hi.
 *   theta    host double [8]: g1, g2, sigma_e, mu_f, sigma_f, a_f, mu_s, sigma_s.
 *   out      double [9] = {value, d/dtheta[0..7]}, device or host as in
 *            bs_shear_loglike.  data->b must be NULL.
 * Workspace: bs_shear_workspace_bytes.  Requires |g| < 1, sigma_e, sigma_f,
 * sigma_s > 0. */
bs_status bs_shear_loglike_full(const bs_shear_data *data, const float *lf, const float *ls,
                                const double interim[4], const double theta[8], double *out,
                                int32_t out_on_host, void *workspace, size_t workspace_bytes,
                                void *stream);

/* The same likelihood and gradient for callers that cannot allocate device
 * memory or pass a workspace (code under another framework's fixed memory
 * budget, real-time loops that must not allocate).  The paper has no
 * counterpart: this is a deployment variant of bs_shear_loglike.
 *   out: device double [4] = {value, d/dg1, d/dg2, d/dalpha}.
 * The scratch (four FP64 partials -- value, d/dg1, d/dg2 and the weighted
 * sum of |eps|^2 -- per reduction block, at most 2048 blocks, 64 KB) is a
 * static device array of the library, held on every GPU that loads it until
 * exit.  The first call on a device looks up the array's device address and
 * keeps it for the life of the process; make that call before any stream
 * capture, and do not call this entry point after a cudaDeviceReset of that
 * device (the reset unloads the library's device data, and the kept address
 * would then be stale).  All calls share the array, so calls that overlap on
 * the GPU race.  Returns BS_ERR_UNSUPPORTED
 * when the device's reduction grid needs more than 2048 partial slots; the
 * number of galaxies and samples is not limited.  Calls no allocating
 * routine. */
bs_status bs_shear_loglike_noalloc(const bs_shear_data *data, double g1, double g2,
                                   double alpha, double *out, void *stream);

/* Optional sum over processes of the 4 doubles {value, grad} of each
 * evaluation, for a galaxy set sharded across ranks (a no-op when NULL). */
typedef void (*bs_allreduce_fn)(double *buf4, void *user);

typedef struct {
    int32_t free_alpha;     /* 0: infer g with alpha fixed; 1: (g, alpha) */
    double alpha;           /* fixed value, or the starting value if free */
    double alpha_lo, alpha_hi;  /* uniform hyperprior when free */
    int32_t n_gh;           /* Gauss-Hermite points per dimension (1..32) */
    bs_allreduce_fn allreduce;  /* NULL for one process */
    void *allreduce_user;
} bs_estimate_cfg;

/* Posterior mean (and covariance) of g (and alpha) under a uniform prior on
 * the unit disk (and alpha ~ U(alpha_lo, alpha_hi)): Newton iterations to the
 * mode, then tensor Gauss-Hermite quadrature on the Laplace-scaled grid.
 *   mean host double [3] (g1, g2, alpha); cov host double [9] or NULL;
 *   n_evals host int32 or NULL: number of bs_shear_loglike passes used.
 * Synchronises `stream`. */
bs_status bs_shear_estimate(const bs_shear_data *data, const bs_estimate_cfg *cfg,
                            double *mean, double *cov, int32_t *n_evals, void *workspace,
                            size_t workspace_bytes, void *stream);

/* A log-likelihood over (g1, g2, alpha) supplied by the caller: for m points
 * x[m][3] write out[m][4] = {value, d/dg1, d/dg2, d/dalpha}; return 0 on
 * success. */
typedef int32_t (*bs_loglike_points_fn)(const double *x, int32_t m, double *out, void *user);

/* The same estimate (Newton, Laplace-scaled Gauss-Hermite quadrature, the
 * optional all-reduce of cfg after every evaluation) over the caller's
 * likelihood instead of a GPU pass: host code only, e.g. a rank's share of a
 * galaxy set evaluated elsewhere.  A failing callback gives
 * BS_ERR_INVALID_ARG. */
bs_status bs_shear_estimate_custom(bs_loglike_points_fn fn, void *user, const bs_estimate_cfg *cfg,
                                   double *mean, double *cov, int32_t *n_evals);

/* ------------------------------------------------------------------------ */
/* Shear sampling phase as MCMC (Sec. 3.2 "Shear Sampling Phase")            */
/* ------------------------------------------------------------------------ */

/* The paper's uniform hyperpriors (Sec. 3.3): sigma_e ~ U(1e-4, 1),
 * mu_f ~ U(-2, 6), sigma_f ~ U(0, 2), a_f ~ U(-100, 100), mu_s ~ U(-2, 2),
 * sigma_s ~ U(0, 0.5); entries 0, 1 (g, on the unit disk) are -1, 1. */
void bs_shear_hyperprior_default(double lo[8], double hi[8]);

typedef struct {
    uint32_t free_mask;       /* bit i: theta[i] is sampled; bits 0 and 1 (g)
                                 must be set.  theta = (g1, g2, sigma_e, mu_f,
                                 sigma_f, a_f, mu_s, sigma_s) */
    double theta0[8];         /* start, and the value of each fixed parameter */
    double lo[8], hi[8];      /* uniform prior of each sampled theta[2..7]
                                 (open interval); g: uniform on the unit disk */
    const float *lf, *ls;     /* device [n_gal][K] log10 flux and log10 hlr
                                 samples (bs_shear_loglike_full), or both NULL:
                                 ellipticities only (bs_shear_loglike; only
                                 bits 0..2 may be set) */
    double interim[4];        /* lf_lo, lf_hi, ls_lo, ls_hi of the interim prior */
    int32_t n_warmup, n_samples, n_leapfrog;
    float target_accept;      /* dual-averaging target */
    int32_t random_steps;     /* L_i uniform on 1..n_leapfrog, else fixed */
    uint64_t seed;
    bs_allreduce_fn allreduce;  /* sums each evaluation over ranks (or NULL) */
    void *allreduce_user;
} bs_shear_sample_cfg;

/* HMC on g and the chosen hyperparameters with the likelihood of
 * Eq. likelihood-shear evaluated on the GPU at every leapfrog step; the chain
 * itself runs on the host in FP64 (diagonal metric and step size adapted in
 * the warmup, as in the image phase).
 *   samples     host double [n_samples][8] (fixed parameters repeated)
 *   accept_rate, step_size (host double, may be NULL), n_evals (host int32,
 *   may be NULL): likelihood passes used.
 * Workspace: bs_shear_workspace_bytes.  Synchronises `stream` at every
 * step.  Errors: BS_ERR_INVALID_ARG (bad mask or sizes, theta0 outside the
 * prior support), and those of the likelihood calls. */
bs_status bs_shear_sample(const bs_shear_data *data, const bs_shear_sample_cfg *cfg, double *samples,
                          double *accept_rate, double *step_size, int32_t *n_evals, void *workspace,
                          size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Multiplicative and additive shear bias (Sec. 3.4)                        */
/* ------------------------------------------------------------------------ */

/* An estimator of the shear of one dataset whose galaxies carry the weights
 * `weight` (host float [n_gal]: the counts of a bootstrap resample, times the
 * base weights if any; NULL: the original sample, every galaxy once) summing
 * to weight_sum.  Writes g[2] = (g1, g2); returns 0 on success, anything else
 * ends the bias call with BS_ERR_INVALID_ARG. */
typedef int32_t (*bs_g_estimator_fn)(const float *weight, double weight_sum, double *g, void *user);

typedef struct {
    double g_abs;             /* |g| of the applied shear: the plus dataset is
                                 sheared by g = (g_abs, 0), the minus one by -g */
    int32_t n_boot;           /* bootstrap resamples (>= 0; below 2 the
                                 standard deviations are NaN) */
    uint64_t seed;            /* resample r draws galaxy floor(n_gal x / 2^64)
                                 at draw j, x = word (j mod 4) of the
                                 Philox4x64-10 block with key (seed, r) and
                                 counter (floor(j / 4), 0, 1, 0) */
    const float *base_weight; /* host [n_gal] or NULL: multiplies the weights
                                 of the original sample and of every resample
                                 (0 leaves a galaxy out of both datasets) */
    double *m_boot, *c_boot;  /* host [n_boot] or NULL: m and c per resample */
} bs_bias_cfg;

/* Shape-noise cancellation (Sec. 3.4): for two datasets that share their
 * galaxies and noise and are sheared by +g and -g,
 *     m = (g+_1 - g-_1) / (2 |g|) - 1,   c = (g+_2 + g-_2) / 2
 * from the original sample, with bootstrap standard deviations (n_boot - 1
 * in the denominator) over resamples that draw the n_gal galaxies with
 * replacement and apply the same counts to both datasets.
 *   out host double [4] = {m, c, sd(m), sd(c)}.
 * bs_shear_bias_custom takes the two estimators from the caller (any
 * estimator of g from weighted galaxies); it runs on the host only. */
bs_status bs_shear_bias_custom(int64_t n_gal, bs_g_estimator_fn est_plus, void *user_plus,
                               bs_g_estimator_fn est_minus, void *user_minus, const bs_bias_cfg *cfg,
                               double *out);

enum { BS_BIAS_QUADRATURE = 0, BS_BIAS_HMC = 1 };

/* The same with the library's estimators on two device datasets of equal
 * n_gal: the posterior mean of g by bs_shear_estimate (method
 * BS_BIAS_QUADRATURE, configuration est) or the mean of the g draws of
 * bs_shear_sample (BS_BIAS_HMC, configuration smp; each evaluation reruns
 * the sampler with the same seed).  Each evaluation's weights are copied to
 * weight_dev (device float [n_gal], caller-owned; required when n_boot > 0
 * or base_weight is set) and passed as both datasets' gal_weight, whose own
 * gal_weight is ignored.  Workspace: bs_shear_workspace_bytes of the
 * datasets.  Synchronises `stream`.  Errors: BS_ERR_INVALID_ARG (sizes,
 * method, g_abs, negative or non-finite base weights) and those of the
 * estimate or sampler calls. */
bs_status bs_shear_bias(const bs_shear_data *plus, const bs_shear_data *minus, int32_t method,
                        const bs_estimate_cfg *est, const bs_shear_sample_cfg *smp, const bs_bias_cfg *cfg,
                        float *weight_dev, double *out, void *workspace, size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif
