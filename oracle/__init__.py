"""FP64 CPU oracle for Bayesian shear inference with a known PSF and sky level.

TEST INFRASTRUCTURE ONLY.  This package checks the CUDA path; only the test
suite, the package smoke check and the CPU-baseline leg of the benchmark may
import it.  It shares no code with the CUDA path, which never calls it.

The arithmetic lives in plain C (``or_*.c``, double precision, one direct
restatement of each definition of Mendoza et al., "Differentiable Forward
Modeling for Efficient and Accurate Shear Inference"); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Parameter vector theta = (log10 flux, log10 hlr [arcsec], e1, e2, dx, dy [px]).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["or_random.c", "or_render.c", "or_like.c", "or_hmc.c", "or_diag.c", "or_shear.c"]
_LIBPATH = os.path.join(_HERE, "liboracle.so")

PSF_NONE, PSF_GAUSSIAN, PSF_MOFFAT = 0, 1, 2
EPRIOR_BA14, EPRIOR_TRUNC_GAUSS = 0, 1


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the sources (atomic rename)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIBPATH):
        lib_m = os.path.getmtime(_LIBPATH)
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "bs_oracle.h")])
        if lib_m >= newest:
            return _LIBPATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


class _Psf(C.Structure):
    _fields_ = [("kind", C.c_int), ("fwhm", C.c_double), ("beta", C.c_double)]


class _Prior(C.Structure):
    _fields_ = [("lf_lo", C.c_double), ("lf_hi", C.c_double), ("ls_lo", C.c_double),
                ("ls_hi", C.c_double), ("sigma_xy", C.c_double), ("sigma_e", C.c_double)]


class _Hmc(C.Structure):
    _fields_ = [("n_chains", C.c_int), ("n_warmup", C.c_int), ("n_samples", C.c_int),
                ("n_leapfrog", C.c_int), ("target_accept", C.c_double), ("jitter", C.c_double),
                ("adapt_mass", C.c_int), ("seed", C.c_uint64), ("random_steps", C.c_int)]


_lib = None
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_philox4x64_10.argtypes = [C.POINTER(C.c_uint64)] * 3
        L.or_uniforms8.argtypes = [C.c_uint64] * 5 + [_D]
        L.or_hlr_over_r0.restype = C.c_double
        L.or_bessel_k.restype = C.c_double
        L.or_bessel_k.argtypes = [C.c_double, C.c_double]
        L.or_psf_ft.restype = C.c_double
        L.or_psf_ft.argtypes = [C.POINTER(_Psf), C.c_double]
        L.or_exp_profile_ft.restype = C.c_double
        L.or_exp_profile_ft.argtypes = [C.c_double] * 5
        L.or_model_spectrum.argtypes = [C.c_int, C.c_double, C.POINTER(_Psf), _D, _D]
        L.or_transfer_table.argtypes = [C.c_int, C.c_double, C.POINTER(_Psf), _D]
        L.or_idft_image.argtypes = [C.c_int, _D, _D, C.c_int]
        L.or_render.argtypes = [C.c_int, C.c_double, C.POINTER(_Psf), _D, _D, C.c_int]
        L.or_render_many.argtypes = [C.c_int, C.c_int, C.c_double, C.POINTER(_Psf), C.c_int, _D, _D]
        L.or_render_realspace_gauss.argtypes = [C.c_int, C.c_double, C.c_double, _D, C.c_int, C.c_int, _D]
        L.or_log_prior.restype = C.c_double
        L.or_log_prior.argtypes = [C.POINTER(_Prior), _D, _D]
        L.or_log_z_ba14.restype = C.c_double
        L.or_log_z_ba14.argtypes = [C.c_double]
        L.or_loglike.restype = C.c_double
        L.or_loglike.argtypes = [C.c_int, C.c_double, C.POINTER(_Psf), _D, _D, C.c_double, _D, _D]
        L.or_loglike_p.restype = C.c_double
        L.or_loglike_p.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double, C.POINTER(_Psf), _D, C.c_double,
                                   _D, _D]
        L.or_profile_ft.restype = C.c_double
        L.or_profile_ft.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_hlr_over_r0_p.restype = C.c_double
        L.or_hlr_over_r0_p.argtypes = [C.c_int, C.c_double]
        L.or_loglike_dense.restype = C.c_double
        L.or_loglike_dense.argtypes = [C.c_int, C.c_double, C.POINTER(_Psf), _D, _D, _D, _D]
        L.or_loglike_cov.restype = C.c_double
        L.or_loglike_cov.argtypes = [C.c_int, C.c_int, C.c_double, C.POINTER(_Psf), _D, _D, _D, _D, _D]
        L.or_logpost.restype = C.c_double
        L.or_logpost.argtypes = [C.c_int, C.c_double, C.POINTER(_Psf), _D, _D, C.c_double,
                                 C.POINTER(_Prior), _D, _D]
        L.or_window_schedule.restype = C.c_int
        L.or_window_schedule.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int]
        L.or_fit_galaxies.restype = C.c_int
        L.or_fit_galaxies.argtypes = [C.c_int, C.c_int, C.c_double, C.POINTER(_Psf), C.c_int, _D, _D,
                                      C.POINTER(_Prior), C.POINTER(_Hmc), C.POINTER(C.c_uint64), _D,
                                      _D, _D, C.POINTER(C.c_uint8), _D, _D, C.POINTER(C.c_int32), _D,
                                      C.POINTER(C.c_int32), _D, _D, C.POINTER(C.c_uint8), _D, _D, C.c_int]
        L.or_hmc_gauss.restype = C.c_int
        L.or_hmc_gauss.argtypes = [_D, _D, C.POINTER(_Hmc), C.c_uint64, _D, _D, _D, _D, _D, _D]
        L.or_step_search_gauss.restype = C.c_double
        L.or_step_search_gauss.argtypes = [_D, _D, _D, _D, C.c_uint64, C.c_uint64, C.c_int, C.c_double]
        L.or_dual_averaging.argtypes = [C.c_int, _D, C.c_double, C.c_double, _D, _D]
        L.or_ess.restype = C.c_double
        L.or_ess.argtypes = [_D, C.c_int, C.c_int]
        L.or_rhat.restype = C.c_double
        L.or_rhat.argtypes = [_D, C.c_int, C.c_int]
        L.or_log_z_eprior.restype = C.c_double
        L.or_log_z_eprior.argtypes = [C.c_int, C.c_double, C.c_double]
        L.or_log_eprior.restype = C.c_double
        L.or_log_eprior.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_shear_loglike.restype = C.c_double
        L.or_shear_loglike.argtypes = [_F, _F, _F, C.c_int64, C.c_int, C.c_int, C.c_double,
                                       C.c_double, C.c_double, C.c_double, C.c_double, _D]
        L.or_shear_loglike_w.restype = C.c_double
        L.or_shear_loglike_w.argtypes = [_F, _F, _F, _F, C.c_int64, C.c_int, C.c_int, C.c_double,
                                         C.c_double, C.c_double, C.c_double, C.c_double, _D]
        L.or_shear_estimate_w.restype = C.c_int
        L.or_shear_estimate_w.argtypes = [_F, _F, _F, _F, C.c_int64, C.c_int, C.c_int, C.c_double,
                                          C.c_double, C.c_int, C.c_double, C.c_double, C.c_double,
                                          C.c_int, _D, _D]
        L.or_shear_estimate.restype = C.c_int
        L.or_shear_estimate.argtypes = [_F, _F, _F, C.c_int64, C.c_int, C.c_int, C.c_double,
                                        C.c_double, C.c_int, C.c_double, C.c_double, C.c_double,
                                        C.c_int, _D, _D]
        L.or_log_ndtr.restype = C.c_double
        L.or_log_ndtr.argtypes = [C.c_double]
        L.or_log_skewnorm.restype = C.c_double
        L.or_log_skewnorm.argtypes = [C.c_double] * 4
        L.or_shear_loglike_full.restype = C.c_double
        L.or_shear_loglike_full.argtypes = [_F, _F, _F, _F, C.c_int64, C.c_int, C.c_int, C.c_double,
                                            C.c_double, _D, _D, _D]
        L.or_shear_loglike_full_w.restype = C.c_double
        L.or_shear_loglike_full_w.argtypes = [_F, _F, _F, _F, _F, C.c_int64, C.c_int, C.c_int, C.c_double,
                                              C.c_double, _D, _D, _D]
        L.or_gauss_hermite.restype = C.c_int
        L.or_gauss_hermite.argtypes = [C.c_int, _D, _D]
        for nm in ("or_shear_apply", "or_shear_invert"):
            getattr(L, nm).argtypes = [C.c_double] * 4 + [_D, _D]
        L.or_shear_jacobian.restype = C.c_double
        L.or_shear_jacobian.argtypes = [C.c_double] * 4
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _fp(a):
    return a.ctypes.data_as(_F) if a is not None else None


def _psf(psf):
    """psf: (kind, fwhm[, beta]) tuple, or None for a point PSF."""
    if psf is None:
        return _Psf(PSF_NONE, 0.0, 0.0)
    kind, fwhm = int(psf[0]), float(psf[1])
    beta = float(psf[2]) if len(psf) > 2 else 3.0
    return _Psf(kind, fwhm, beta)


def _prior(prior):
    if prior is None:
        return _Prior(-1.0, 9.0, -2.0, 1.0, 0.5, 0.3)
    return _Prior(*[float(x) for x in prior])


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- generator ----------------------------------------------------------------

def philox4x64_10(ctr, key):
    c = (C.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def uniforms8(seed, chain_key, c0, c1, c2):
    u = np.zeros(8)
    lib().or_uniforms8(seed, chain_key, c0, c1, c2, _dp(u))
    return u


# ---- forward model --------------------------------------------------------------

def hlr_over_r0():
    return lib().or_hlr_over_r0()


def bessel_k(nu, x):
    return lib().or_bessel_k(nu, x)


def psf_ft(psf, k):
    p = _psf(psf)
    return lib().or_psf_ft(C.byref(p), float(k))


def exp_profile_ft(kx, ky, r0, e1, e2):
    return lib().or_exp_profile_ft(kx, ky, r0, e1, e2)


def model_spectrum(N, p, psf, theta):
    """Full N x N spectrum, [v+c][u+c], complex128."""
    out = np.zeros((N, N, 2))
    ps = _psf(psf)
    lib().or_model_spectrum(N, p, C.byref(ps), _dp(_d(theta)), _dp(out))
    return out[..., 0] + 1j * out[..., 1]


def transfer_table(N, p, psf):
    out = np.zeros((N, N))
    ps = _psf(psf)
    lib().or_transfer_table(N, p, C.byref(ps), _dp(out))
    return out


def idft_image(M, method=0):
    M = np.asarray(M)
    N = M.shape[0]
    buf = np.ascontiguousarray(np.stack([M.real, M.imag], axis=-1))
    img = np.zeros((N, N))
    lib().or_idft_image(N, _dp(buf), _dp(img), method)
    return img


def render(N, p, psf, theta, method=0):
    img = np.zeros((N, N))
    ps = _psf(psf)
    lib().or_render(N, p, C.byref(ps), _dp(_d(theta)), _dp(img), method)
    return img


def render_many(N, p, psf, theta):
    """theta [n, 6]; psf: tuple (shared) or list of tuples.  Returns [n, N, N]."""
    theta = _d(theta)
    n = theta.shape[0]
    if isinstance(psf, list):
        ps = (_Psf * n)(*[_psf(x) for x in psf])
        npsf = n
    else:
        ps = (_Psf * 1)(_psf(psf))
        npsf = 1
    img = np.zeros((n, N, N))
    lib().or_render_many(n, N, p, ps, npsf, _dp(theta), _dp(img))
    return img


def render_realspace_gauss(N, p, fwhm, theta, nsub, nimg):
    img = np.zeros((N, N))
    lib().or_render_realspace_gauss(N, p, fwhm, _dp(_d(theta)), nsub, nimg, _dp(img))
    return img


# ---- likelihood -------------------------------------------------------------------

def log_prior(theta, prior=None, grad=False):
    pr = _prior(prior)
    g = np.zeros(6)
    v = lib().or_log_prior(C.byref(pr), _dp(_d(theta)), _dp(g))
    return (v, g) if grad else v


def log_z_ba14(alpha):
    return lib().or_log_z_ba14(alpha)


def loglike(N, p, psf, data, sigma, theta, weights=None):
    """Returns (log-likelihood, gradient[6])."""
    ps = _psf(psf)
    g = np.zeros(6)
    w = _d(weights) if weights is not None else None
    v = lib().or_loglike(N, p, C.byref(ps), _dp(_d(data)), _dp(w), sigma, _dp(_d(theta)), _dp(g))
    return v, g


def logpost(N, p, psf, data, sigma, theta, prior=None, weights=None):
    ps = _psf(psf)
    pr = _prior(prior)
    g = np.zeros(6)
    w = _d(weights) if weights is not None else None
    v = lib().or_logpost(N, p, C.byref(ps), _dp(_d(data)), _dp(w), sigma, C.byref(pr),
                         _dp(_d(theta)), _dp(g))
    return v, g


PROFILE_EXPONENTIAL, PROFILE_SPERGEL, PROFILE_GAUSSIAN = 0, 1, 2


def profile_ft(profile, nu, t):
    return lib().or_profile_ft(profile, nu, t)


def hlr_over_r0(profile=PROFILE_EXPONENTIAL, nu=0.5):
    return lib().or_hlr_over_r0_p(profile, nu)


def loglike_p(profile, nu, N, p, psf, data, sigma, theta):
    """Eq. likelihood-pixels with a Spergel (nu) or Gaussian profile
    (Appendix B).  Returns (log-likelihood, gradient[6])."""
    ps = _psf(psf)
    g = np.zeros(6)
    v = lib().or_loglike_p(profile, nu, N, p, C.byref(ps), _dp(_d(data)), sigma, _dp(_d(theta)), _dp(g))
    return v, g


def loglike_dense(N, p, psf, data, Sigma, theta):
    """Appendix C, general covariance: (value, gradient[6]); Sigma [N*N, N*N]."""
    data = _d(data)
    S = _d(Sigma)
    g = np.zeros(6)
    ps = _psf(psf)
    v = lib().or_loglike_dense(N, p, C.byref(ps), _dp(data), _dp(S), _dp(_d(theta)), _dp(g))
    return v, g


def loglike_cov(N, p, psfs, data, sigmas, theta, corr=None):
    """Appendix C: exposures data [J, N, N] with PSFs psfs (J tuples), pixel
    sds sigmas [J] and noise correlations corr [J, N, N] at centred lag (None:
    white).  Returns (log-likelihood, gradient[6])."""
    data = _d(data).reshape(-1, N, N)
    J = data.shape[0]
    ps = (_Psf * J)(*[_psf(x) for x in psfs])
    cr = _d(corr).reshape(J, N, N) if corr is not None else None
    g = np.zeros(6)
    v = lib().or_loglike_cov(J, N, p, ps, _dp(data), _dp(_d(sigmas)), _dp(cr), _dp(_d(theta)), _dp(g))
    return v, g


# ---- HMC ---------------------------------------------------------------------------

def window_schedule(n_warmup, adapt_mass=True):
    s = (C.c_int * 64)()
    e = (C.c_int * 64)()
    n = lib().or_window_schedule(n_warmup, int(adapt_mass), s, e, 64)
    return [(s[i], e[i]) for i in range(n)]


def fit_galaxies(data, sigma, psf, init, *, pixel_scale=0.2, n_warmup=200, n_samples=200,
                 n_leapfrog=8, target_accept=0.8, jitter=0.1, adapt_mass=True, seed=0,
                 ids=None, prior=None, n_threads=0, psf_per_gal=None, random_steps=False,
                 init_step_size=None, init_inv_mass=None):
    """data: [n_gal, N, N]; init: [n_gal, n_chains, 6]; psf: tuple or list of tuples.

    Returns a dict with samples [6, n_gal, n_chains, n_samples], logp, accept,
    accept_rate, step_size, n_div, inv_mass."""
    data = _d(data)
    n_gal, N, _ = data.shape
    init = _d(init)
    n_chains = init.shape[1]
    if isinstance(psf, list):
        ps = (_Psf * n_gal)(*[_psf(x) for x in psf])
        per = 1
    else:
        ps = (_Psf * 1)(_psf(psf))
        per = 0
    pr = _prior(prior)
    cfg = _Hmc(n_chains, n_warmup, n_samples, n_leapfrog, target_accept, jitter, int(adapt_mass), seed,
               int(random_steps))
    sig = _d(np.broadcast_to(np.asarray(sigma, dtype=np.float64), (n_gal,)).copy())
    idarr = None
    if ids is not None:
        idarr = np.ascontiguousarray(ids, dtype=np.uint64)
    S = n_samples
    out = dict(samples=np.zeros((6, n_gal, n_chains, S)), logp=np.zeros((n_gal, n_chains, S)),
               accept=np.zeros((n_gal, n_chains, S), dtype=np.uint8),
               accept_rate=np.zeros((n_gal, n_chains)), step_size=np.zeros((n_gal, n_chains)),
               n_div=np.zeros((n_gal, n_chains), dtype=np.int32),
               inv_mass=np.zeros((n_gal, n_chains, 6)), n_grad=np.zeros((n_gal, n_chains), dtype=np.int32),
               warm_accept=np.zeros((n_gal, n_chains, n_warmup), dtype=np.uint8),
               warm_stat=np.zeros((n_gal, n_chains, n_warmup)), warm_step=np.zeros((n_gal, n_chains, n_warmup)))
    bad = lib().or_fit_galaxies(
        n_gal, N, pixel_scale, ps, per, _dp(data), _dp(sig), C.byref(pr), C.byref(cfg),
        idarr.ctypes.data_as(C.POINTER(C.c_uint64)) if idarr is not None else None, _dp(init),
        _dp(out["samples"]), _dp(out["logp"]), out["accept"].ctypes.data_as(C.POINTER(C.c_uint8)),
        _dp(out["accept_rate"]), _dp(out["step_size"]),
        out["n_div"].ctypes.data_as(C.POINTER(C.c_int32)), _dp(out["inv_mass"]),
        out["n_grad"].ctypes.data_as(C.POINTER(C.c_int32)),
        _dp(_d(init_step_size) if init_step_size is not None else None),
        _dp(_d(init_inv_mass) if init_inv_mass is not None else None),
        out["warm_accept"].ctypes.data_as(C.POINTER(C.c_uint8)), _dp(out["warm_stat"]), _dp(out["warm_step"]),
        int(n_threads))
    out["bad_init"] = bad
    return out


def hmc_gauss(mu, s, init, *, n_warmup=1000, n_samples=500, n_leapfrog=8, target_accept=0.8, jitter=0.0,
              adapt_mass=False, seed=0, random_steps=True, chain_key0=0):
    """The sampler on the Gaussian N(mu, diag(s^2)); init: [n_chains, 6]."""
    init = _d(init)
    n_chains = init.shape[0]
    cfg = _Hmc(n_chains, n_warmup, n_samples, n_leapfrog, target_accept, jitter, int(adapt_mass), seed,
               int(random_steps))
    out = dict(samples=np.zeros((6, n_chains, n_samples)), accept_rate=np.zeros(n_chains),
               step_size=np.zeros(n_chains), inv_mass=np.zeros((n_chains, 6)),
               warm_stat=np.zeros((n_chains, n_warmup)))
    lib().or_hmc_gauss(_dp(_d(mu)), _dp(_d(s)), C.byref(cfg), chain_key0, _dp(init), _dp(out["samples"]),
                       _dp(out["accept_rate"]), _dp(out["step_size"]), _dp(out["inv_mass"]),
                       _dp(out["warm_stat"]))
    return out


def step_search_gauss(mu, s, x, im, seed, key, search, eps0):
    return lib().or_step_search_gauss(_dp(_d(mu)), _dp(_d(s)), _dp(_d(x)), _dp(_d(im)), seed, key, search, eps0)


def dual_averaging(accept_stat, delta, eps0):
    a = _d(accept_stat)
    le = np.zeros(len(a))
    lebar = np.zeros(len(a))
    lib().or_dual_averaging(len(a), _dp(a), delta, eps0, _dp(le), _dp(lebar))
    return le, lebar


# ---- diagnostics ---------------------------------------------------------------------

def ess(x):
    """x: [n_chains, n_samples]."""
    x = _d(x)
    return lib().or_ess(_dp(x), x.shape[0], x.shape[1])


def rhat(x):
    x = _d(x)
    return lib().or_rhat(_dp(x), x.shape[0], x.shape[1])


# ---- shear stage ------------------------------------------------------------------------

def log_z_eprior(family, alpha, trunc_r=0.7):
    return lib().or_log_z_eprior(family, alpha, trunc_r)


def log_eprior(family, alpha, e1, e2, trunc_r=0.7):
    return lib().or_log_eprior(family, alpha, trunc_r, e1, e2)


def shear_apply(e1, e2, g1, g2):
    a, b = C.c_double(), C.c_double()
    lib().or_shear_apply(e1, e2, g1, g2, C.byref(a), C.byref(b))
    return a.value, b.value


def shear_invert(e1, e2, g1, g2):
    a, b = C.c_double(), C.c_double()
    lib().or_shear_invert(e1, e2, g1, g2, C.byref(a), C.byref(b))
    return a.value, b.value


def shear_jacobian(e1p, e2p, g1, g2):
    return lib().or_shear_jacobian(e1p, e2p, g1, g2)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def shear_loglike(e1p, e2p, g1, g2, alpha, *, b=None, family=EPRIOR_BA14, trunc_r=0.7,
                  sigma_e0=0.3, weights=None):
    """e1p, e2p: [n_gal, K] float32; weights: per-galaxy weights or None.
    Returns (value, grad[3])."""
    e1p = _f32(e1p)
    e2p = _f32(e2p)
    n_gal, K = e1p.shape
    bb = _f32(b) if b is not None else None
    ww = _f32(weights) if weights is not None else None
    g = np.zeros(3)
    v = lib().or_shear_loglike_w(_fp(e1p), _fp(e2p), _fp(bb), _fp(ww), n_gal, K, family, trunc_r, sigma_e0,
                                 g1, g2, alpha, _dp(g))
    return v, g


def log_ndtr(t):
    return lib().or_log_ndtr(float(t))


def log_skewnorm(x, mu, sigma, a):
    return lib().or_log_skewnorm(float(x), float(mu), float(sigma), float(a))


def shear_loglike_full(e1p, e2p, lfp, lsp, theta, *, family=EPRIOR_BA14, trunc_r=0.7, sigma_e0=0.3,
                       interim=(-1.0, 9.0, -2.0, 1.0), weights=None):
    """All-free shear likelihood; theta = (g1, g2, sigma_e, mu_f, sigma_f, a_f,
    mu_s, sigma_s); optional per-galaxy weights.  Returns (value, grad[8])."""
    e1p, e2p, lfp, lsp = _f32(e1p), _f32(e2p), _f32(lfp), _f32(lsp)
    ww = _f32(weights) if weights is not None else None
    n_gal, K = e1p.shape
    th = np.ascontiguousarray(theta, dtype=np.float64)
    im = np.ascontiguousarray(interim, dtype=np.float64)
    g = np.zeros(8)
    v = lib().or_shear_loglike_full_w(_fp(e1p), _fp(e2p), _fp(lfp), _fp(lsp), _fp(ww), n_gal, K, family, trunc_r,
                                      sigma_e0, _dp(im), _dp(th), _dp(g))
    return v, g


def shear_estimate(e1p, e2p, *, b=None, family=EPRIOR_BA14, trunc_r=0.7, sigma_e0=0.3,
                   free_alpha=False, alpha=0.2, alpha_lo=1e-4, alpha_hi=1.0, n_gh=7, weights=None):
    e1p = _f32(e1p)
    e2p = _f32(e2p)
    n_gal, K = e1p.shape
    bb = _f32(b) if b is not None else None
    ww = _f32(weights) if weights is not None else None
    mean = np.zeros(3)
    cov = np.zeros(9)
    st = lib().or_shear_estimate_w(_fp(e1p), _fp(e2p), _fp(bb), _fp(ww), n_gal, K, family, trunc_r, sigma_e0,
                                   int(free_alpha), alpha, alpha_lo, alpha_hi, n_gh, _dp(mean), _dp(cov))
    if st != 0:
        raise RuntimeError("oracle shear estimate failed")
    n = 3 if free_alpha else 2
    return mean[:n], cov.reshape(3, 3)[:n, :n]


def gauss_hermite(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().or_gauss_hermite(n, _dp(x), _dp(w)) != 0:
        raise ValueError(n)
    return x, w
