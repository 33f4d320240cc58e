"""Seeded synthetic inputs for the galaxy-fit and shear stages.

This module draws the random inputs: the true parameters of each galaxy,
pixel-noise fields and the random parts of the chain initialisation, every
draw from ``numpy.random.Generator(PCG64(seed))``.  It renders nothing and
evaluates no likelihood: callers turn the draws into images with a renderer of
their own.  Two pieces of input preparation do touch the method's formulas:
``shear_ellipticity`` applies the shear transform (Eq. shear-transform) to
make the sheared truths, and ``toy_interim_ellipticities`` builds the
Appendix-A toy's interim samples (that transform, the eta map and importance
resampling).  They make inputs only; the library never calls this module, and
the oracle neither imports it nor shares its code.

Workloads (stand-ins for the paper's 320k GalSim images of Sec. 2, which are
not available): isolated exponential galaxies at 0.2 arcsec / pixel with
  * half-light radius: ln hlr ~ N(ln 0.8, 0.3) (median 0.8 arcsec),
  * intrinsic ellipticity: (e1, e2) i.i.d. N(0, 0.2) per component, redrawn
    until |e| < 0.7,
  * centroid offset: uniform within the central pixel, U(-0.5, 0.5)^2 px
    (Sec. 2),
  * S/N = sqrt(sum I^2 / b) (Sec. 2 footnote) drawn U(15, 50) (tiny / plain
    batched) or log-uniform on [10, 100] (ragged),
  * white noise sigma = 1 (b = 1, sky dominated, Sec. 2),
  * constant shear g = (+-0.02, 0) (Sec. 3.4).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_DATA = 2604
SEED_CHAINS = 22048
SEED_ARRIVALS = 7

PIXEL_SCALE = 0.2


@dataclass
class Truth:
    """True (intrinsic) galaxy parameters; the shear is applied by the renderer."""
    hlr: np.ndarray            # arcsec
    e_int: np.ndarray          # [n, 2] intrinsic ellipticity
    offset: np.ndarray         # [n, 2] pixels
    snr: np.ndarray            # target S/N
    side: np.ndarray           # stamp side per galaxy (odd)
    psf_fwhm: np.ndarray       # arcsec, per galaxy
    psf_kind: str              # "gaussian" or "moffat"
    psf_beta: float = 3.0
    g: tuple = (0.02, 0.0)
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return len(self.hlr)


def subset(truth: Truth, idx):
    """The galaxies idx of a draw (one rank's share of a dataset)."""
    idx = np.asarray(idx, dtype=np.int64)
    return Truth(hlr=truth.hlr[idx], e_int=truth.e_int[idx], offset=truth.offset[idx], snr=truth.snr[idx],
                 side=truth.side[idx], psf_fwhm=truth.psf_fwhm[idx], psf_kind=truth.psf_kind,
                 psf_beta=truth.psf_beta, g=truth.g, extra=dict(truth.extra))


def _trunc_gauss_e(rng, n, sigma=0.2, rmax=0.7):
    out = np.empty((n, 2))
    filled = 0
    while filled < n:
        e = rng.normal(0.0, sigma, size=(2 * (n - filled) + 8, 2))
        e = e[np.hypot(e[:, 0], e[:, 1]) < rmax]
        take = min(len(e), n - filled)
        out[filled:filled + take] = e[:take]
        filled += take
    return out


def draw_plain(n, side, *, seed=SEED_DATA, snr_range=(15.0, 50.0), psf_fwhm=0.7,
               g=(0.02, 0.0)):
    """Fixed stamp size, one Gaussian PSF: the tiny (25 px, 10 galaxies) and the
    plain batched (53 px, 10^4 galaxies) workloads."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hlr = np.exp(rng.normal(np.log(0.8), 0.3, size=n))
    e = _trunc_gauss_e(rng, n)
    off = rng.uniform(-0.5, 0.5, size=(n, 2))
    snr = rng.uniform(snr_range[0], snr_range[1], size=n)
    return Truth(hlr=hlr, e_int=e, offset=off, snr=snr, side=np.full(n, side, dtype=np.int32),
                 psf_fwhm=np.full(n, psf_fwhm), psf_kind="gaussian", g=tuple(g))


def ragged_side(hlr, fwhm, pixel_scale=PIXEL_SCALE, lo=25, hi=101):
    """Stamp side scaled with size: 2 ceil(4.43 hlr/p + 1.5 FWHM/p) + 1, clipped
    to [lo, hi] (4.43 hlr encloses 99.5% of an exponential's flux)."""
    half = np.ceil(4.43 * hlr / pixel_scale + 1.5 * fwhm / pixel_scale)
    return np.clip(2 * half + 1, lo, hi).astype(np.int32)


def draw_ragged(n, *, seed=SEED_DATA, g=(0.02, 0.0)):
    """Uneven stamp sizes 25..101 px with per-galaxy Moffat(beta = 3) PSFs of
    FWHM U(0.6, 0.9) arcsec and log-uniform S/N on [10, 100]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hlr = np.exp(rng.normal(np.log(0.8), 0.3, size=n))
    e = _trunc_gauss_e(rng, n)
    off = rng.uniform(-0.5, 0.5, size=(n, 2))
    snr = np.exp(rng.uniform(np.log(10.0), np.log(100.0), size=n))
    fwhm = rng.uniform(0.6, 0.9, size=n)
    side = ragged_side(hlr, fwhm)
    return Truth(hlr=hlr, e_int=e, offset=off, snr=snr, side=side, psf_fwhm=fwhm,
                 psf_kind="moffat", psf_beta=3.0, g=tuple(g))


def noise_fields(truth: Truth, sigma=1.0, *, seed=SEED_DATA + 1):
    """One white-noise field per galaxy (list of [side, side] arrays).  The same
    seed gives the same noise for the +g and -g datasets (Sec. 3.4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.normal(0.0, sigma, size=(int(s), int(s))) for s in truth.side]


def init_offsets(truth: Truth, n_chains, *, seed=SEED_CHAINS):
    """Random parts of the chain initialisation of Eq. initialize:
    log10 hlr offsets U(-0.015, 0.015) and ellipticity offsets U(-0.1, 0.1)
    per component.  Returns [n, n_chains, 3] = (d ls, d e1, d e2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d_ls = rng.uniform(-0.015, 0.015, size=(truth.n, n_chains, 1))
    d_e = rng.uniform(-0.1, 0.1, size=(truth.n, n_chains, 2))
    return np.concatenate([d_ls, d_e], axis=-1)


def initial_theta(stamp_sums, ls_true, e_true, offsets):
    """Chain starting points of Eq. initialize from the data sums, the true
    log10 hlr and the true (sheared) ellipticity: flux = sum of pixels, size and
    shape in small boxes around the truth, centroid offset 0.  An ellipticity
    start on or outside the unit circle is pulled back to |e| = 0.95."""
    n, n_chains, _ = offsets.shape
    th = np.zeros((n, n_chains, 6))
    th[..., 0] = np.log10(np.maximum(np.asarray(stamp_sums, dtype=np.float64), 1.0))[:, None]
    th[..., 1] = np.asarray(ls_true)[:, None] + offsets[..., 0]
    e = np.asarray(e_true)[:, None, :] + offsets[..., 1:3]
    r = np.hypot(e[..., 0], e[..., 1])
    scale = np.where(r >= 0.95, 0.95 / np.maximum(r, 1e-300), 1.0)
    th[..., 2:4] = e * scale[..., None]
    return th


def draw_ba14_e(rng, n, sigma=0.2):
    """Intrinsic ellipticities from the (1 - |e|^2)^2 exp(-|e|^2 / 2 sigma^2)
    density on the unit disk (Eq. ellip-mag-prior with its orientation
    uniform): Gaussian proposals of width sigma inside the disk, accepted with
    probability (1 - |e|^2)^2."""
    out = np.empty((n, 2))
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 16
        e = rng.normal(0.0, sigma, size=(m, 2))
        E = (e ** 2).sum(axis=1)
        keep = (E < 1.0) & (rng.uniform(size=m) < (1.0 - np.minimum(E, 1.0)) ** 2)
        e = e[keep]
        take = min(len(e), n - filled)
        out[filled:filled + take] = e[:take]
        filled += take
    return out


def shear_ellipticity(e, g):
    """Sheared ellipticity (e + g) / (1 + conj(g) e) of complex ellipticities e
    (numpy array or torch tensor) under the shear g (a complex number), in the
    reduced-shear convention of Eq. shear-transform."""
    return (e + g) / (1 + g.conjugate() * e)


def shear_ellipticity_pairs(e_int, g):
    """shear_ellipticity on (e1, e2) rows: e_int [n, 2], g (g1, g2) -> [n, 2]."""
    ep = shear_ellipticity(e_int[:, 0] + 1j * e_int[:, 1], complex(g[0], g[1]))
    return np.stack([ep.real, ep.imag], axis=1)


def toy_interim_ellipticities(e_int, g, K, rng, *, sigma_eta=0.1, n_prop=3000, sigma_e0=0.3):
    """Appendix-A toy, first phase: the intrinsic ellipticities e_int [n, 2] are
    sheared by g (Eq. shear-transform), mapped to eta = 2 atanh|e| e/|e|
    (Eq. eta-transform) and observed with N(0, sigma_eta) noise per component
    (Eq. noisy-eta-like); K draws per galaxy from the interim posterior of
    eta' -- that likelihood times the interim ellipticity prior (width
    sigma_e0) times |d eps'/d eta'| -- by sampling-importance-resampling of
    n_prop proposals drawn from the likelihood.  Returns the sheared
    ellipticity samples e1, e2 [n, K] (float32)."""
    n = len(e_int)
    ep = shear_ellipticity(e_int[:, 0] + 1j * e_int[:, 1], complex(g[0], g[1]))
    r = np.maximum(np.abs(ep), 1e-12)
    eta = ep * (2 * np.arctanh(r) / r)
    eta_obs = eta + sigma_eta * (rng.normal(size=n) + 1j * rng.normal(size=n))
    e1 = np.empty((n, K), np.float32)
    e2 = np.empty((n, K), np.float32)
    for i in range(n):
        prop = eta_obs[i] + sigma_eta * (rng.normal(size=n_prop) + 1j * rng.normal(size=n_prop))
        rho = np.maximum(np.abs(prop), 1e-12)
        t = np.tanh(rho / 2)
        eps = prop * (t / rho)
        E = t * t
        logw = 2 * np.log1p(-E) - E / (2 * sigma_e0 ** 2) + np.log(0.5 * (1 - E) * t / rho)
        w = np.exp(logw - logw.max())
        pick = rng.choice(n_prop, size=K, replace=True, p=w / w.sum())
        e1[i] = eps[pick].real
        e2[i] = eps[pick].imag
    return e1, e2


def smoothing_kernel_1d(a):
    """Taps (a, 1, a) of the separable smoothing that correlates pixel noise."""
    return np.array([a, 1.0, a])


def noise_correlation(N, a):
    """Correlation at centred pixel lag [N, N] (lag (dy, dx) at [dy + c, dx + c])
    of white noise smoothed periodically by the separable kernel (a, 1, a) in
    each axis: c1(l) = sum_i k(i) k(i + l), corr = c1(dy) c1(dx) / c1(0)^2."""
    k = smoothing_kernel_1d(a)
    c1 = np.zeros(N)
    cc = (N - 1) // 2
    for lag in range(-2, 3):
        c1[cc + lag] = sum(k[i] * k[i + lag] for i in range(3) if 0 <= i + lag < 3)
    return np.outer(c1, c1) / c1[cc] ** 2


def correlated_noise(rng, n, N, a, sigma=1.0):
    """n periodic N x N noise fields with pixel sd sigma and the correlation of
    noise_correlation(N, a): white noise smoothed by (a, 1, a) in each axis
    (periodic), rescaled."""
    k = smoothing_kernel_1d(a)
    w = rng.normal(size=(n, N, N))
    x = sum(k[i] * np.roll(w, i - 1, axis=2) for i in range(3))
    y = sum(k[i] * np.roll(x, i - 1, axis=1) for i in range(3))
    return sigma * y / float((k ** 2).sum())


def dense_covariance(N, rng, *, a=0.3, sigma=(0.7, 1.5), stray=0.4):
    """A pixel covariance that is neither stationary nor diagonal (Appendix C,
    general Sigma): Sigma = D^1/2 C D^1/2 + s^2 v v^T, with C the periodic
    correlation of noise_correlation(N, a), D the pixel variances of a noise
    level rising linearly across the stamp from sigma[0] to sigma[1] with a
    random tilt, and v a smooth stray-light pattern (a random plane wave of
    amplitude `stray`).  Returns Sigma [N*N, N*N] (float64, rows iy*N + ix)."""
    c = (N - 1) // 2
    corr = noise_correlation(N, a)
    y, x = np.divmod(np.arange(N * N), N)
    C = corr[(y[:, None] - y[None, :] + c) % N, (x[:, None] - x[None, :] + c) % N]
    ang = rng.uniform(0.0, 2.0 * np.pi)
    t = ((x - c) * np.cos(ang) + (y - c) * np.sin(ang)) / max(c, 1)
    sd = sigma[0] + (sigma[1] - sigma[0]) * 0.5 * (t + 1.0)
    kx, ky = rng.uniform(-0.5, 0.5, 2)
    v = np.cos(kx * (x - c) + ky * (y - c) + rng.uniform(0.0, 2.0 * np.pi))
    return sd[:, None] * C * sd[None, :] + stray ** 2 * np.outer(v, v)


def dense_noise(Sigma, rng):
    """One noise field with covariance Sigma (through its Cholesky factor)."""
    n = Sigma.shape[0]
    N = int(round(np.sqrt(n)))
    return (np.linalg.cholesky(Sigma) @ rng.normal(size=n)).reshape(N, N)
