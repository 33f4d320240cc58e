"""The oracle pinned to things other than itself: library routines (numpy's
Philox and Gauss-Hermite, scipy's Bessel K, quadrature and root finding),
closed forms, geometric identities, brute force, and the paper's printed
constants (tests/golden/paper_constants.json).  CPU only."""
import json
import os

import numpy as np
import pytest
import scipy.integrate as si
import scipy.linalg as sl
import scipy.optimize as so
import scipy.special as sp

import oracle as O
from paper_2604_22048_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ---------------------------------------------------------------- generator

@pytest.mark.parametrize("ctr,key", [([1, 0, 0, 0], [0, 0]), ([5, 7, 0, 1], [11, 22]),
                                     ([2 ** 40 + 3, 1, 2, 3], [2 ** 63 + 5, 12345]),
                                     ([123, 1, 60, 0], [22048, 4 * 9999 + 3])])
def test_philox_matches_numpy(ctr, key):
    # numpy's Philox (4x64, 10 rounds) increments its counter before each block
    bg = np.random.Philox(counter=np.array([ctr[0] - 1] + ctr[1:], dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    assert O.philox4x64_10(ctr, key) == [int(x) for x in bg.random_raw(4)]


def test_uniforms_are_philox_top_bits():
    seed, key = 22048, 77
    w = O.philox4x64_10([9, 1, 3, 0], [seed, key])
    u = O.uniforms8(seed, key, 9, 1, 3)
    bits = []
    for x in w:
        bits += [(x >> 32) >> 8, (x & 0xFFFFFFFF) >> 8]
    assert np.array_equal(np.floor(u * 2 ** 24).astype(np.int64), np.array(bits))
    assert ((u > 0) & (u < 1)).all()


# ---------------------------------------------------------------- profile

def test_hlr_constant():
    root = so.brentq(lambda x: 1 - (1 + x) * np.exp(-x) - 0.5, 1.0, 3.0, xtol=1e-15)
    assert abs(O.hlr_over_r0() - root) < 1e-12
    # the enclosed-flux formula itself, by integrating the profile
    enc = si.quad(lambda r: r * np.exp(-r), 0, root, epsabs=1e-14)[0]
    assert abs(enc - 0.5) < 1e-12


@pytest.mark.parametrize("nu,x", [(2, 0.5), (2, 3.0), (2, 1e-3), (1.5, 0.7), (0.5, 2.0), (2, 25.0)])
def test_bessel_k_vs_scipy(nu, x):
    assert abs(O.bessel_k(nu, x) / sp.kv(nu, x) - 1) < 1e-12


def _hankel(f, k, rmax):
    return 2 * np.pi * si.quad(lambda r: f(r) * sp.j0(k * r) * r, 0, rmax, limit=2000, epsabs=1e-13)[0]


@pytest.mark.parametrize("k", [0.0, 0.7, 3.0, 11.0])
def test_exponential_ft_vs_hankel(k):
    r0 = 0.4
    num = _hankel(lambda r: np.exp(-r / r0) / (2 * np.pi * r0 ** 2), k, 60 * r0)
    assert abs(O.exp_profile_ft(k, 0.0, r0, 0.0, 0.0) - num) < 1e-9


@pytest.mark.parametrize("k", [0.0, 0.5, 2.0, 6.0])
def test_moffat_and_gaussian_ft_vs_hankel(k):
    fwhm, beta = 0.8, 3.0
    rd = fwhm / (2 * np.sqrt(2 ** (1 / beta) - 1))
    assert abs((1 + (fwhm / 2) ** 2 / rd ** 2) ** -beta - 0.5) < 1e-12          # FWHM definition
    mof = lambda r: (beta - 1) / (np.pi * rd ** 2) * (1 + (r / rd) ** 2) ** -beta
    assert abs(O.psf_ft((O.PSF_MOFFAT, fwhm, beta), k) - _hankel(mof, k, 4000 * rd)) < 2e-7
    s = fwhm / (2 * np.sqrt(2 * np.log(2)))
    assert abs(np.exp(-(fwhm / 2) ** 2 / (2 * s * s)) - 0.5) < 1e-12
    gau = lambda r: np.exp(-r * r / (2 * s * s)) / (2 * np.pi * s * s)
    assert abs(O.psf_ft((O.PSF_GAUSSIAN, fwhm), k) - _hankel(gau, k, 20 * s)) < 1e-10


# ---------------------------------------------------------------- renderer

TH = [2.5, np.log10(0.6), 0.2, -0.15, 0.3, -0.2]


def test_render_direct_separable_and_numpy_fft_agree():
    N = 15
    a = O.render(N, 0.2, (O.PSF_GAUSSIAN, 0.7), TH, 0)
    b = O.render(N, 0.2, (O.PSF_GAUSSIAN, 0.7), TH, 1)
    M = O.model_spectrum(N, 0.2, (O.PSF_GAUSSIAN, 0.7), TH)
    c = np.real(np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(M))))
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    assert np.abs(a - c).max() < 1e-13 * np.abs(a).max()


def test_render_total_flux_is_F():
    for N in (9, 25, 53):
        img = O.render(N, 0.2, (O.PSF_MOFFAT, 0.8, 3.0), TH)
        assert abs(img.sum() / 10 ** TH[0] - 1) < 1e-12


def test_render_matches_realspace_bruteforce():
    """Periodic pixel integrals of exponential * Gaussian PSF by midpoint
    quadrature in real space; the k-space render differs only by the spectrum
    beyond the grid (< 1e-10 here) and the quadrature error."""
    N, p, fw = 9, 0.2, 0.8
    th = [2.0, np.log10(1.0), 0.15, -0.1, 0.25, -0.3]
    k = O.render(N, p, (O.PSF_GAUSSIAN, fw), th)
    r = O.render_realspace_gauss(N, p, fw, th, 32, 10)
    assert np.abs(k - r).max() < 2e-8 * k.max()


@pytest.mark.parametrize("e", [(0.3, -0.2), (0.0, 0.0), (-0.5, 0.1)])
def test_second_moments_closed_form(e):
    """Exponential: <x x^T> = 3 r0^2 S S^T; the Gaussian PSF adds s^2 I and the
    pixel p^2/12 I; the centroid is at the offset."""
    N, p, fw, hlr = 151, 0.2, 0.8, 0.5
    e1, e2 = e
    th = [3.0, np.log10(hlr), e1, e2, 0.3, -0.4]
    img = O.render(N, p, (O.PSF_GAUSSIAN, fw), th)
    x = (np.arange(N) - (N - 1) / 2) * p
    X, Y = np.meshgrid(x, x)
    F = img.sum()
    mx, my = (img * X).sum() / F, (img * Y).sum() / F
    assert abs(mx / p - 0.3) < 1e-8 and abs(my / p + 0.4) < 1e-8
    I = np.array([[(img * (X - mx) ** 2).sum(), (img * (X - mx) * (Y - my)).sum()],
                  [(img * (X - mx) * (Y - my)).sum(), (img * (Y - my) ** 2).sum()]]) / F
    r0 = hlr / O.hlr_over_r0()
    E = e1 * e1 + e2 * e2
    SS = np.array([[1 + 2 * e1 + E, 2 * e2], [2 * e2, 1 - 2 * e1 + E]]) / (1 - E)
    s = fw / (2 * np.sqrt(2 * np.log(2)))
    want = 3 * r0 ** 2 * SS + (s * s + p * p / 12) * np.eye(2)
    assert np.abs(I - want).max() < 1e-8 * np.abs(want).max()


def test_square_aperture_flux_matches_hankel():
    """Flux of exponential * Gaussian PSF inside centred squares of half-width a:
    (4/pi) int_0^{pi/4} E(a / cos phi) dphi with the circular enclosed flux
    E(R) = R int_0^inf F(k) J1(k R) dk of the radial transform F."""
    N, p, fw, hlr = 101, 0.2, 0.8, 0.5
    th = [0.0, np.log10(hlr), 0.0, 0.0, 0.0, 0.0]
    img = O.render(N, p, (O.PSF_GAUSSIAN, fw), th)
    r0 = hlr / O.hlr_over_r0()
    s = fw / (2 * np.sqrt(2 * np.log(2)))
    Fk = lambda k: (1 + (k * r0) ** 2) ** -1.5 * np.exp(-0.5 * (k * s) ** 2)
    Ecirc = lambda R: R * si.quad(lambda k: Fk(k) * sp.j1(k * R), 0, 60.0 / s, limit=4000, epsabs=1e-13)[0]
    c = (N - 1) // 2
    for half in (2, 5, 12):
        a = (half + 0.5) * p
        want = 4 / np.pi * si.quad(lambda ph: Ecirc(a / np.cos(ph)), 0, np.pi / 4, epsabs=1e-11)[0]
        got = img[c - half:c + half + 1, c - half:c + half + 1].sum()
        assert abs(got - want) < 2e-7, (half, got, want)


# ---------------------------------------------------------------- likelihood and prior

@pytest.mark.parametrize("psf", [(O.PSF_GAUSSIAN, 0.7), (O.PSF_MOFFAT, 0.8, 3.0)])
@pytest.mark.parametrize("weighted", [False, True])
def test_logpost_gradient_matches_central_differences(psf, weighted):
    rng = np.random.default_rng(1)
    N = 25
    th = np.array([2.6, np.log10(0.7), 0.25, -0.1, 0.2, -0.35])
    data = O.render(N, 0.2, psf, [2.55, np.log10(0.75), 0.2, -0.05, 0.1, -0.3]) + rng.normal(0, 1, (N, N))
    w = rng.uniform(0.5, 1.5, (N, N)) if weighted else None
    v, g = O.logpost(N, 0.2, psf, data, 1.3, th, weights=w)
    fd = np.zeros(6)
    for i in range(6):
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (O.logpost(N, 0.2, psf, data, 1.3, tp, weights=w)[0] - O.logpost(N, 0.2, psf, data, 1.3, tm, weights=w)[0]) / (2 * h)
    assert np.abs(fd - g).max() < 1e-7 * np.abs(g).max()


def test_loglike_is_pixel_chi2():
    rng = np.random.default_rng(2)
    N = 21
    data = rng.normal(0, 1, (N, N)) + O.render(N, 0.2, (O.PSF_GAUSSIAN, 0.7), TH)
    m = O.render(N, 0.2, (O.PSF_GAUSSIAN, 0.7), TH)
    v, _ = O.loglike(N, 0.2, (O.PSF_GAUSSIAN, 0.7), data, 1.7, TH)
    assert abs(v + 0.5 * ((data - m) ** 2).sum() / 1.7 ** 2) < 1e-10 * abs(v)


def test_interim_prior_normalised_and_support():
    # ellipticity density integrates to one over the unit disk (polar quadrature)
    se = 0.3
    lz = O.log_z_ba14(se)
    tot = si.dblquad(lambda r, t: r * np.exp(2 * np.log1p(-r * r) - r * r / (2 * se * se) - lz),
                     0, 2 * np.pi, 0, 1, epsabs=1e-13)[0]
    assert abs(tot - 1) < 1e-10
    # the full prior at one point: uniform * uniform * Gaussian * Gaussian * e density
    th = [3.0, -0.2, 0.3, 0.1, 0.2, -0.1]
    want = (-np.log(10) - np.log(3) - np.log(2 * np.pi * 0.25) - (0.04 + 0.01) / 0.5
            + 2 * np.log1p(-0.1) - 0.1 / 0.18 - lz)
    assert abs(O.log_prior(th) - want) < 1e-12
    assert O.log_prior([3.0, -0.2, 0.8, 0.7, 0, 0]) == -np.inf
    assert O.log_prior([9.5, -0.2, 0.1, 0.1, 0, 0]) == -np.inf


def test_golden_paper_constants():
    g = json.load(open(GOLDEN))
    ip = g["interim_prior"]
    from paper_2604_22048_gb300 import api
    want = (*ip["log10_flux_uniform"], *ip["log10_hlr_uniform"], ip["sigma_xy_pixels"], ip["sigma_e"])
    assert tuple(api.DEFAULT_PRIOR) == want
    assert O._prior(None).sigma_e == ip["sigma_e"] and O._prior(None).sigma_xy == ip["sigma_xy_pixels"]
    assert synth.PIXEL_SCALE == g["pixel_scale_arcsec"]["value"]
    assert synth.draw_plain(3, 25).g[0] == g["applied_shear_g1"]["value"]
    off = synth.init_offsets(synth.draw_plain(50, 25), 4)
    assert np.abs(off[..., 0]).max() <= g["chain_init_boxes"]["log10_hlr_halfwidth"]
    assert np.abs(off[..., 1:]).max() <= g["chain_init_boxes"]["ellipticity_halfwidth"]


# ---------------------------------------------------------------- shear transform

def _S(e1, e2):
    E = e1 * e1 + e2 * e2
    return np.array([[1 + e1, e2], [e2, 1 - e1]]) / np.sqrt(1 - E)


@pytest.mark.parametrize("e,g", [((0.3, -0.2), (0.02, 0.0)), ((-0.6, 0.5), (0.1, -0.07)), ((0.0, 0.0), (0.05, 0.05))])
def test_shear_composition(e, g):
    """Shearing an ellipse: S_g S_eps = S_eps' R with R a rotation (polar
    decomposition), eps' = (eps + g)/(1 + g* eps) (Eq. shear-transform)."""
    M = _S(*g) @ _S(*e)
    P = sl.sqrtm(M @ M.T).real
    ep = O.shear_apply(*e, *g)
    assert np.abs(P - _S(*ep)).max() < 1e-12
    R = np.linalg.solve(P, M)
    assert np.abs(R @ R.T - np.eye(2)).max() < 1e-12
    back = O.shear_invert(*ep, *g)
    assert np.abs(np.array(back) - e).max() < 1e-14


def test_jacobian_matches_fd_determinant():
    g1, g2, h = 0.03, -0.02, 1e-6
    for e in [(0.4, 0.3), (-0.7, 0.1), (0.0, 0.0)]:
        inv = lambda a, b: np.array(O.shear_invert(a, b, g1, g2))
        J = np.column_stack([(inv(e[0] + h, e[1]) - inv(e[0] - h, e[1])) / (2 * h),
                             (inv(e[0], e[1] + h) - inv(e[0], e[1] - h)) / (2 * h)])
        assert abs(abs(np.linalg.det(J)) / O.shear_jacobian(*e, g1, g2) - 1) < 1e-8


@pytest.mark.parametrize("a", [0.15, 0.2, 0.3, 0.8])
def test_ellipticity_normalisers_vs_quadrature(a):
    z = si.dblquad(lambda r, t: r * (1 - r * r) ** 2 * np.exp(-r * r / (2 * a * a)), 0, 2 * np.pi, 0, 1,
                   epsabs=1e-14, epsrel=1e-13)[0]
    assert abs(O.log_z_ba14(a) - np.log(z)) < 1e-12
    zt = si.quad(lambda r: 2 * np.pi * r * np.exp(-r * r / (2 * a * a)), 0, 0.7, epsabs=1e-15)[0]
    assert abs(O.log_z_eprior(O.EPRIOR_TRUNC_GAUSS, a, 0.7) - np.log(zt)) < 1e-12


# ---------------------------------------------------------------- shear likelihood

def _samples(rng, n, K, s=0.2):
    e = rng.normal(0, s, (n, K, 2))
    r = np.hypot(e[..., 0], e[..., 1])
    e[r > 0.9] *= (0.9 / r[r > 0.9])[:, None]
    return e[..., 0].astype(np.float32), e[..., 1].astype(np.float32)


def test_shear_loglike_zero_when_true_prior_is_interim():
    """g = 0 and the true density equal to the interim one: every weight is 1."""
    rng = np.random.default_rng(0)
    e1, e2 = _samples(rng, 30, 17)
    v, _ = O.shear_loglike(e1, e2, 0.0, 0.0, 0.3, family=O.EPRIOR_BA14, sigma_e0=0.3)
    assert abs(v) < 1e-12


@pytest.mark.parametrize("family", [O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS])
def test_shear_loglike_gradient_fd(family):
    rng = np.random.default_rng(2)
    e1, e2 = _samples(rng, 50, 40)
    b = rng.normal(0, 0.5, (50, 40)).astype(np.float32)
    x = np.array([0.02, -0.01, 0.25])
    _, g = O.shear_loglike(e1, e2, *x, b=b, family=family)
    for i in range(3):
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (O.shear_loglike(e1, e2, *xp, b=b, family=family)[0] - O.shear_loglike(e1, e2, *xm, b=b, family=family)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * np.abs(g).max()


def test_shear_likelihood_recovers_g_noise_free():
    """One exact sheared ellipticity per galaxy (K = 1): the shear likelihood is
    the likelihood of g for the sheared shapes, so the estimate sits on g; with
    the same intrinsic shapes sheared by +g and -g the shape noise cancels."""
    n = 20000
    t = synth.draw_plain(n, 25, seed=4)
    est = {}
    for sgn in (1, -1):
        g = (0.02 * sgn, 0.0)
        ep = np.array([O.shear_apply(a, b, *g) for a, b in t.e_int])
        m, cov = O.shear_estimate(ep[:, :1].astype(np.float32), ep[:, 1:].astype(np.float32),
                                  family=O.EPRIOR_TRUNC_GAUSS, alpha=0.2)
        assert abs(m[0] - g[0]) < 4 * np.sqrt(cov[0, 0])
        assert abs(m[1] - g[1]) < 4 * np.sqrt(cov[1, 1])
        est[sgn] = m
    # g1 shape noise cancels in the pair; g2 shape noise does not (only g1 flips)
    m_hat = (est[1][0] - est[-1][0]) / 0.04 - 1
    assert abs(m_hat) < 2e-3, m_hat


def test_gauss_hermite_vs_numpy():
    for n in (1, 3, 7, 12):
        x, w = O.gauss_hermite(n)
        xr, wr = np.polynomial.hermite.hermgauss(n)
        assert np.abs(x - xr).max() < 1e-12 and np.abs(w - wr).max() < 1e-12


# ---------------------------------------------------------------- sampler pieces

def test_window_schedule_documented_example():
    # Stan's documented schedule for 1000 warmup iterations: 75 fast, slow
    # windows of 25, 50, 100, 200 and a stretched 500, 50 fast
    assert O.window_schedule(1000) == [(75, 100), (100, 150), (150, 250), (250, 450), (450, 950)]
    assert O.window_schedule(300) == [(75, 100), (100, 150), (150, 250)]
    assert O.window_schedule(100) == [(15, 90)]
    assert O.window_schedule(10) == [] and O.window_schedule(300, False) == []


def test_ess_iid_and_ar1():
    rng = np.random.default_rng(0)
    C, S = 4, 20000
    x = rng.normal(size=(C, S))
    assert abs(O.ess(x) / (C * S) - 1) < 0.1
    rho = 0.5
    y = np.zeros((C, S))
    y[:, 0] = rng.normal(size=C)
    for s in range(1, S):
        y[:, s] = rho * y[:, s - 1] + np.sqrt(1 - rho * rho) * rng.normal(size=C)
    assert abs(O.ess(y) / (C * S * (1 - rho) / (1 + rho)) - 1) < 0.1
    assert O.rhat(x) < 1.01
    z = x + np.arange(C)[:, None] * 0.5
    assert O.rhat(z) > 1.1


def test_rhat_matches_its_large_sample_limit_with_planted_chain_shifts():
    # Gelman & Rubin (1992): with within-chain variance v and chain means
    # spread with sample variance b, var+ -> v + b and R-hat -> sqrt(1 + b/v)
    # as the chains grow.
    rng = np.random.default_rng(12)
    C, S, v = 4, 40000, 2.0
    for shifts in ([-0.6, -0.2, 0.2, 0.6], [0.0, 0.0, 0.0, 1.5], [0.3, -0.1, 0.25, -0.4]):
        sh = np.asarray(shifts)
        x = rng.normal(0.0, np.sqrt(v), (C, S)) + sh[:, None]
        limit = np.sqrt(1.0 + sh.var(ddof=1) / v)
        assert abs(O.rhat(x) / limit - 1) < 0.01, (shifts, O.rhat(x), limit)


# ---- warmup adaptation (Sec. 3.3, the warmup footnote: dual averaging of the
# step size, Hoffman & Gelman 2014 Sec. 3.2 with gamma 0.05, t0 10, kappa 0.75,
# mu = log(10 eps); Stan's step-size search and windowed diagonal metric)

_GMU = np.array([0.3, -1.0, 0.0, 2.0, 0.5, -0.2])
_GS = np.array([0.05, 0.3, 1.0, 2.0, 0.5, 1.5])


def test_dual_averaging_equals_the_averaged_form_of_the_iterates():
    # Hoffman & Gelman write the iterate with the running mean of the
    # statistics: x_t = mu - sqrt(t)/gamma * (1/(t + t0)) sum_{i<=t} (delta - a_i),
    # and x-bar_t as the average sum_j x_j eta_j prod_{i>j} (1 - eta_i),
    # eta_j = j^-kappa; the oracle updates both recursively.
    rng = np.random.default_rng(4)
    a = rng.uniform(0.0, 1.0, 300)
    delta, eps0 = 0.8, 0.37
    le, lebar = O.dual_averaging(a, delta, eps0)
    t = np.arange(1, len(a) + 1, dtype=np.float64)
    x = np.log(10 * eps0) - np.sqrt(t) / 0.05 * np.cumsum(delta - a) / (t + 10.0)
    assert np.abs(le - x).max() < 1e-9
    eta = t ** -0.75
    for M in (1, 2, 7, 60, 300):
        w = np.array([eta[j] * np.prod(1.0 - eta[j + 1:M]) for j in range(M)])
        assert abs(w.sum() - 1.0) < 1e-12
        assert abs(lebar[M - 1] - (w * x[:M]).sum()) < 1e-9, M
    # statistics equal to the target leave both at mu = log(10 eps0)
    le, lebar = O.dual_averaging(np.full(40, 0.65), 0.65, 0.2)
    assert np.abs(le - np.log(2.0)).max() < 1e-14 and np.abs(lebar - np.log(2.0)).max() < 1e-14


def _box_muller6(u):
    z = np.empty(6)
    for j in range(3):
        r = np.sqrt(-2.0 * np.log(u[2 * j]))
        z[2 * j], z[2 * j + 1] = r * np.cos(2 * np.pi * u[2 * j + 1]), r * np.sin(2 * np.pi * u[2 * j + 1])
    return z


def _gauss_one_step_logacc(x, im, z, eps):
    """log acceptance H0 - H1 of one leapfrog step on N(_GMU, diag(_GS^2))
    with inverse metric im and momentum z / sqrt(im)."""
    H = lambda q, p: 0.5 * (((q - _GMU) / _GS) ** 2).sum() + 0.5 * (im * p * p).sum()
    grad = lambda q: -(q - _GMU) / _GS ** 2
    p = z / np.sqrt(im)
    H0 = H(x, p)
    p = p + 0.5 * eps * grad(x)
    q = x + eps * im * p
    p = p + 0.5 * eps * grad(q)
    return H0 - H(q, p)


@pytest.mark.parametrize("eps0,search", [(1e-3, 0), (1.0, 0), (30.0, 2), (0.05, 1)])
def test_step_search_stops_at_the_first_crossing_of_log_0p8(eps0, search):
    # Trial t of search s draws its momentum from Philox counter (s, 1, t); the
    # step doubles while the one-step log acceptance stays above ln 0.8 (or
    # halves while it stays at or below), and the search returns the first
    # step on the other side.  The acceptance here is the exact one of the
    # Gaussian target, computed independently.
    rng = np.random.default_rng(int(eps0 * 1000) + search)
    seed, key = 22048, 17
    for _ in range(4):
        x = _GMU + _GS * rng.normal(size=6)
        im = _GS ** 2 * rng.uniform(0.5, 2.0, 6)
        eps = O.step_search_gauss(_GMU, _GS, x, im, seed, key, search, eps0)
        t_end = int(round(np.log2(eps / eps0)))
        assert abs(eps / (eps0 * 2.0 ** t_end) - 1) < 1e-12
        thr = np.log(0.8)
        acc = lambda t, e: _gauss_one_step_logacc(x, im, _box_muller6(O.uniforms8(seed, key, search, 1, t)), e)
        up = acc(0, eps0) > thr
        assert (t_end > 0) == up and t_end != 0
        for t in range(abs(t_end)):          # every earlier trial continued the search
            e = eps0 * 2.0 ** (t if up else -t)
            assert (acc(t, e) > thr) == up, (t, e)
        assert (acc(abs(t_end), eps) > thr) != up   # and this one ended it


def test_dual_averaging_drives_the_mean_acceptance_to_the_target():
    # Dual averaging solves E[a] = delta for the statistic the chain sees, so
    # the mean statistic over the second half of a long warmup (no metric
    # windows) is delta; a larger delta needs a smaller step.  The warmup ends
    # on eps-bar: the returned step is exp of the averaged iterate of the
    # statistics, restarted at the initial search.
    C, W = 8, 1000
    init = _GMU + _GS * np.random.default_rng(0).normal(size=(C, 6))
    med = []
    for delta in (0.6, 0.8, 0.95):
        r = O.hmc_gauss(_GMU, _GS, init, n_warmup=W, n_samples=1, n_leapfrog=8, target_accept=delta,
                        adapt_mass=False, seed=5, chain_key0=100)
        a = r["warm_stat"]
        assert np.abs(a[:, W // 2:].mean(axis=1) - delta).max() < 0.01, (delta, a[:, W // 2:].mean(axis=1))
        for c in range(C):
            eps0 = O.step_search_gauss(_GMU, _GS, init[c], np.ones(6), 5, 100 + c, 0, 1.0)
            _, lebar = O.dual_averaging(a[c], delta, eps0)
            assert abs(r["step_size"][c] / np.exp(lebar[-1]) - 1) < 1e-12
        med.append(np.median(r["step_size"]))
    assert med[0] > med[1] > med[2], med


def test_windowed_metric_adapts_to_the_target_variances():
    # Stan's windows estimate the diagonal inverse metric as the regularised
    # variance of the window's draws, so it approaches diag(s^2) of the target.
    C = 8
    init = _GMU + _GS * np.random.default_rng(1).normal(size=(C, 6))
    r = O.hmc_gauss(_GMU, _GS, init, n_warmup=1000, n_samples=1, n_leapfrog=8, target_accept=0.8,
                    adapt_mass=True, seed=9)
    ratio = (r["inv_mass"] / _GS ** 2).mean(axis=0)
    assert np.abs(ratio - 1).max() < 0.15, ratio


@pytest.mark.slow
def test_hmc_matches_laplace_on_bright_galaxy():
    """High S/N: the posterior is close to a Gaussian with covariance (-H)^-1 at
    the mode; the sampler's moments must agree within Monte Carlo error."""
    N = 25
    theta = np.array([np.log10(2000.0), np.log10(0.6), 0.2, -0.1, 0.1, -0.2])
    rng = np.random.default_rng(3)
    data = O.render(N, 0.2, (O.PSF_GAUSSIAN, 0.7), theta) + rng.normal(0, 1, (N, N))
    f = lambda t: -O.logpost(N, 0.2, (O.PSF_GAUSSIAN, 0.7), data, 1.0, t)[0]
    gr = lambda t: -O.logpost(N, 0.2, (O.PSF_GAUSSIAN, 0.7), data, 1.0, t)[1]
    mode = so.minimize(f, theta, jac=gr, method="BFGS", options={"gtol": 1e-9}).x
    H = np.zeros((6, 6))
    for j in range(6):
        h = 1e-5
        tp, tm = mode.copy(), mode.copy()
        tp[j] += h
        tm[j] -= h
        H[:, j] = (gr(tp) - gr(tm)) / (2 * h)
    cov = np.linalg.inv(0.5 * (H + H.T))
    C = 4
    init = np.repeat(mode[None, None, :], C, axis=1) + rng.normal(0, 1e-3, (1, C, 6))
    out = O.fit_galaxies(data[None], 1.0, (O.PSF_GAUSSIAN, 0.7), init, n_warmup=300, n_samples=1000,
                         n_leapfrog=16, random_steps=True, seed=5)
    s = out["samples"][:, 0]                     # [6, C, S]
    flat = s.reshape(6, -1)
    for k in range(6):
        ess = O.ess(s[k])
        sd = np.sqrt(cov[k, k])
        assert abs(flat[k].mean() - mode[k]) < 5 * sd / np.sqrt(ess) + 0.05 * sd, k
        assert abs(flat[k].std() / sd - 1) < 0.12, (k, flat[k].std() / sd)
        assert O.rhat(s[k]) < 1.01


# ---- all properties free: skew-normal log-flux, normal log-size (Eq. lflux-lsize-dist)

def test_log_ndtr_matches_scipy():
    from scipy import special
    for t in np.concatenate([np.linspace(-80.0, 12.0, 185), [-20.0, -20.000001, -19.99999, 5.0, 5.000001]]):
        ref = special.log_ndtr(t)
        assert abs(O.log_ndtr(t) - ref) <= 1e-11 * max(1.0, abs(ref)), (t, O.log_ndtr(t), ref)


def test_log_skewnorm_matches_scipy_and_normalises():
    from scipy import integrate, stats
    rng = np.random.default_rng(8)
    for _ in range(200):
        mu, sig, a = rng.uniform(-2, 6), rng.uniform(0.05, 2), rng.uniform(-100, 100)
        x = mu + sig * rng.normal(0, 3)
        ref = stats.skewnorm.logpdf(x, a, loc=mu, scale=sig)
        if np.isfinite(ref) and ref > -700:
            assert abs(O.log_skewnorm(x, mu, sig, a) - ref) <= 1e-9 * max(1.0, abs(ref)), (x, mu, sig, a)
    # the paper's log-flux distribution integrates to one
    tot, _ = integrate.quad(lambda x: np.exp(O.log_skewnorm(x, 2.45, 0.4, 14.0)), -2, 8, points=[2.45], limit=200)
    assert abs(tot - 1.0) < 1e-9


def _full_inputs(rng, n, K, const_fs=False):
    e1, e2 = [], []
    for _ in range(n):
        r = 0.25 * np.sqrt(rng.uniform(0, 1, K))
        ph = rng.uniform(0, 2 * np.pi, K)
        e1.append(r * np.cos(ph))
        e2.append(r * np.sin(ph))
    e1, e2 = np.array(e1, np.float32), np.array(e2, np.float32)
    if const_fs:
        lf = np.repeat(rng.uniform(2.3, 3.3, (n, 1)), K, axis=1).astype(np.float32)
        ls = np.repeat(rng.normal(-0.4, 0.05, (n, 1)), K, axis=1).astype(np.float32)
    else:
        lf = rng.uniform(2.3, 3.3, (n, K)).astype(np.float32)
        ls = rng.normal(-0.4, 0.06, (n, K)).astype(np.float32)
    return e1, e2, lf, ls


def test_full_loglike_reduces_to_ellipticity_part_plus_constants():
    """With one log-flux and log-size per galaxy (the same for all its samples)
    the flux/size ratio is a per-galaxy constant: the value is the
    ellipticity-only likelihood plus the sum of the scipy log densities, and
    the hyperparameter gradient is the sum of their parameter derivatives
    (central differences of scipy)."""
    from scipy import stats
    rng = np.random.default_rng(12)
    e1, e2, lf, ls = _full_inputs(rng, 6, 9, const_fs=True)
    th = np.array([0.02, -0.01, 0.22, 2.5, 0.45, 9.0, -0.38, 0.06])
    v, g = O.shear_loglike_full(e1, e2, lf, ls, th, family=O.EPRIOR_BA14)
    ve, ge = O.shear_loglike(e1, e2, th[0], th[1], th[2], family=O.EPRIOR_BA14)

    def b_sum(h):
        x, y = lf[:, 0].astype(np.float64), ls[:, 0].astype(np.float64)
        return float(np.sum(stats.skewnorm.logpdf(x, h[2], loc=h[0], scale=h[1]) +
                            stats.norm.logpdf(y, loc=h[3], scale=h[4]) + np.log(10.0) + np.log(3.0)))

    assert abs(v - (ve + b_sum(th[3:]))) < 1e-9 * max(1.0, abs(v))
    assert np.allclose(g[:3], ge, rtol=1e-10, atol=1e-10)
    for i in range(5):
        h = 1e-6 * max(1.0, abs(th[3 + i]))
        hp, hm = th[3:].copy(), th[3:].copy()
        hp[i] += h
        hm[i] -= h
        fd = (b_sum(hp) - b_sum(hm)) / (2 * h)
        assert abs(g[3 + i] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, g[3 + i], fd)


def test_full_loglike_gradient_by_central_differences():
    rng = np.random.default_rng(13)
    e1, e2, lf, ls = _full_inputs(rng, 5, 12)
    for fam in (O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS):
        th = np.array([0.03, 0.02, 0.24, 2.55, 0.5, 6.0, -0.41, 0.07])
        v, g = O.shear_loglike_full(e1, e2, lf, ls, th, family=fam)
        assert np.isfinite(v)
        for i in range(8):
            h = 1e-6 * max(1.0, abs(th[i]))
            tp, tm = th.copy(), th.copy()
            tp[i] += h
            tm[i] -= h
            fd = (O.shear_loglike_full(e1, e2, lf, ls, tp, family=fam)[0] -
                  O.shear_loglike_full(e1, e2, lf, ls, tm, family=fam)[0]) / (2 * h)
            assert abs(g[i] - fd) <= 2e-5 * max(1.0, abs(fd)), (fam, i, g[i], fd)


def test_weighted_likelihood_equals_duplicated_galaxies():
    """Integer galaxy weights (a bootstrap resample) give exactly the likelihood
    of the sample in which each galaxy appears that many times; weight 0
    removes a galaxy."""
    rng = np.random.default_rng(31)
    n, K = 7, 11
    e1 = (0.3 * rng.uniform(-1, 1, (n, K))).astype(np.float32)
    e2 = (0.3 * rng.uniform(-1, 1, (n, K))).astype(np.float32)
    w = np.array([0, 1, 2, 3, 1, 0, 2], dtype=np.float32)
    rep = np.repeat(np.arange(n), w.astype(int))
    for fam in (O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS):
        vw, gw = O.shear_loglike(e1, e2, 0.03, -0.02, 0.25, family=fam, weights=w)
        vr, gr = O.shear_loglike(e1[rep], e2[rep], 0.03, -0.02, 0.25, family=fam)
        assert abs(vw - vr) <= 1e-12 * max(1.0, abs(vr))
        assert np.allclose(gw, gr, rtol=1e-12, atol=1e-12)
    lf = rng.uniform(1.5, 4.0, (n, K)).astype(np.float32)
    ls = rng.uniform(-1.0, 0.3, (n, K)).astype(np.float32)
    th = (0.03, -0.02, 0.25, 2.45, 0.4, 5.0, -0.4, 0.2)
    vw, gw = O.shear_loglike_full(e1, e2, lf, ls, th, weights=w)
    vr, gr = O.shear_loglike_full(e1[rep], e2[rep], lf[rep], ls[rep], th)
    assert abs(vw - vr) <= 1e-12 * max(1.0, abs(vr)) and np.allclose(gw, gr, rtol=1e-12, atol=1e-12)
    mw, cw = O.shear_estimate(e1, e2, family=O.EPRIOR_BA14, alpha=0.25, weights=w)
    mr, cr = O.shear_estimate(e1[rep], e2[rep], family=O.EPRIOR_BA14, alpha=0.25)
    assert np.allclose(mw, mr, rtol=1e-9, atol=1e-12) and np.allclose(cw, cr, rtol=1e-8, atol=1e-14)


# ---- Appendix C: pixel covariance and exposures ------------------------------------------

def _cov_case(N=11, J=2, a=0.3, seed=5):
    rng = np.random.default_rng(seed)
    th = np.array([2.3, -0.45, 0.12, -0.2, 0.3, -0.25])
    psfs = [(O.PSF_GAUSSIAN, 0.7), (O.PSF_MOFFAT, 0.9, 3.0)][:J]
    sig = np.array([1.0, 1.7])[:J]
    corr = np.stack([synth.noise_correlation(N, a)] * J)
    noise = synth.correlated_noise(rng, J, N, a)
    data = np.stack([O.render(N, 0.2, psfs[j], th) + sig[j] * noise[j] for j in range(J)])
    return N, th, psfs, sig, corr, data


def _circulant(corr, s2):
    """Dense pixel covariance s2 corr(x_a - x_b), lags wrapped to -c..c."""
    N = corr.shape[0]
    c = (N - 1) // 2
    y, x = np.divmod(np.arange(N * N), N)
    dy = (y[:, None] - y[None, :] + c) % N
    dx = (x[:, None] - x[None, :] + c) % N
    return s2 * corr[dy, dx]


def test_loglike_cov_white_is_the_pixel_likelihood():
    """One exposure, white noise: the covariance form is Eq. likelihood-pixels."""
    N, th, psfs, sig, corr, data = _cov_case(J=1)
    v, g = O.loglike_cov(N, 0.2, psfs, data, sig, th)
    vr, gr = O.loglike(N, 0.2, psfs[0], data[0], sig[0], th)
    assert abs(v - vr) <= 1e-11 * abs(vr) and np.allclose(g, gr, rtol=1e-10, atol=1e-10)


def test_loglike_cov_matches_multivariate_normal_and_the_circulant_spectrum():
    """Two exposures (Gaussian and Moffat PSFs, sigma 1 and 1.7) with
    correlated noise: the value equals scipy's multivariate normal log density
    of each exposure without its normalisation, and the circulant identity
    r^T Sigma^-1 r = sum_k |R_k|^2 / (sigma^2 N^2 lambda_k), lambda = FFT of the
    correlation at lag."""
    from scipy import stats
    N, th, psfs, sig, corr, data = _cov_case()
    v, _ = O.loglike_cov(N, 0.2, psfs, data, sig, th, corr=corr)
    ref = fft = 0.0
    for j in range(2):
        m = O.render(N, 0.2, psfs[j], th)
        S = _circulant(corr[j], sig[j] ** 2)
        _, logdet = np.linalg.slogdet(2 * np.pi * S)
        ref += stats.multivariate_normal(mean=m.ravel(), cov=S).logpdf(data[j].ravel()) + 0.5 * logdet
        lam = np.fft.fft2(np.fft.ifftshift(corr[j])).real
        R = np.fft.fft2(data[j] - m)
        fft += -0.5 * (np.abs(R) ** 2 / lam).sum() / (sig[j] ** 2 * N * N)
    assert abs(v - ref) <= 1e-9 * abs(ref), (v, ref)
    assert abs(v - fft) <= 1e-9 * abs(fft), (v, fft)


def test_loglike_cov_gradient_central_differences():
    N, th, psfs, sig, corr, data = _cov_case()
    _, g = O.loglike_cov(N, 0.2, psfs, data, sig, th, corr=corr)
    for i in range(6):
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.loglike_cov(N, 0.2, psfs, data, sig, tp, corr=corr)[0] -
              O.loglike_cov(N, 0.2, psfs, data, sig, tm, corr=corr)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), (i, fd, g[i])


def _dense_case(N=11, seed=8):
    rng = np.random.default_rng(seed)
    th = np.array([2.3, -0.45, 0.12, -0.2, 0.3, -0.25])
    psf = (O.PSF_MOFFAT, 0.8, 3.0)
    S = synth.dense_covariance(N, rng)
    data = O.render(N, 0.2, psf, th) + synth.dense_noise(S, rng)
    return N, th, psf, S, data


def test_loglike_dense_reduces_to_the_white_and_stationary_cases():
    """Sigma = sigma^2 I is Eq. likelihood-pixels; a circulant Sigma is the
    stationary correlated-noise likelihood of one exposure."""
    N, th, psf, _, data = _dense_case()
    v, g = O.loglike_dense(N, 0.2, psf, data, 1.7 ** 2 * np.eye(N * N), th)
    vr, gr = O.loglike(N, 0.2, psf, data, 1.7, th)
    assert abs(v - vr) <= 1e-11 * abs(vr) and np.allclose(g, gr, rtol=1e-10, atol=1e-10)
    corr = synth.noise_correlation(N, 0.3)
    v, g = O.loglike_dense(N, 0.2, psf, data, _circulant(corr, 1.3 ** 2), th)
    vr, gr = O.loglike_cov(N, 0.2, [psf], data[None], np.array([1.3]), th, corr=corr[None])
    assert abs(v - vr) <= 1e-9 * abs(vr) and np.allclose(g, gr, rtol=1e-8, atol=1e-9)


def test_loglike_dense_matches_multivariate_normal():
    """A Sigma that is neither stationary nor diagonal: the value is scipy's
    multivariate normal log density of the stamp without its normalisation."""
    from scipy import stats
    N, th, psf, S, data = _dense_case()
    v, _ = O.loglike_dense(N, 0.2, psf, data, S, th)
    m = O.render(N, 0.2, psf, th)
    _, logdet = np.linalg.slogdet(2 * np.pi * S)
    ref = stats.multivariate_normal(mean=m.ravel(), cov=S).logpdf(data.ravel()) + 0.5 * logdet
    assert abs(v - ref) <= 1e-9 * abs(ref), (v, ref)


def test_loglike_dense_gradient_central_differences():
    N, th, psf, S, data = _dense_case()
    _, g = O.loglike_dense(N, 0.2, psf, data, S, th)
    for i in range(6):
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.loglike_dense(N, 0.2, psf, data, S, tp)[0] - O.loglike_dense(N, 0.2, psf, data, S, tm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_loglike_cov_rejects_a_covariance_that_is_not_positive_definite():
    N, th, psfs, sig, corr, data = _cov_case(J=1)
    bad = np.zeros((1, N, N))
    c = (N - 1) // 2
    bad[0, c, c] = 1.0
    bad[0, c + 1, c] = bad[0, c - 1, c] = bad[0, c, c + 1] = bad[0, c, c - 1] = 0.8
    v, _ = O.loglike_cov(N, 0.2, psfs, data, sig, th, corr=bad)
    assert np.isnan(v)


# ---- Appendix B: Spergel and Gaussian profiles ---------------------------------------------

def _spergel_radial(x, nu):
    """Unnormalised Spergel profile x^nu K_nu(x), x = r / r0 (scipy's kv)."""
    return x ** nu * sp.kv(nu, x)


@pytest.mark.parametrize("nu", [-0.6, 0.0, 0.5, 1.5, 3.0])
def test_spergel_half_light_radius_encloses_half_the_flux(nu):
    """hlr / r0 from the oracle's closed-form enclosed flux (its own Bessel K)
    against scipy quadrature of the real-space profile x^nu K_nu(x)."""
    h = O.hlr_over_r0(O.PROFILE_SPERGEL, nu)
    f = lambda x: _spergel_radial(x, nu) * x
    inside = si.quad(f, 0, h, limit=200)[0]
    total = si.quad(f, 0, h, limit=200)[0] + si.quad(f, h, np.inf, limit=200)[0]
    assert abs(inside / total - 0.5) < 1e-8, (nu, h, inside / total)
    if nu == 0.5:
        assert abs(h - O.hlr_over_r0()) < 1e-10


@pytest.mark.parametrize("nu", [-0.6, 1.5])
def test_spergel_transform_is_the_hankel_transform_of_the_profile(nu):
    """(1 + k^2 r0^2)^-(1+nu) is the unit-flux 2-D transform of x^nu K_nu(x)
    (r0 = 1): int I(r) J0(k r) r dr / int I(r) r dr by quadrature."""
    f = lambda x: _spergel_radial(x, nu) * x
    total = si.quad(f, 0, 1, limit=200)[0] + si.quad(f, 1, np.inf, limit=200)[0]
    for k in (0.3, 1.0, 2.5):
        num = si.quad(lambda x: f(x) * sp.j0(k * x), 0, 1, limit=400)[0] + \
            si.quad(lambda x: f(x) * sp.j0(k * x), 1, 80, limit=800)[0]
        assert abs(num / total - O.profile_ft(O.PROFILE_SPERGEL, nu, k * k)) < 2e-6, (nu, k)


def test_gaussian_profile_transform_and_half_light_radius():
    s = 1.0
    f = lambda x: np.exp(-0.5 * x * x) * x
    h = O.hlr_over_r0(O.PROFILE_GAUSSIAN, 0.0)
    assert abs(si.quad(f, 0, h)[0] / si.quad(f, 0, np.inf)[0] - 0.5) < 1e-12
    for k in (0.3, 1.0, 2.5):
        num = si.quad(lambda x: f(x) * sp.j0(k * x), 0, 40, limit=400)[0]
        assert abs(num / si.quad(f, 0, np.inf)[0] - O.profile_ft(O.PROFILE_GAUSSIAN, 0.0, (k * s) ** 2)) < 1e-9


def _profile_case(seed=3, N=15):
    rng = np.random.default_rng(seed)
    th = np.array([2.4, -0.4, 0.15, -0.1, 0.2, -0.3])
    data = O.render(N, 0.2, (O.PSF_GAUSSIAN, 0.7), th) + rng.normal(size=(N, N))
    return N, th, data


def test_spergel_half_is_the_exponential_likelihood():
    N, th, data = _profile_case()
    v, g = O.loglike_p(O.PROFILE_SPERGEL, 0.5, N, 0.2, (O.PSF_GAUSSIAN, 0.7), data, 1.0, th)
    vr, gr = O.loglike(N, 0.2, (O.PSF_GAUSSIAN, 0.7), data, 1.0, th)
    assert abs(v - vr) <= 1e-10 * abs(vr) and np.allclose(g, gr, rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("profile,nu", [(1, -0.6), (1, 2.0), (2, 0.0)])
def test_profile_likelihood_gradient_central_differences(profile, nu):
    N, th, data = _profile_case()
    psf = (O.PSF_MOFFAT, 0.8, 3.0)
    _, g = O.loglike_p(profile, nu, N, 0.2, psf, data, 1.0, th)
    for i in range(6):
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (O.loglike_p(profile, nu, N, 0.2, psf, data, 1.0, tp)[0] -
              O.loglike_p(profile, nu, N, 0.2, psf, data, 1.0, tm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), (profile, nu, i, fd, g[i])


def test_weighted_loglike_is_the_weighted_pixel_chi2():
    """Appendix C, spatially variable noise: -1/2 sum w (d - m)^2 / sigma^2 with m
    the oracle's rendered image, summed by numpy; pixels of weight 0 (a mask)
    do not enter, whatever their data."""
    rng = np.random.default_rng(12)
    N, sig = 23, 1.4
    th = np.array([2.5, -0.4, 0.1, 0.2, -0.3, 0.15])
    psf = (O.PSF_MOFFAT, 0.8, 3.0)
    m = O.render(N, 0.2, psf, th)
    data = m + rng.normal(0, sig, (N, N))
    w = rng.uniform(0.2, 2.0, (N, N))
    w[3:7, 10:18] = 0.0
    v, g = O.loglike(N, 0.2, psf, data, sig, th, weights=w)
    assert abs(v - (-0.5 * (w * (data - m) ** 2).sum() / sig ** 2)) < 1e-9 * abs(v)
    bad = data.copy()
    bad[3:7, 10:18] = 1e6
    vb, gb = O.loglike(N, 0.2, psf, bad, sig, th, weights=w)
    assert abs(vb - v) < 1e-9 * abs(v) and np.allclose(gb, g, rtol=1e-9, atol=1e-9)
