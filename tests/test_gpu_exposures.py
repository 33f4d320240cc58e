"""Appendix C on the GPU: several exposures of a galaxy with their own PSFs and
stationary correlated pixel noise, folded into one spectrum at setup.  Log
posterior and gradient against the oracle's dense pixel-space covariance
likelihood; the fit on folded exposures against the fit on their
inverse-variance mean; the status of a correlation that is no covariance."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu

P = 0.2
PSFS = [(O.PSF_GAUSSIAN, 0.7, 3.0), (O.PSF_MOFFAT, 0.9, 3.0), (O.PSF_MOFFAT, 0.6, 2.5)]


def _galaxies(sides, J, a, seed):
    """Stamps of each galaxy's J exposures back to back, correlated noise
    (a = None: white) with per-exposure sd, oracle-rendered models."""
    rng = np.random.default_rng(seed)
    n = len(sides)
    th = np.stack([[rng.uniform(2.2, 2.6), rng.uniform(-0.55, -0.35), rng.uniform(-0.2, 0.2),
                    rng.uniform(-0.2, 0.2), rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4)] for _ in range(n)])
    sig = rng.uniform(0.8, 1.6, (n, J))
    data, corr, offs = [], [], []
    off = 0
    for i, N in enumerate(sides):
        offs.append(off)
        cr = synth.noise_correlation(N, a) if a is not None else np.zeros((N, N))
        if a is None:
            cr[(N - 1) // 2, (N - 1) // 2] = 1.0
        noise = synth.correlated_noise(rng, J, N, a) if a is not None else rng.normal(size=(J, N, N))
        for j in range(J):
            data.append((O.render(N, P, PSFS[j], th[i]) + sig[i, j] * noise[j]).ravel())
            corr.append(cr.ravel())
        off += J * N * N
    kinds = np.array([PSFS[j][0] for _ in range(n) for j in range(J)], dtype=np.int32)
    fwhm = np.array([PSFS[j][1] for _ in range(n) for j in range(J)], dtype=np.float32)
    beta = np.array([PSFS[j][2] for _ in range(n) for j in range(J)], dtype=np.float32)
    return th, sig, np.concatenate(data), np.concatenate(corr), np.array(offs), kinds, fwhm, beta


def _psf_table(kinds, fwhm, beta, cuda):
    rec = np.zeros(len(kinds), dtype=[("kind", "<i4"), ("fwhm", "<f4"), ("beta", "<f4")])
    rec["kind"], rec["fwhm"], rec["beta"] = kinds, fwhm, beta
    return torch.from_numpy(rec.view(np.uint8).copy()).to(cuda), len(kinds)


@pytest.mark.parametrize("sides,J,a", [([25, 31, 35], 2, 0.3), ([33, 27], 3, None), ([29], 1, 0.25)])
def test_logpost_matches_dense_covariance_oracle(cuda, sides, J, a):
    th, sig, data, corr, offs, kinds, fwhm, beta = _galaxies(sides, J, a, seed=len(sides) * 10 + J)
    t = lambda x, dt=torch.float32: torch.as_tensor(x, dtype=dt, device=cuda)
    rng = np.random.default_rng(3)
    pts, gal = [], []
    for i in range(len(sides)):
        for k in range(3):
            pts.append(th[i] + rng.normal(0, [0.02, 0.02, 0.03, 0.03, 0.05, 0.05]))
            gal.append(i)
    pts = np.array(pts, dtype=np.float32)
    lp, g = api.logpost_points(t(data), t(offs, torch.int64), t(sides, torch.int32),
                               _psf_table(kinds, fwhm, beta, cuda), t(sig.ravel()), t(gal, torch.int32), t(pts),
                               pixel_scale=P, n_exposures=J, noise_corr=t(corr) if a is not None else None)
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    for q, i in enumerate(gal):
        N = sides[i]
        d = data[offs[i]:offs[i] + J * N * N].reshape(J, N, N)
        cr = corr[offs[i]:offs[i] + J * N * N].reshape(J, N, N) if a is not None else None
        psfs = [PSFS[j][:2] if PSFS[j][0] == O.PSF_GAUSSIAN else PSFS[j] for j in range(J)]
        vl, gl = O.loglike_cov(N, P, psfs, d, sig[i], pts[q].astype(np.float64), corr=cr)
        vp, gp = O.log_prior(pts[q].astype(np.float64), grad=True)
        v, gr = vl + vp, gl + gp
        assert abs(lp[q] - v) <= 1e-5 * max(abs(v), N * N), (q, lp[q], v)
        assert np.abs(g[q] - gr).max() <= 1e-4 * np.abs(gr).max() + 1e-3, (q, g[q], gr)


def test_folded_exposures_fit_like_their_mean(cuda):
    """J exposures with one PSF and white noise sigma_j carry the likelihood
    of their inverse-variance mean with sigma^-2 = sum sigma_j^-2 (up to a
    constant): the two fits sample the same posterior."""
    sides, J, n, C = [33] * 12, 3, 12, 4
    rng = np.random.default_rng(11)
    sig = np.array([1.0, 1.5, 2.0])
    w = sig ** -2
    stamps, mean = [], []
    psf = (O.PSF_GAUSSIAN, 0.7)
    for i in range(n):
        th = np.array([2.6, -0.4, 0.1 * rng.normal(), 0.1 * rng.normal(), 0.2 * rng.normal(), 0.2 * rng.normal()])
        m = O.render(33, P, psf, th)
        ex = [m + s * rng.normal(size=(33, 33)) for s in sig]
        stamps.append(np.concatenate([e.ravel() for e in ex]))
        mean.append((sum(wj * e for wj, e in zip(w, ex)) / w.sum()).ravel())
    init = np.tile(np.array([2.6, -0.4, 0.0, 0.0, 0.0, 0.0], np.float32), (n, C, 1))
    init += np.random.default_rng(2).normal(0, 0.01, init.shape).astype(np.float32)
    t = lambda x, dt=torch.float32: torch.as_tensor(np.asarray(x), dtype=dt, device=cuda)
    cfg = api.FitConfig(n_chains=C, n_warmup=300, n_samples=600, n_leapfrog=12)
    tab = api.psf_table("gaussian", 0.7, device=cuda)
    multi = api.fit_galaxies(t(np.concatenate(stamps)), t(np.arange(n) * J * 33 * 33, torch.int64),
                             t(sides, torch.int32), tab, t(np.tile(sig, n)), t(init), cfg, n_exposures=J)
    one = api.fit_galaxies(t(np.concatenate(mean)), t(np.arange(n) * 33 * 33, torch.int64), t(sides, torch.int32),
                           tab, t(np.full(n, 1.0 / np.sqrt(w.sum()))), t(init), cfg)
    assert (multi["status"] == 0).all() and (one["status"] == 0).all()
    a, b = multi["samples"].cpu().numpy(), one["samples"].cpu().numpy()
    worst = 0.0
    for i in range(n):
        for k in range(6):
            x, y = a[k, i].astype(np.float64), b[k, i].astype(np.float64)
            se = np.hypot(x.std() / np.sqrt(O.ess(x)), y.std() / np.sqrt(O.ess(y)))
            worst = max(worst, abs(x.mean() - y.mean()) / se)
            assert 0.8 < x.std() / y.std() < 1.25, (i, k)
    assert worst < 5.0, worst


def test_correlation_without_a_covariance_is_status_3(cuda):
    N, J = 25, 1
    c = (N - 1) // 2
    bad = np.zeros((N, N), np.float32)
    bad[c, c] = 1.0
    bad[c + 1, c] = bad[c - 1, c] = bad[c, c + 1] = bad[c, c - 1] = 0.8
    good = synth.noise_correlation(N, 0.3).astype(np.float32)
    t = lambda x, dt=torch.float32: torch.as_tensor(np.asarray(x), dtype=dt, device=cuda)
    data = np.random.default_rng(1).normal(size=2 * N * N)
    init = np.tile(np.array([2.0, -0.4, 0, 0, 0, 0], np.float32), (2, 2, 1))
    cfg = api.FitConfig(n_chains=2, n_warmup=10, n_samples=10, n_leapfrog=4)
    res = api.fit_galaxies(t(data), t([0, N * N], torch.int64), t([N, N], torch.int32),
                           api.psf_table("gaussian", 0.7, device=cuda), t([1.0, 1.0]), t(init), cfg,
                           n_exposures=J, noise_corr=t(np.concatenate([bad.ravel(), good.ravel()])))
    assert list(res["status"].cpu().numpy()) == [3, 0]
