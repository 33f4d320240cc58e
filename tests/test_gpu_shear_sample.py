"""Shear sampling phase as MCMC (bs_shear_sample): HMC on g and hyperparameters
with the GPU likelihood at every leapfrog step, checked against posterior
means the oracle or the mathematics fix."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _interim_ellipticities(n, K, g, seed):
    """Ellipticity-only interim samples: intrinsic shapes from the workload's
    truncated Gaussian, sheared by g, scattered by measurement noise."""
    rng = np.random.default_rng(seed)
    t = synth.draw_plain(n, 25, seed=seed)
    ep = np.array([O.shear_apply(a, b, *g) for a, b in t.e_int])
    noise = rng.normal(0, 0.05, (n, K, 2))
    return ((ep[:, None, 0] + noise[..., 0]).astype(np.float32),
            (ep[:, None, 1] + noise[..., 1]).astype(np.float32))


def _mcse(x):
    return x.std() / math.sqrt(O.ess(x[None, :].astype(np.float64)))


def _check_g_sigma(draws, e1, e2):
    mo, _ = O.shear_estimate(e1, e2, family=O.EPRIOR_TRUNC_GAUSS, free_alpha=True, alpha=0.2,
                             alpha_lo=0.1, alpha_hi=0.4)
    for k in range(3):
        x = draws[:, k]
        assert abs(x.mean() - mo[k]) < 4.5 * _mcse(x) + 1e-6, (k, x.mean(), mo[k], _mcse(x))


LO = [-1, -1, 0.1, -2.0, 0.0, -100.0, -2.0, 0.0]
HI = [1, 1, 0.4, 6.0, 2.0, 100.0, 2.0, 0.5]


def test_sample_g_sigma_matches_gauss_hermite(cuda):
    e1, e2 = _interim_ellipticities(3000, 24, (0.02, -0.01), 41)
    t = lambda a: torch.from_numpy(a).to(cuda)
    plan = api.ShearPlan(t(e1), t(e2), family=O.EPRIOR_TRUNC_GAUSS, trunc_r=0.7)
    th0 = [0.0, 0.0, 0.22, 2.45, 0.4, 14.0, -0.4, 0.05]
    draws, info = plan.sample(th0, free=("g1", "g2", "sigma_e"), lo=LO, hi=HI, n_warmup=400, n_samples=3000,
                              n_leapfrog=8, seed=5)
    assert 0.5 < info["accept_rate"] <= 1.0
    assert np.all(draws[:, 3:] == np.array(th0[3:]))
    _check_g_sigma(draws, e1, e2)


def test_sample_all_free_factorises(cuda):
    """One log-flux and log-size per galaxy (the same for its samples): the
    flux/size ratio no longer couples to g, so (g, sigma_e) follow the
    ellipticity-only posterior, and (mu_s, sigma_s) the flat-prior normal
    posterior: E[mu_s] = mean(y), E[sigma_s] = sqrt(S/2) G((n-3)/2)/G((n-2)/2),
    S = sum (y - mean y)^2."""
    n, K = 3000, 24
    e1, e2 = _interim_ellipticities(n, K, (0.02, -0.01), 43)
    rng = np.random.default_rng(44)
    from scipy import stats
    lf_g = stats.skewnorm.rvs(14.0, loc=2.45, scale=0.4, size=n, random_state=rng)
    ls_g = rng.normal(-0.4, 0.05, n)
    lf = np.repeat(lf_g[:, None], K, axis=1).astype(np.float32)
    ls = np.repeat(ls_g[:, None], K, axis=1).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    plan = api.ShearPlan(t(e1), t(e2), family=O.EPRIOR_TRUNC_GAUSS, trunc_r=0.7)
    th0 = [0.0, 0.0, 0.22, 2.5, 0.45, 10.0, -0.39, 0.06]
    draws, info = plan.sample(th0, free=("g1", "g2", "sigma_e", "mu_f", "sigma_f", "a_f", "mu_s", "sigma_s"),
                              lf=t(lf), ls=t(ls), lo=LO, hi=HI, n_warmup=1000, n_samples=4000, n_leapfrog=10,
                              seed=7)
    assert 0.5 < info["accept_rate"] <= 1.0
    assert np.isfinite(draws).all()
    _check_g_sigma(draws, e1, e2)
    y = ls[:, 0].astype(np.float64)
    S = ((y - y.mean()) ** 2).sum()
    e_sig = math.sqrt(S / 2) * math.exp(math.lgamma((n - 3) / 2) - math.lgamma((n - 2) / 2))
    for k, ref in ((6, y.mean()), (7, e_sig)):
        x = draws[:, k]
        assert abs(x.mean() - ref) < 4.5 * _mcse(x), (k, x.mean(), ref, _mcse(x))
    # the skew-normal hyperparameters land near the values that drew the fluxes
    for k, true in ((3, 2.45), (4, 0.4), (5, 14.0)):
        x = draws[:, k]
        assert abs(x.mean() - true) < 5 * x.std() + 0.05 * abs(true), (k, x.mean(), x.std(), true)


def test_sample_allreduce_hook(cuda):
    """A hook that doubles each evaluation stands for two ranks holding the same
    galaxies: the posterior keeps its mean and narrows by sqrt(2)."""
    e1, e2 = _interim_ellipticities(2000, 24, (0.02, -0.01), 45)
    t = lambda a: torch.from_numpy(a).to(cuda)
    plan = api.ShearPlan(t(e1), t(e2), family=O.EPRIOR_TRUNC_GAUSS, trunc_r=0.7)
    th0 = [0.02, -0.01, 0.2, 2.45, 0.4, 14.0, -0.4, 0.05]
    one, _ = plan.sample(th0, free=("g1", "g2"), n_warmup=300, n_samples=3000, seed=11)
    two, info = plan.sample(th0, free=("g1", "g2"), n_warmup=300, n_samples=3000, seed=11,
                            allreduce=lambda x: 2.0 * x)
    assert info["accept_rate"] > 0.5
    for k in range(2):
        ratio = two[:, k].std() / one[:, k].std()
        assert 0.6 < ratio < 0.85, (k, ratio)
        assert abs(two[:, k].mean() - one[:, k].mean()) < 4.5 * math.hypot(_mcse(one[:, k]), _mcse(two[:, k]))
