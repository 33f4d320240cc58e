"""Per-galaxy weights in the shear stage (bootstrap resamples, Sec. 3.4):
weighted likelihoods and estimates against the oracle, zero weights, and the
bootstrap errors of m and c on the Appendix-A toy."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import _ffi as F
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _resample(n, rng):
    """Counts of n galaxies drawn with replacement (float32 [n])."""
    return np.bincount(rng.integers(0, n, n), minlength=n).astype(np.float32)


def _samples(rng, n, K, spread):
    e = rng.normal(0.0, spread, (n, K, 2))
    r = np.hypot(e[..., 0], e[..., 1])
    e[r > 0.9] *= (0.9 / r[r > 0.9])[:, None]
    return e[..., 0].astype(np.float32), e[..., 1].astype(np.float32)


def _weights(rng, n):
    w = rng.uniform(0.0, 3.0, n).astype(np.float32)
    w[rng.uniform(size=n) < 0.2] = 0.0
    return w


@pytest.mark.parametrize("family", [O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS])
@pytest.mark.parametrize("K,with_b", [(300, False), (300, True), (37, False), (1, True)])
def test_weighted_loglike_matches_oracle(cuda, family, K, with_b):
    """Both kernels (cp.async ring for K % 4 == 0, register pipeline
    otherwise), real-valued weights with a fifth of them zero; the noalloc
    entry point reads the same weights."""
    rng = np.random.default_rng(100 + K + 7 * family)
    n = 2000
    e1, e2 = _samples(rng, n, K, 0.12 if family == O.EPRIOR_TRUNC_GAUSS else 0.2)
    b = rng.normal(0, 0.7, (n, K)).astype(np.float32) if with_b else None
    w = _weights(rng, n)
    t = lambda a: None if a is None else torch.from_numpy(a).to(cuda)
    plan = api.ShearPlan(t(e1), t(e2), t(b), family=family, weights=w)
    out = torch.empty(4, dtype=torch.float64, device=cuda)
    for (g1, g2, a) in [(0.02, 0.0, 0.2), (-0.04, 0.03, 0.27)]:
        got = plan.loglike(g1, g2, a, host=True)
        v, gr = O.shear_loglike(e1, e2, g1, g2, a, b=b, family=family, weights=w)
        assert np.isfinite(v)
        assert abs(got[0] - v) <= 1e-5 * max(abs(v), n), (got[0], v)
        assert np.abs(got[1:] - gr).max() <= 1e-4 * np.abs(gr).max() + 1e-6 * n, (got[1:], gr)
        F.check(F.lib().bs_shear_loglike_noalloc(C.byref(plan.data), g1, g2, a, out.data_ptr(),
                                                  torch.cuda.current_stream().cuda_stream))
        assert np.array_equal(out.cpu().numpy(), got)


@pytest.mark.parametrize("family", [O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS])
def test_weighted_full_matches_oracle(cuda, family):
    rng = np.random.default_rng(31 + family)
    n, K = 1500, 96
    e1, e2 = _samples(rng, n, K, 0.12 if family == O.EPRIOR_TRUNC_GAUSS else 0.2)
    lf = rng.normal(2.8, 0.35, (n, K)).astype(np.float32)
    ls = rng.normal(-0.4, 0.06, (n, K)).astype(np.float32)
    w = _weights(rng, n)
    t = lambda a: torch.from_numpy(a).to(cuda)
    plan = api.ShearPlan(t(e1), t(e2), family=family, weights=t(w))
    th = [0.02, -0.01, 0.21, 2.45, 0.4, 14.0, -0.4, 0.05]
    got_v, got_g = plan.loglike_full(t(lf), t(ls), th)
    v, g = O.shear_loglike_full(e1, e2, lf, ls, th, family=family, weights=w)
    assert abs(got_v - v) <= 1e-5 * max(abs(v), n), (got_v, v)
    assert np.abs(got_g - g).max() <= 1e-4 * np.abs(g).max() + 1e-6 * n, (got_g, g)


def test_zero_weight_drops_a_zero_likelihood_galaxy(cuda):
    """Truncated Gaussian: a galaxy with every sample beyond R makes the value
    -inf; weighted 0 it is left out and the rest matches the oracle."""
    rng = np.random.default_rng(8)
    e1, e2 = _samples(rng, 64, 40, 0.1)
    e1[5] = e2[5] = 0.8
    w = np.ones(64, np.float32)
    t = lambda a: torch.from_numpy(a).to(cuda)
    plan = api.ShearPlan(t(e1), t(e2), family=O.EPRIOR_TRUNC_GAUSS)
    assert plan.loglike(0.0, 0.0, 0.2, host=True)[0] == -np.inf
    with pytest.raises(F.BsError, match="weight 0"):     # fails loudly, no NaN estimate
        plan.estimate(alpha=0.2)
    w[5] = 0.0
    plan.set_weights(w)
    assert np.isfinite(plan.estimate(alpha=0.2)[0]).all()
    got = plan.loglike(0.01, 0.0, 0.2, host=True)
    keep = np.arange(64) != 5
    v, gr = O.shear_loglike(e1[keep], e2[keep], 0.01, 0.0, 0.2, family=O.EPRIOR_TRUNC_GAUSS)
    assert abs(got[0] - v) <= 1e-5 * abs(v) and np.abs(got[1:] - gr).max() <= 1e-4 * np.abs(gr).max()
    plan.set_weights(None)
    assert plan.loglike(0.0, 0.0, 0.2, host=True)[0] == -np.inf


def test_weighted_estimate_matches_oracle(cuda):
    rng = np.random.default_rng(12)
    n, K = 3000, 32
    e_int = synth.draw_ba14_e(rng, n, sigma=0.2)
    e1, e2 = synth.toy_interim_ellipticities(e_int, (0.02, -0.01), K, rng, n_prop=300)
    w = _resample(n, rng)
    plan = api.ShearPlan(torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda), weights=w)
    mg, cg = plan.estimate(free_alpha=True, alpha=0.2, alpha_lo=0.1, alpha_hi=0.4)
    mo, co = O.shear_estimate(e1, e2, family=O.EPRIOR_BA14, free_alpha=True, alpha=0.2, alpha_lo=0.1,
                              alpha_hi=0.4, weights=w)
    assert np.abs(mg - mo).max() < 2e-6, (mg, mo)
    # covariance relative to the scale of its entries, sqrt(c_ii c_jj): the
    # cross terms are ~1e-4 of it and carry the FP32 rounding of the passes
    scale = np.sqrt(np.outer(np.diag(co), np.diag(co)))
    assert np.abs(cg - co).max() <= 1e-3 * scale.min(), (cg, co)


def test_bootstrap_bias_on_the_toy(cuda):
    """The +g / -g toy pair (same intrinsic shapes and noise, g1 = 0.02):
    m is consistent with 0 within 3.5 bootstrap sigma; m and c are those of
    the unweighted estimates; the bootstrap spread of one dataset's g1 matches
    its posterior sd (the estimate is the posterior mean)."""
    n, K, g = 20000, 100, 0.02
    rng = np.random.default_rng(77)
    e_int = synth.draw_ba14_e(rng, n, sigma=0.2)
    t = lambda a: torch.from_numpy(a).to(cuda)
    plans = []
    for sgn in (1, -1):
        e1, e2 = synth.toy_interim_ellipticities(e_int, (sgn * g, 0.0), K, np.random.default_rng(78), n_prop=500)
        plans.append(api.ShearPlan(t(e1), t(e2)))
    r = api.shear_bias_plans(*plans, g_abs=g, n_boot=100, seed=3, alpha=0.2)
    gp, cov = plans[0].estimate(alpha=0.2)
    gm, _ = plans[1].estimate(alpha=0.2)
    assert r["m"] == (gp[0] - gm[0]) / (2 * g) - 1 and r["c"] == 0.5 * (gp[1] + gm[1])
    assert np.isfinite(r["m_sd"]) and r["m_sd"] > 0
    assert abs(r["m"]) < 3.5 * r["m_sd"], r
    assert abs(r["c"]) < 3.5 * r["c_sd"], r
    assert plans[0].data.gal_weight is None
    boot = []
    brng = np.random.default_rng(5)
    for _ in range(100):
        plans[0].set_weights(_resample(n, brng), float(n))
        boot.append(plans[0].estimate(alpha=0.2)[0][0])
    ratio = np.std(boot, ddof=1) / np.sqrt(cov[0, 0])
    assert 0.75 < ratio < 1.3, ratio
