"""Shape-noise cancellation m and c with bootstrap errors (Sec. 3.4): the host
logic of api.shear_bias, with exact fake estimators and with the oracle's
posterior mean as the estimator."""
import numpy as np

import oracle as O
from paper_2604_22048_gb300 import api, synth


def test_bootstrap_weights_are_a_resample():
    rng = np.random.default_rng(3)
    w = api.bootstrap_weights(1000, rng)
    assert w.dtype == np.float32 and w.shape == (1000,)
    assert w.sum() == 1000 and np.all(w == np.round(w)) and w.min() >= 0
    # each count is Binomial(n, 1/n): mean 1, variance ~ 1
    ws = np.stack([api.bootstrap_weights(1000, rng) for _ in range(50)])
    assert abs(ws.var() - (1 - 1 / 1000)) < 0.05


def test_linear_estimator_recovers_m_and_c_exactly():
    """An estimator g_hat = (1 + m0) g + c0 + noise(w), with the same noise in
    the +g and -g datasets: the g1 noise cancels, so every resample gives m0
    (sd 0); c is c0 plus the g2 noise, and its bootstrap sd is that of the
    noise over the same resamples."""
    n, g, m0, c0 = 500, 0.02, 3e-3, np.array([1e-3, -5e-4])
    z = np.random.default_rng(9).normal(0, 0.3, (n, 2))

    def noise(w):
        w = np.ones(n) if w is None else w.astype(np.float64)
        return (w[:, None] * z).sum(0) / w.sum()

    plus = lambda w: (1 + m0) * np.array([g, 0.0]) + c0 + noise(w)
    minus = lambda w: (1 + m0) * np.array([-g, 0.0]) + c0 + noise(w)
    r = api.shear_bias(plus, minus, n, g_abs=g, n_boot=40, seed=5)
    assert abs(r["m"] - m0) < 1e-12 and np.allclose(r["m_boot"], m0, atol=1e-12) and r["m_sd"] < 1e-12
    assert abs(r["c"] - (c0[1] + noise(None)[1])) < 1e-15
    rng = np.random.default_rng(5)
    ref = [c0[1] + noise(api.bootstrap_weights(n, rng))[1] for _ in range(40)]
    assert np.allclose(r["c_boot"], ref, rtol=0, atol=1e-15)
    assert abs(r["c_sd"] - np.std(ref, ddof=1)) < 1e-15


def test_bias_with_oracle_posterior_mean():
    """Appendix-A toy pair sheared by +-g with the same intrinsic shapes and
    noise, the oracle's posterior mean as the estimator: m is consistent with
    0 within its bootstrap errors, the seed fixes every resample, and a
    resample's weights equal duplicating its galaxies."""
    n, K, g = 300, 30, 0.02
    rng = np.random.default_rng(21)
    e_int = synth.draw_ba14_e(rng, n, sigma=0.2)
    e_p = synth.toy_interim_ellipticities(e_int, (g, 0.0), K, np.random.default_rng(22), n_prop=400)
    e_m = synth.toy_interim_ellipticities(e_int, (-g, 0.0), K, np.random.default_rng(22), n_prop=400)

    def est(e):
        return lambda w: O.shear_estimate(e[0], e[1], family=O.EPRIOR_BA14, alpha=0.2, weights=w)[0][:2]

    r = api.shear_bias(est(e_p), est(e_m), n, g_abs=g, n_boot=30, seed=4)
    assert np.isfinite(r["m_sd"]) and r["m_sd"] > 0 and r["c_sd"] > 0
    assert abs(r["m"]) < 4 * r["m_sd"] + 0.05, r
    r2 = api.shear_bias(est(e_p), est(e_m), n, g_abs=g, n_boot=3, seed=4)
    assert np.array_equal(r2["m_boot"], r["m_boot"][:3])
    w = api.bootstrap_weights(n, np.random.default_rng(4))
    rep = np.repeat(np.arange(n), w.astype(int))
    gw = est(e_p)(w)
    gr = O.shear_estimate(e_p[0][rep], e_p[1][rep], family=O.EPRIOR_BA14, alpha=0.2)[0][:2]
    assert np.allclose(gw, gr, rtol=1e-9, atol=1e-12)
