"""Shape-noise cancellation m and c with bootstrap errors (Sec. 3.4): the host
logic of the library's bs_shear_bias_custom (through api.shear_bias), with
exact fake estimators and with the oracle's posterior mean as the estimator.
The library runs these estimators on the host; no GPU is needed."""
import numpy as np

import oracle as O
from paper_2604_22048_gb300 import api, synth


def _recording(f, log):
    def g(w):
        log.append(None if w is None else w.copy())
        return f(w)
    return g


def _documented_counts(n, seed, r):
    """Resample r as the header defines it: draw j picks galaxy
    floor(n x / 2^64), x = word (j mod 4) of the Philox4x64-10 block with key
    (seed, r) and counter (floor(j / 4), 0, 1, 0) (the oracle's Philox, pinned
    to numpy's)."""
    c = np.zeros(n)
    for b in range((n + 3) // 4):
        words = O.philox4x64_10([b, 0, 1, 0], [seed, r])
        for k in range(min(4, n - 4 * b)):
            c[(words[k] * n) >> 64] += 1
    return c


def test_resamples_are_the_documented_draws_with_replacement():
    n, seed = 1001, 12
    log = []
    est = _recording(lambda w: (0.0, 0.0), log)
    api.shear_bias(est, lambda w: (0.0, 0.0), n, n_boot=40, seed=seed)
    assert log[0] is None and len(log) == 41
    ws = np.stack(log[1:])
    assert ws.dtype == np.float32 and (ws.sum(axis=1) == n).all() and (ws >= 0).all()
    for r in (0, 1, 39):
        assert np.array_equal(ws[r], _documented_counts(n, seed, r))
    # each count is Binomial(n, 1/n): mean 1, variance 1 - 1/n
    assert abs(ws.var() - (1 - 1 / n)) < 0.05


def test_base_weights_multiply_every_resample():
    n = 50
    base = (np.arange(n) % 3 != 0).astype(np.float32)
    log = []
    api.shear_bias(_recording(lambda w: (0.0, 0.0), log), lambda w: (0.0, 0.0), n, n_boot=5, seed=1,
                   base_weights=base)
    assert np.array_equal(log[0], base)
    for r in range(5):
        assert np.array_equal(log[1 + r], _documented_counts(n, 1, r) * base)


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

    log = []
    plus = _recording(lambda w: (1 + m0) * np.array([g, 0.0]) + c0 + noise(w), log)
    minus = lambda w: (1 + m0) * np.array([-g, 0.0]) + c0 + noise(w)
    r = api.shear_bias(plus, minus, n, g_abs=g, n_boot=40, seed=5)
    assert abs(r["m"] - m0) < 1e-12 and np.allclose(r["m_boot"], m0, atol=1e-12) and r["m_sd"] < 1e-12
    assert abs(r["c"] - (c0[1] + noise(None)[1])) < 1e-15
    ref = [c0[1] + noise(w)[1] for w in log[1:]]
    assert np.allclose(r["c_boot"], ref, rtol=0, atol=1e-15)
    assert abs(r["c_sd"] - np.std(ref, ddof=1)) < 1e-15


def test_estimator_errors_and_bad_arguments_are_reported():
    def bad(w):
        raise FloatingPointError("planted")
    try:
        api.shear_bias(bad, lambda w: (0.0, 0.0), 10, n_boot=2)
        raise AssertionError("the estimator's exception was not raised")
    except FloatingPointError:
        pass
    for kw in (dict(g_abs=0.0), dict(n_boot=-1), dict(base_weights=np.full(10, -1.0))):
        try:
            api.shear_bias(lambda w: (0.0, 0.0), lambda w: (0.0, 0.0), 10, **kw)
            raise AssertionError(kw)
        except RuntimeError as e:
            assert "BS_ERR_INVALID_ARG" in str(e), e
    r = api.shear_bias(lambda w: (0.02, 0.0), lambda w: (-0.02, 0.0), 10, n_boot=1)
    assert r["m"] == 0.0 and np.isnan(r["m_sd"])


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

    log = []
    r = api.shear_bias(_recording(est(e_p), log), est(e_m), n, g_abs=g, n_boot=30, seed=4)
    assert np.isfinite(r["m_sd"]) and r["m_sd"] > 0 and r["c_sd"] > 0
    assert abs(r["m"]) < 4 * r["m_sd"] + 0.05, r
    r2 = api.shear_bias(est(e_p), est(e_m), n, g_abs=g, n_boot=3, seed=4)
    assert np.array_equal(r2["m_boot"], r["m_boot"][:3])
    w = log[1]
    rep = np.repeat(np.arange(n), w.astype(int))
    gw = est(e_p)(w)
    gr = O.shear_estimate(e_p[0][rep], e_p[1][rep], family=O.EPRIOR_BA14, alpha=0.2)[0][:2]
    assert np.allclose(gw, gr, rtol=1e-9, atol=1e-12)
