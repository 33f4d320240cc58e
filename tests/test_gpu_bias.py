"""m and c by shape-noise cancellation (Sec. 3.4) through the C ABI
(bs_shear_bias): on a +-g pair of the Appendix-A toy the library's m and c,
and those of its first bootstrap resamples, equal the ones the oracle's
posterior-mean estimate gives on the same galaxies and counts (|dm| < 1e-4,
and c to the same shear accuracy, 2 |g| 1e-4)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth
from tests.test_bootstrap import _documented_counts

pytestmark = pytest.mark.gpu


def _mc(est_p, est_m, g):
    return (est_p[0] - est_m[0]) / (2 * g) - 1, 0.5 * (est_p[1] + est_m[1])


@pytest.mark.parametrize("family", [O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS])
def test_shear_bias_matches_oracle(cuda, family):
    n, K, g, seed = 3000, 40, 0.02, 11
    rng = np.random.default_rng(41)
    e_int = synth.draw_ba14_e(rng, n, sigma=0.2)
    pair = [synth.toy_interim_ellipticities(e_int, (s * g, 0.0), K, np.random.default_rng(42), n_prop=400)
            for s in (1, -1)]
    if family == O.EPRIOR_TRUNC_GAUSS:
        # every galaxy keeps a sample well inside the truncation radius
        pair = [(0.8 * e1, 0.8 * e2) for (e1, e2) in pair]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    plans = [api.ShearPlan(t(e1), t(e2), family=family) for (e1, e2) in pair]
    r = api.shear_bias_plans(*plans, g_abs=g, n_boot=3, seed=seed, alpha=0.2)

    def oracle_mc(w):
        est = [O.shear_estimate(e1, e2, family=family, alpha=0.2, weights=w)[0] for (e1, e2) in pair]
        return _mc(est[0], est[1], g)

    m0, c0 = oracle_mc(None)
    assert abs(r["m"] - m0) < 1e-4 and abs(r["c"] - c0) < 2 * g * 1e-4, (r["m"], m0, r["c"], c0)
    for k in range(3):
        mk, ck = oracle_mc(_documented_counts(n, seed, k).astype(np.float32))
        assert abs(r["m_boot"][k] - mk) < 1e-4 and abs(r["c_boot"][k] - ck) < 2 * g * 1e-4, (k, r["m_boot"][k], mk)
    assert np.isclose(r["m_sd"], np.std(r["m_boot"], ddof=1), rtol=1e-12)
