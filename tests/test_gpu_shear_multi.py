"""Several (g1, g2, alpha) points per pass over the interim samples
(bs_shear_loglike_multi): against one pass per point, against the oracle,
with galaxy weights, point counts that are not a multiple of the batch, and
the estimate that batches its Hessian and quadrature nodes through it."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api

pytestmark = pytest.mark.gpu


def _samples(rng, n, K, spread):
    e = rng.normal(0.0, spread, (n, K, 2))
    r = np.hypot(e[..., 0], e[..., 1])
    e[r > 0.9] *= (0.9 / r[r > 0.9])[:, None]
    return e[..., 0].astype(np.float32), e[..., 1].astype(np.float32)


@pytest.mark.parametrize("family", [O.EPRIOR_BA14, O.EPRIOR_TRUNC_GAUSS])
@pytest.mark.parametrize("K", [300, 37])
@pytest.mark.parametrize("weighted", [False, True])
def test_multi_matches_single_point_passes(cuda, family, K, weighted):
    rng = np.random.default_rng(K + 3 * family + weighted)
    n = 3000
    e1, e2 = _samples(rng, n, K, 0.12 if family == O.EPRIOR_TRUNC_GAUSS else 0.2)
    w = rng.uniform(0.0, 2.0, n).astype(np.float32) if weighted else None
    plan = api.ShearPlan(torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda), family=family, weights=w)
    pts = np.column_stack([rng.uniform(-0.05, 0.05, 7), rng.uniform(-0.05, 0.05, 7), rng.uniform(0.15, 0.3, 7)])
    multi = plan.loglike_multi(pts)
    dev = plan.loglike_multi(pts, host=False).cpu().numpy()
    assert np.array_equal(multi, dev)
    for i, p in enumerate(pts):
        one = plan.loglike(*p, host=True)
        assert abs(multi[i, 0] - one[0]) <= 1e-6 * max(abs(one[0]), n), (i, multi[i], one)
        assert np.abs(multi[i, 1:] - one[1:]).max() <= 1e-5 * np.abs(one[1:]).max() + 1e-6 * n, (i, multi[i], one)
    v, g = O.shear_loglike(e1, e2, *pts[2], family=family, weights=w)
    assert abs(multi[2, 0] - v) <= 1e-5 * max(abs(v), n) and np.abs(multi[2, 1:] - g).max() <= 1e-4 * np.abs(g).max()


def test_multi_point_counts(cuda):
    rng = np.random.default_rng(5)
    e1, e2 = _samples(rng, 500, 64, 0.2)
    plan = api.ShearPlan(torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda))
    assert plan.loglike_multi(np.zeros((0, 3))).shape == (0, 4)
    pts = np.column_stack([np.linspace(-0.04, 0.04, 9), np.zeros(9), np.full(9, 0.22)])
    a = plan.loglike_multi(pts)
    b = np.concatenate([plan.loglike_multi(pts[i:i + 1]) for i in range(9)])
    assert np.allclose(a, b, rtol=0, atol=0)          # a point's result does not depend on its batch
