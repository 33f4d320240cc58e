"""Posterior calibration on toy ellipticities (Appendix A): the whole shear
inference repeated on independent datasets, each with its true shear drawn
from the unit-disk prior; the true shear must fall inside the central q'
interval of the shear posterior in about a fraction q' of the runs."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu

N_RUNS, N_GAL, K = 100, 500, 100
LEVELS = (0.2, 0.4, 0.6, 0.8, 0.9)


def test_shear_posterior_coverage(cuda):
    rng = np.random.default_rng(674)
    inside = {q: [] for q in LEVELS}
    for run in range(N_RUNS):
        # true shear uniform on the unit disk (kept a little inside the edge)
        r, ph = 0.95 * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
        g = (r * np.cos(ph), r * np.sin(ph))
        e_int = synth.draw_ba14_e(rng, N_GAL, sigma=0.2)
        e1, e2 = synth.toy_interim_ellipticities(e_int, g, K, rng, n_prop=1000)
        plan = api.ShearPlan(torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda), family=O.EPRIOR_BA14)
        g0 = np.array([e1.mean(), e2.mean()])
        g0 *= min(1.0, 0.9 / max(np.hypot(*g0), 1e-12))
        draws, info = plan.sample([g0[0], g0[1], 0.2, 2.45, 0.4, 14.0, -0.4, 0.05], free=("g1", "g2"),
                                  n_warmup=200, n_samples=600, n_leapfrog=8, seed=1000 + run)
        assert info["accept_rate"] > 0.3, (run, info)
        for q in LEVELS:
            for k in range(2):
                lo, hi = np.quantile(draws[:, k], [(1 - q) / 2, (1 + q) / 2])
                inside[q].append(lo <= g[k] <= hi)
    for q in LEVELS:
        realised = float(np.mean(inside[q]))
        assert abs(realised - q) <= 0.12, (q, realised)
