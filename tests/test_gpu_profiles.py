"""Appendix B on the GPU: the fit with a Spergel profile of fixed index nu or a
Gaussian profile as the forward model.  Log posterior and gradient against
the oracle; the Spergel kernel at nu = 1/2 against the exponential one; and the
model bias of fitting exponential galaxies with the wrong profile, measured by
shape-noise cancellation with bootstrap errors (Sec. 3.4)."""
import numpy as np
import pytest
import torch

import datagen
import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _points(ds, rng, per=3):
    pts, gal = [], []
    for i in range(ds.truth.n):
        for _ in range(per):
            pts.append(ds.theta[i] + rng.normal(0, [0.02, 0.02, 0.03, 0.03, 0.05, 0.05]))
            gal.append(i)
    return np.array(pts, np.float32), np.array(gal, np.int32)


@pytest.mark.parametrize("side", [25, 41])
@pytest.mark.parametrize("profile,nu", [(1, -0.6), (1, 1.5), (2, 0.0)])
def test_profile_logpost_matches_oracle(cuda, side, profile, nu):
    truth = synth.draw_plain(4, side, seed=30 + side)
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sides = datagen.pack(ds)
    pts, gal = _points(ds, np.random.default_rng(side + profile))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    lp, g = api.logpost_points(t(flat), t(offs), t(sides), api.psf_table("gaussian", 0.7, device=cuda),
                               t(ds.sigma.astype(np.float32)), t(gal), t(pts), profile=profile, spergel_nu=nu)
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    for q, i in enumerate(gal):
        th = pts[q].astype(np.float64)
        vl, gl = O.loglike_p(profile, nu, side, 0.2, ds.psf[i], ds.stamps[i], 1.0, th)
        vp, gp = O.log_prior(th, grad=True)
        v, gr = vl + vp, gl + gp
        assert abs(lp[q] - v) <= 1e-5 * max(abs(v), side * side), (q, lp[q], v)
        assert np.abs(g[q] - gr).max() <= 1e-4 * np.abs(gr).max() + 1e-3, (q, g[q], gr)


def test_spergel_half_matches_the_exponential_kernel(cuda):
    truth = synth.draw_plain(6, 33, seed=41)
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sides = datagen.pack(ds)
    pts, gal = _points(ds, np.random.default_rng(5))
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    args = (t(flat), t(offs), t(sides), api.psf_table("gaussian", 0.7, device=cuda),
            t(ds.sigma.astype(np.float32)), t(gal), t(pts))
    a, ga = api.logpost_points(*args)
    b, gb = api.logpost_points(*args, profile=1, spergel_nu=0.5)
    a, b, ga, gb = a.cpu().numpy(), b.cpu().numpy(), ga.cpu().numpy(), gb.cpu().numpy()
    assert np.all(np.abs(a - b) <= 1e-5 * np.maximum(np.abs(a), 33 * 33))
    assert np.all(np.abs(ga - gb) <= 1e-4 * np.abs(ga).max(axis=1, keepdims=True) + 1e-3)
