"""Edge cases of the fit path: an empty batch, the smallest and the largest
stamp sides (3 and 127 px, the most shared memory a launch stages), and one
plan spanning all four column-slot classes with both extremes in it."""
import numpy as np
import pytest
import torch

import datagen
import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _truth(sides, seed):
    t = synth.draw_ragged(len(sides), seed=seed)
    t.side = np.asarray(sides, dtype=np.int64)
    return t


def test_empty_batch(cuda):
    cfg = api.FitConfig(n_chains=2, n_warmup=10, n_samples=10, n_leapfrog=4)
    z = lambda *s, dt=torch.float32: torch.zeros(s, dtype=dt, device=cuda)
    res = api.fit_galaxies(z(0), z(0, dt=torch.int64), z(0, dt=torch.int32), api.psf_table("gaussian", 0.7,
                           device=cuda), z(0), z(0, 2, 6), cfg, max_side=25)
    assert res["samples"].shape == (6, 0, 2, 10)
    lp, g = api.logpost_points(z(25 * 25), z(1, dt=torch.int64), torch.full((1,), 25, dtype=torch.int32,
                               device=cuda), api.psf_table("gaussian", 0.7, device=cuda), torch.ones(1, device=cuda),
                               z(0, dt=torch.int32), z(0, 6))
    assert lp.shape == (0,) and g.shape == (0, 6)


@pytest.mark.parametrize("sides", [[3, 5, 7], [125, 127]])
def test_extreme_sides_logpost(cuda, sides):
    truth = _truth(sides, seed=90 + sides[0])
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sd = datagen.pack(ds)
    rng = np.random.default_rng(sides[0])
    pts = (ds.theta + rng.normal(0, [0.02, 0.02, 0.03, 0.03, 0.05, 0.05], ds.theta.shape)).astype(np.float32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), truth.psf_beta, device=cuda)
    lp, g = api.logpost_points(t(flat), t(offs), t(sd), psf, t(ds.sigma.astype(np.float32)),
                               t(np.arange(len(sides), dtype=np.int32)), t(pts))
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    for i, N in enumerate(sides):
        d = flat[offs[i]:offs[i] + N * N].astype(np.float64).reshape(N, N)
        ref, gref = O.logpost(N, 0.2, ds.psf[i], d, 1.0, pts[i].astype(np.float64))
        assert abs(lp[i] - ref) <= 1e-5 * abs(ref), (N, lp[i], ref)
        assert np.abs(g[i] - gref).max() <= 1e-4 * np.abs(gref).max() + 1e-3, (N, g[i], gref)


def test_plan_over_all_slot_classes(cuda):
    sides = [3, 31, 33, 63, 65, 95, 97, 127, 27, 127, 3, 45]
    truth = _truth(sides, seed=7)
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sd = datagen.pack(ds)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), truth.psf_beta, device=cuda)
    cfg = api.FitConfig(n_chains=2, n_warmup=60, n_samples=40, n_leapfrog=8)
    plan = api.RaggedFitPlan(t(flat), t(offs), t(sd), psf, t(ds.sigma.astype(np.float32)),
                             t(ds.init.astype(np.float32)), cfg, capture=True, autotune=False)
    assert sorted(i["slot_class"] for i in plan.info()) == [1, 2, 3, 4]
    plan.run()
    torch.cuda.synchronize()
    assert (plan.status.cpu().numpy() == 0).all()
    samples, logp = plan.samples.cpu().numpy(), plan.logp.cpu().numpy()
    for i, N in enumerate(sides):
        th = samples[:, i, 1, 39].astype(np.float64)
        d = flat[offs[i]:offs[i] + N * N].astype(np.float64).reshape(N, N)
        ref, _ = O.logpost(N, 0.2, ds.psf[i], d, 1.0, th)
        assert abs(logp[i, 1, 39] - ref) <= 1e-5 * abs(ref), (N, logp[i, 1, 39], ref)
