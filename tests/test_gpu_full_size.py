"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times, on outputs the oracle can compute one by one:

- plain batched, 10^4 galaxies of 53 px, one autotuned plan captured as a CUDA
  graph: for sampled galaxies, chains and draws, the log posterior the fit
  stored equals the oracle's at the stored draw;
- ragged, 10^5 galaxies of 25-101 px with per-galaxy Moffat PSFs: the same;
- the shear stage at 10^6 galaxies x 300 samples: the full pass equals the sum
  of passes over shards, a 2,000-galaxy subset selected by 0/1 weights inside
  the full launch matches the oracle, and the several-point pass matches the
  one-point pass.

Inputs are drawn by the seeded generators and rendered by the oracle."""
import os

import numpy as np
import pytest
import torch

import datagen
import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _fit_and_check(cuda, truth, psf, max_side=None, n_check=24, seed=1):
    ds = datagen.make_dataset(truth, 4)
    flat, offs, sides = datagen.pack(ds)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    cfg = api.FitConfig(n_chains=4, n_warmup=100, n_samples=100, n_leapfrog=16, random_steps=True)
    plan = api.RaggedFitPlan(t(flat), t(offs), t(sides), psf, t(ds.sigma.astype(np.float32)),
                             t(ds.init.astype(np.float32)), cfg, capture=True, autotune=True, max_side=max_side)
    plan.run()
    torch.cuda.synchronize()
    assert (plan.status.cpu().numpy() == 0).all()
    samples = plan.samples.cpu().numpy()
    logp = plan.logp.cpu().numpy()
    assert np.isfinite(samples).all() and np.isfinite(logp).all()
    rng = np.random.default_rng(seed)
    worst = 0.0
    for i in rng.choice(truth.n, n_check, replace=False):
        for _ in range(2):
            c, s = rng.integers(4), rng.integers(100)
            th = samples[:, i, c, s].astype(np.float64)
            N = int(sides[i])
            d = flat[offs[i]:offs[i] + N * N].astype(np.float64).reshape(N, N)
            ref, _ = O.logpost(N, 0.2, ds.psf[i], d, 1.0, th)
            rel = abs(logp[i, c, s] - ref) / abs(ref)
            worst = max(worst, rel)
            assert rel <= 1e-5, (i, c, s, logp[i, c, s], ref)
    ess, _ = api.chain_ess(plan.samples)
    assert float(ess.mean(dim=1).mean()) >= 300.0
    return worst


def test_plain_batched_full_size(cuda):
    truth = synth.draw_plain(10000, 53)
    _fit_and_check(cuda, truth, api.psf_table("gaussian", 0.7, device=cuda), max_side=53)


def test_ragged_full_size(cuda):
    truth = synth.draw_ragged(100000)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), truth.psf_beta, device=cuda)
    _fit_and_check(cuda, truth, psf, n_check=32, seed=2)


def test_shear_full_size(cuda):
    n, K = 1_000_000, 300
    rng = np.random.default_rng(13)
    e = rng.normal(0.0, 0.2, (n, 2))
    e1 = (e[:, :1] + rng.normal(0.0, 0.05, (n, K))).astype(np.float32)
    e2 = (e[:, 1:] + rng.normal(0.0, 0.05, (n, K))).astype(np.float32)
    r = np.hypot(e1, e2)
    big = r > 0.9
    e1[big] *= 0.9 / r[big]
    e2[big] *= 0.9 / r[big]
    d1, d2 = torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda)
    point = (0.02, -0.01, 0.22)
    plan = api.ShearPlan(d1, d2)
    full = plan.loglike(*point, host=True)
    # additivity over shards
    parts = sum(api.ShearPlan(d1[a:a + n // 4], d2[a:a + n // 4]).loglike(*point, host=True)
                for a in range(0, n, n // 4))
    assert abs(parts[0] - full[0]) <= 1e-9 * abs(full[0]) and np.allclose(parts[1:], full[1:], rtol=1e-7)
    # a subset through 0/1 weights in the full launch against the oracle
    sub = np.sort(rng.choice(n, 2000, replace=False))
    w = np.zeros(n, np.float32)
    w[sub] = 1.0
    plan.set_weights(w)
    got = plan.loglike(*point, host=True)
    v, g = O.shear_loglike(e1[sub], e2[sub], *point)
    assert abs(got[0] - v) <= 1e-5 * max(abs(v), 2000), (got[0], v)
    assert np.abs(got[1:] - g).max() <= 1e-4 * np.abs(g).max(), (got[1:], g)
    plan.set_weights(None)
    # several points per pass at full size
    pts = np.array([point, (0.0, 0.0, 0.2), (-0.03, 0.02, 0.27)])
    multi = plan.loglike_multi(pts)
    assert abs(multi[0, 0] - full[0]) <= 1e-6 * abs(full[0]) and np.allclose(multi[0, 1:], full[1:], rtol=1e-5)


def _oracle_chunk(args):
    path1, path2, a, b, point = args
    import numpy as np
    import oracle as O
    e1 = np.load(path1, mmap_mode="r")[a:b]
    e2 = np.load(path2, mmap_mode="r")[a:b]
    v, g = O.shear_loglike(np.ascontiguousarray(e1), np.ascontiguousarray(e2), *point,
                           family=O.EPRIOR_TRUNC_GAUSS)
    return v, g


def test_shear_full_size_against_the_oracle(cuda, tmp_path):
    """The whole 10^6 x 300 pass against the oracle's FP64 likelihood over all
    3 x 10^8 samples (a sum over galaxies, so it is evaluated in chunks on a
    spawn pool): the per-galaxy log-sum-exp runs in FP32 on the GPU (totals in
    FP64), and its cost in nats is printed; value within 1e-5 relative,
    gradient 1e-4 of its max-norm."""
    import multiprocessing as mp
    n, K = 1_000_000, 300
    rng = np.random.default_rng(29)
    e = rng.normal(0.0, 0.2, (n, 2))
    e1 = (e[:, :1] + rng.normal(0.0, 0.05, (n, K))).astype(np.float32)
    e2 = (e[:, 1:] + rng.normal(0.0, 0.05, (n, K))).astype(np.float32)
    r = np.hypot(e1, e2)
    small = r.min(axis=1) < 0.6                  # every galaxy keeps a sample inside the truncation
    e1, e2 = np.ascontiguousarray(e1[small]), np.ascontiguousarray(e2[small])
    n = len(e1)
    p1, p2 = str(tmp_path / "e1.npy"), str(tmp_path / "e2.npy")
    np.save(p1, e1)
    np.save(p2, e2)
    plan = api.ShearPlan(torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda), family=O.EPRIOR_TRUNC_GAUSS)
    workers = min(16, os.cpu_count() or 1)
    step = (n + 63) // 64
    with mp.get_context("spawn").Pool(workers) as pool:
        for point in [(0.02, -0.01, 0.22), (-0.03, 0.015, 0.18)]:
            got = plan.loglike(*point, host=True)
            parts = pool.map(_oracle_chunk, [(p1, p2, a, min(n, a + step), point) for a in range(0, n, step)])
            v = sum(x[0] for x in parts)
            g = np.sum([x[1] for x in parts], axis=0)
            print(f"\nshear pass {n} x {K} at {point}: GPU - oracle = {got[0] - v:.4e} nat "
                  f"(relative {(got[0] - v) / abs(v):.2e}); gradient max diff {np.abs(got[1:] - g).max():.3e} "
                  f"of max-norm {np.abs(g).max():.3e}")
            assert abs(got[0] - v) <= 1e-5 * abs(v), (got[0], v)
            assert np.abs(got[1:] - g).max() <= 1e-4 * np.abs(g).max(), (got[1:], g)
