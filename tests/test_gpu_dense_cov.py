"""Appendix C with a general pixel covariance (Eq. covar-pixel-likelihood):
Sigma neither stationary nor diagonal.  The precision matrices computed on
the GPU (bs_dense_precision) against numpy's inverse; the log posterior and
its gradient (bs_logpost_points with pixel_prec) against the oracle's
Cholesky solve at 11, 25 and 31 px; a fit whose stored log posteriors match
the oracle at sampled draws.  Tolerances as in the other parity tests: log
posterior 1e-5 relative, gradient 1e-4 of its max-norm."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu

PSF = (O.PSF_MOFFAT, 0.8, 3.0)


def _dataset(sides, seed):
    rng = np.random.default_rng(seed)
    th, covs, stamps = [], [], []
    for N in sides:
        t = np.array([rng.uniform(2.6, 3.2), np.log10(rng.uniform(0.35, 0.6)), rng.uniform(-0.3, 0.3),
                      rng.uniform(-0.3, 0.3), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5)])
        S = synth.dense_covariance(N, rng)
        d = O.render(N, 0.2, PSF, t) + synth.dense_noise(S, rng)
        th.append(t)
        covs.append(S)
        stamps.append(d.astype(np.float32))
    return th, covs, stamps


def _upload(sides, covs, stamps, cuda):
    offs = np.cumsum([0] + [N * N for N in sides[:-1]]).astype(np.int64)
    coffs = np.cumsum([0] + [N ** 4 for N in sides[:-1]]).astype(np.int64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    data = t(np.concatenate([s.ravel() for s in stamps]).astype(np.float32))
    cov = t(np.concatenate([S.ravel() for S in covs]).astype(np.float32))
    side = t(np.array(sides, dtype=np.int32))
    return data, t(offs), side, cov, t(coffs)


def test_dense_precision_is_the_inverse(cuda):
    sides = [11, 25, 9]
    _, covs, stamps = _dataset(sides, 3)
    bad = covs[2].copy()
    bad[0, 0] = -1.0                        # not positive definite
    covs[2] = bad
    data, offs, side, cov, coffs = _upload(sides, covs, stamps, cuda)
    prec, status = api.dense_precision(cov, coffs, side)
    prec = prec.cpu().numpy()
    assert status.cpu().numpy().tolist() == [0, 0, 3]
    c = coffs.cpu().numpy()
    for i, N in enumerate(sides[:2]):
        n = N * N
        P = prec[c[i]:c[i] + n * n].reshape(n, n).astype(np.float64)
        ref = np.linalg.inv(covs[i].astype(np.float32).astype(np.float64))
        assert np.abs(P - ref).max() <= 1e-5 * np.abs(ref).max(), (N, np.abs(P - ref).max() / np.abs(ref).max())
        assert np.array_equal(P, P.T)
    assert not prec[c[2]:].any()


@pytest.mark.parametrize("sides", [[11, 25], [31, 13]])
def test_logpost_dense_matches_oracle(cuda, sides):
    th, covs, stamps = _dataset(sides, 7)
    data, offs, side, cov, coffs = _upload(sides, covs, stamps, cuda)
    prec, status = api.dense_precision(cov, coffs, side)
    assert (status.cpu().numpy() == 0).all()
    rng = np.random.default_rng(1)
    pts, gi = [], []
    for i, t in enumerate(th):
        for _ in range(3):
            q = t.copy()
            q[0] += rng.normal(0, 0.02)
            q[1] += rng.normal(0, 0.03)
            q[2:4] += rng.normal(0, 0.05, 2)
            q[4:6] += rng.normal(0, 0.2, 2)
            pts.append(q)
            gi.append(i)
    pts = np.array(pts, dtype=np.float32)
    psf = api.psf_table("moffat", np.full(len(sides), 0.8, np.float32), 3.0, device=cuda)
    lp, g = api.logpost_points(data, offs, side, psf, torch.ones(len(sides), device=cuda),
                               torch.from_numpy(np.array(gi, np.int32)).to(cuda), torch.from_numpy(pts).to(cuda),
                               pixel_prec=prec, prec_offsets=coffs)
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    for j, q in enumerate(pts.astype(np.float64)):
        i = gi[j]
        N = sides[i]
        v, gv = O.loglike_dense(N, 0.2, PSF, stamps[i].astype(np.float64), covs[i].astype(np.float32)
                                .astype(np.float64), q)
        pv, gp = O.log_prior(q, grad=True)
        ref, gref = v + pv, gv + gp
        assert abs(lp[j] - ref) <= 1e-5 * abs(ref), (N, lp[j], ref)
        assert np.abs(g[j] - gref).max() <= 1e-4 * np.abs(gref).max(), (N, g[j], gref)


def test_fit_dense_matches_oracle_at_sampled_draws(cuda):
    sides = [25, 25, 21]
    th, covs, stamps = _dataset(sides, 11)
    data, offs, side, cov, coffs = _upload(sides, covs, stamps, cuda)
    prec, status = api.dense_precision(cov, coffs, side)
    C = 4
    init = np.repeat(np.array(th, dtype=np.float32)[:, None, :], C, axis=1)
    init[..., 4:6] += np.random.default_rng(2).uniform(-0.1, 0.1, (len(sides), C, 2)).astype(np.float32)
    psf = api.psf_table("moffat", np.full(len(sides), 0.8, np.float32), 3.0, device=cuda)
    cfg = api.FitConfig(n_chains=C, n_warmup=100, n_samples=100, n_leapfrog=8)
    res = api.fit_galaxies(data, offs, side, psf, torch.ones(len(sides), device=cuda),
                           torch.from_numpy(init).to(cuda), cfg, pixel_prec=prec, prec_offsets=coffs,
                           want=("logp", "status", "accept_rate"))
    torch.cuda.synchronize()
    assert (res["status"].cpu().numpy() == 0).all()
    assert res["accept_rate"].cpu().numpy().mean() > 0.5
    samples, logp = res["samples"].cpu().numpy(), res["logp"].cpu().numpy()
    rng = np.random.default_rng(4)
    for _ in range(12):
        i, c, s = rng.integers(len(sides)), rng.integers(C), rng.integers(100)
        q = samples[:, i, c, s].astype(np.float64)
        v, _ = O.loglike_dense(sides[i], 0.2, PSF, stamps[i].astype(np.float64),
                               covs[i].astype(np.float32).astype(np.float64), q)
        ref = v + O.log_prior(q)
        assert abs(logp[i, c, s] - ref) <= 1e-5 * abs(ref), (i, c, s, logp[i, c, s], ref)
