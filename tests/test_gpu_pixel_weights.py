"""Spatially variable noise on the GPU (Appendix C): per-pixel weights w in
log L = -1/2 sum w (d - m)^2 / sigma^2, evaluated by rendering the model and
transforming the weighted residual back each evaluation.  Against the
oracle's pixel-space likelihood; against the spectral path when w = 1; masked
pixels leave the fit bit-identical whatever their data."""
import time

import numpy as np
import pytest
import torch

import datagen
import oracle as O
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _case(side, n, seed, mask=True):
    truth = synth.draw_plain(n, side, seed=seed)
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sides = datagen.pack(ds)
    rng = np.random.default_rng(seed + 1)
    w = np.zeros_like(flat)
    for i in range(n):
        wi = rng.uniform(0.3, 2.0, (side, side))
        if mask:
            wi[2:6, side // 2:side // 2 + 7] = 0.0
        w[offs[i]:offs[i] + side * side] = wi.ravel()
    return truth, ds, flat, offs, sides, w


@pytest.mark.parametrize("side", [3, 9, 25, 41, 63])
def test_pixel_weighted_logpost_matches_oracle(cuda, side):
    truth, ds, flat, offs, sides, w = _case(side, 3, 50 + side)
    rng = np.random.default_rng(side)
    pts, gal = [], []
    for i in range(3):
        for _ in range(3):
            pts.append(ds.theta[i] + rng.normal(0, [0.02, 0.02, 0.03, 0.03, 0.05, 0.05]))
            gal.append(i)
    pts, gal = np.array(pts, np.float32), np.array(gal, np.int32)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    lp, g = api.logpost_points(t(flat), t(offs), t(sides), api.psf_table("gaussian", 0.7, device=cuda),
                               t(ds.sigma.astype(np.float32)), t(gal), t(pts), pixel_weight=t(w))
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    for q, i in enumerate(gal):
        wi = w[offs[i]:offs[i] + side * side].reshape(side, side).astype(np.float64)
        v, gr = O.logpost(side, 0.2, ds.psf[i], ds.stamps[i], 1.0, pts[q].astype(np.float64), weights=wi)
        assert abs(lp[q] - v) <= 1e-5 * max(abs(v), side * side), (q, lp[q], v)
        assert np.abs(g[q] - gr).max() <= 1e-4 * np.abs(gr).max() + 1e-3, (q, g[q], gr)


def test_unit_weights_match_the_spectral_path(cuda):
    truth, ds, flat, offs, sides, w = _case(33, 4, 61, mask=False)
    w[:] = 1.0
    rng = np.random.default_rng(2)
    pts = (ds.theta + rng.normal(0, 0.02, ds.theta.shape)).astype(np.float32)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    args = (t(flat), t(offs), t(sides), api.psf_table("gaussian", 0.7, device=cuda),
            t(ds.sigma.astype(np.float32)), t(np.arange(4, dtype=np.int32)), t(pts))
    a, ga = api.logpost_points(*args)
    b, gb = api.logpost_points(*args, pixel_weight=t(w))
    a, b, ga, gb = a.cpu().numpy(), b.cpu().numpy(), ga.cpu().numpy(), gb.cpu().numpy()
    assert np.all(np.abs(a - b) <= 1e-5 * np.maximum(np.abs(a), 33 * 33)), (a, b)
    assert np.all(np.abs(ga - gb) <= 1e-4 * np.abs(ga).max(axis=1, keepdims=True) + 1e-3)


def test_masked_pixels_do_not_enter_the_fit(cuda):
    """Corrupt the data under the mask: weight 0 multiplies the residual to
    exactly zero, so the chains are bit-identical; the fit also reports its
    speed (one launch)."""
    truth, ds, flat, offs, sides, w = _case(41, 32, 71)
    bad = flat.copy()
    for i in range(32):
        st = bad[offs[i]:offs[i] + 41 * 41].reshape(41, 41)
        st[2:6, 20:27] = 1e5
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    cfg = api.FitConfig(n_chains=4, n_warmup=100, n_samples=100, n_leapfrog=16)
    psf = api.psf_table("gaussian", 0.7, device=cuda)
    init = np.repeat(ds.init, 2, axis=1)[:, :4].astype(np.float32)
    res = []
    for data in (flat, bad):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = api.fit_galaxies(t(data), t(offs), t(sides), psf, t(ds.sigma.astype(np.float32)), t(init), cfg,
                             pixel_weight=t(w))
        torch.cuda.synchronize()
        print(f"pixel-weighted fit: 32 galaxies of 41 px, 4 chains x 200: {time.perf_counter() - t0:.3f} s")
        res.append(r)
    assert (res[0]["status"] == 0).all()
    s0, s1 = res[0]["samples"].cpu().numpy(), res[1]["samples"].cpu().numpy()
    assert np.isfinite(s0).all() and np.array_equal(s0, s1)
    # the posterior sits at the truth within a few sd (flux, size)
    for k in (0, 1):
        x = s0[k].reshape(32, -1)
        z = (x.mean(axis=1) - ds.theta[:, k]) / x.std(axis=1)
        assert np.mean(np.abs(z) < 4) > 0.9, (k, z)


def test_pixel_path_chains_do_not_depend_on_the_batch(cuda):
    """One CTA per chain: six chains run (the pixel path has no chain limit), and
    a galaxy's chains are bit-identical whether it is fitted alone (same galaxy
    id, so the same random streams) or among other galaxies of other sides."""
    truth, ds, flat, offs, sides, w = _case(25, 3, 81)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    C = 6
    cfg = api.FitConfig(n_chains=C, n_warmup=40, n_samples=30, n_leapfrog=8)
    psf = api.psf_table("gaussian", 0.7, device=cuda)
    init = np.repeat(ds.init[:, :1], C, axis=1).astype(np.float32)
    init[..., 4:6] += np.random.default_rng(3).uniform(-0.1, 0.1, (3, C, 2)).astype(np.float32)
    sig = ds.sigma.astype(np.float32)
    full = api.fit_galaxies(t(flat), t(offs), t(sides), psf, t(sig), t(init), cfg, pixel_weight=t(w),
                            gal_id=t(np.arange(3, dtype=np.int64)), want=("status", "logp"))
    one = slice(offs[1], offs[1] + 25 * 25)
    alone = api.fit_galaxies(t(flat[one]), t(np.zeros(1, np.int64)), t(sides[1:2]), psf, t(sig[1:2]),
                             t(init[1:2]), cfg, pixel_weight=t(w[one]), gal_id=t(np.array([1], np.int64)),
                             want=("status", "logp"))
    assert (full["status"].cpu().numpy() == 0).all() and (alone["status"].cpu().numpy() == 0).all()
    a = full["samples"].cpu().numpy()[:, 1]
    b = alone["samples"].cpu().numpy()[:, 0]
    assert np.isfinite(a).all() and np.array_equal(a, b)
    assert np.array_equal(full["logp"].cpu().numpy()[1], alone["logp"].cpu().numpy()[0])


@pytest.mark.parametrize("C", [1, 3])
def test_pixel_path_odd_chain_counts(cuda, C):
    """Two chains per CTA: with an odd count the last CTA of a galaxy runs one chain
    while its second group of warps joins each evaluation with a skip flag; the
    lone chain's draws are those it has in a batch of other galaxies."""
    truth, ds, flat, offs, sides, w = _case(25, 2, 91)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    cfg = api.FitConfig(n_chains=C, n_warmup=40, n_samples=30, n_leapfrog=8)
    psf = api.psf_table("gaussian", 0.7, device=cuda)
    init = np.repeat(ds.init[:, :1], C, axis=1).astype(np.float32)
    init[..., 4:6] += np.random.default_rng(5).uniform(-0.1, 0.1, (2, C, 2)).astype(np.float32)
    sig = ds.sigma.astype(np.float32)
    both = api.fit_galaxies(t(flat), t(offs), t(sides), psf, t(sig), t(init), cfg, pixel_weight=t(w),
                            gal_id=t(np.arange(2, dtype=np.int64)), want=("status", "accept_rate"))
    one = slice(offs[1], offs[1] + 25 * 25)
    alone = api.fit_galaxies(t(flat[one]), t(np.zeros(1, np.int64)), t(sides[1:2]), psf, t(sig[1:2]), t(init[1:2]),
                             cfg, pixel_weight=t(w[one]), gal_id=t(np.array([1], np.int64)), want=("status",))
    assert (both["status"].cpu().numpy() == 0).all() and (alone["status"].cpu().numpy() == 0).all()
    s = both["samples"].cpu().numpy()
    assert np.isfinite(s).all() and both["accept_rate"].cpu().numpy().mean() > 0.5
    assert np.array_equal(s[:, 1], alone["samples"].cpu().numpy()[:, 0])


def test_pixel_points_outside_the_support(cuda):
    """A point outside the prior's support is -inf with NaN gradients, and does not
    disturb the points after it in the same launch."""
    truth, ds, flat, offs, sides, w = _case(25, 2, 93, mask=False)
    pts = np.array([ds.theta[0], ds.theta[1], ds.theta[0]], np.float32)
    pts[1, 2] = 1.2                       # |e| > 1
    gal = np.array([0, 1, 0], np.int32)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    lp, g = api.logpost_points(t(flat), t(offs), t(sides), api.psf_table("gaussian", 0.7, device=cuda),
                               t(ds.sigma.astype(np.float32)), t(gal), t(pts), pixel_weight=t(w))
    lp, g = lp.cpu().numpy(), g.cpu().numpy()
    assert lp[1] == -np.inf and np.isnan(g[1]).all()
    assert np.isfinite(lp[[0, 2]]).all() and lp[0] == lp[2] and np.array_equal(g[0], g[2])


def test_pixel_path_mixed_sides_in_one_launch(cuda):
    """Stamps of 25, 41 and 63 px in one launch (the transforms' constants are
    rebuilt for each galaxy's side, the tables sized for the largest): each galaxy's
    chains are those it has when fitted alone with the same launch shape."""
    parts = [_case(s, 1, 100 + s, mask=False) for s in (25, 41, 63)]
    flats, ws, offs, sides, sig, init = [], [], [], [], [], []
    pos = 0
    for truth, ds, flat, off, side, w in parts:
        n = int(side[0]) ** 2
        size = (n + 3) // 4 * 4
        flats.append(np.pad(flat[:n], (0, size - n)))
        ws.append(np.pad(w[:n], (0, size - n)))
        offs.append(pos)
        pos += size
        sides.append(int(side[0]))
        sig.append(ds.sigma[0])
        init.append(np.repeat(ds.init[0:1, :1], 2, axis=1))
    flat, w = np.concatenate(flats), np.concatenate(ws)
    offs, sides = np.array(offs, np.int64), np.array(sides, np.int32)
    sig, init = np.array(sig, np.float32), np.concatenate(init).astype(np.float32)
    init[:, 1, 4:6] += 0.05
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(cuda)
    cfg = api.FitConfig(n_chains=2, n_warmup=40, n_samples=30, n_leapfrog=8)
    psf = api.psf_table("gaussian", 0.7, device=cuda)
    allr = api.fit_galaxies(t(flat), t(offs), t(sides), psf, t(sig), t(init), cfg, pixel_weight=t(w), max_side=63,
                            gal_id=t(np.arange(3, dtype=np.int64)), want=("status",))
    s_all = allr["samples"].cpu().numpy()
    assert (allr["status"].cpu().numpy() == 0).all() and np.isfinite(s_all).all()
    for i in range(3):
        n = int(sides[i]) ** 2
        sl = slice(int(offs[i]), int(offs[i]) + n)
        one = api.fit_galaxies(t(flat[sl]), t(np.zeros(1, np.int64)), t(sides[i:i + 1]), psf, t(sig[i:i + 1]),
                               t(init[i:i + 1]), cfg, pixel_weight=t(w[sl]), max_side=63,
                               gal_id=t(np.array([i], np.int64)), want=("status",))
        assert np.array_equal(s_all[:, i], one["samples"].cpu().numpy()[:, 0]), sides[i]
