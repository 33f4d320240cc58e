"""Differentiation through torch.autograd.Function: the hand-written adjoints of
the shear likelihood and of the render/likelihood, checked against central
finite differences of the same GPU forward and against the oracle gradient."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth
from tests import datagen

pytestmark = pytest.mark.gpu


def test_shear_loglike_autograd_matches_fd_and_oracle(cuda):
    rng = np.random.default_rng(3)
    n, K = 5000, 64
    e = rng.normal(0, 0.2, (n, K, 2))
    e *= np.minimum(1.0, 0.9 / np.hypot(e[..., 0], e[..., 1]))[..., None]
    e1, e2 = e[..., 0].astype(np.float32), e[..., 1].astype(np.float32)
    plan = api.ShearPlan(torch.from_numpy(e1).to(cuda), torch.from_numpy(e2).to(cuda))
    x = torch.tensor([0.015, -0.02, 0.23], dtype=torch.float64, requires_grad=True)
    v = api.ShearLogLike.apply(x, plan)
    v.backward()
    g = x.grad.numpy()
    # central differences of the GPU forward (FP64 totals, step 1e-4)
    fd = np.zeros(3)
    for i in range(3):
        h = 1e-4
        xp = x.detach().numpy().copy()
        xm = xp.copy()
        xp[i] += h
        xm[i] -= h
        fd[i] = (plan.loglike(*xp, host=True)[0] - plan.loglike(*xm, host=True)[0]) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-3 * np.abs(g).max(), (g, fd)
    _, go = O.shear_loglike(e1, e2, 0.015, -0.02, 0.23)
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max(), (g, go)


def test_render_logpost_autograd_matches_fd_and_oracle(cuda):
    truth = synth.draw_plain(4, 53, seed=21)
    ds = datagen.make_dataset(truth, 1)
    flat, offs, sides = datagen.pack(ds, np.float32)
    data = torch.from_numpy(flat).to(cuda)
    offsets = torch.from_numpy(offs).to(cuda)
    side = torch.from_numpy(sides).to(cuda)
    psf = api.psf_table("gaussian", truth.psf_fwhm.astype(np.float32), device=cuda)
    sigma = torch.ones(4, device=cuda)
    gi = torch.arange(4, dtype=torch.int32, device=cuda)
    th0 = ds.theta.astype(np.float32) + np.float32([0.01, 0.02, 0.03, -0.02, 0.2, -0.1])
    th = torch.from_numpy(th0).to(cuda).requires_grad_(True)
    lp = api.RenderLogPost.apply(th, data, offsets, side, psf, sigma, gi)
    lp.sum().backward()
    g = th.grad.cpu().numpy()
    for i in range(4):
        d = flat[offs[i]:offs[i] + 53 * 53].astype(np.float64).reshape(53, 53)
        _, go = O.logpost(53, 0.2, ds.psf[i], d, 1.0, th0[i].astype(np.float64))
        assert np.abs(g[i] - go).max() <= 1e-4 * np.abs(go).max(), (i, g[i], go)
    # central differences of the GPU forward in FP32 parameters: step 1e-3 of
    # each parameter's scale, tolerance set by FP32 rounding of the forward
    for k, h in enumerate([1e-3, 1e-3, 1e-3, 1e-3, 1e-2, 1e-2]):
        tp = th0.copy()
        tm = th0.copy()
        tp[:, k] += h
        tm[:, k] -= h
        lpp, _ = api.logpost_points(data, offsets, side, psf, sigma, gi, torch.from_numpy(tp).to(cuda))
        lpm, _ = api.logpost_points(data, offsets, side, psf, sigma, gi, torch.from_numpy(tm).to(cuda))
        fd = ((lpp - lpm) / (torch.from_numpy(tp[:, k]).double().to(cuda) - torch.from_numpy(tm[:, k]).double().to(cuda))).cpu().numpy()
        assert np.abs(fd - g[:, k]).max() <= 5e-3 * np.abs(g).max() + 0.1, (k, fd, g[:, k])
