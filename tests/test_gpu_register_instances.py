"""The fit kernel's register budgets the autotuner chooses between (128, 96
and 80 registers per thread), and its layouts (all of a galaxy's chains in one
CTA, or half of them per CTA), give the same chains, bit for bit, so its
choice changes speed only."""
import numpy as np
import pytest
import torch

import datagen
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("side", [25, 53, 75, 101])
def test_register_budgets_give_identical_chains(cuda, side):
    truth = synth.draw_plain(12, side, seed=40 + side)
    ds = datagen.make_dataset(truth, 4)
    flat, offs, sides = datagen.pack(ds, np.float32)
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).to(cuda)
    psf = api.psf_table("gaussian", truth.psf_fwhm.astype(np.float32), device=cuda)
    cfg = api.FitConfig(n_chains=4, n_warmup=60, n_samples=40, n_leapfrog=16, seed=5)
    res = {}
    for regs in (128, 96, 80):
        plan = api.FitPlan(t(flat), t(offs), t(sides), psf, torch.ones(12, device=cuda),
                           t(ds.init, np.float32), cfg, registers=regs)
        plan.run()
        torch.cuda.synchronize()
        res[regs] = {k: v.clone() for k, v in plan.result().items() if v is not None}
    for regs in (96, 80):
        for k, v in res[128].items():
            assert torch.equal(v, res[regs][k]), (regs, k)


@pytest.mark.parametrize("side", [25, 53, 101])
def test_chains_per_cta_layouts_give_identical_chains(cuda, side):
    truth = synth.draw_plain(12, side, seed=60 + side)
    ds = datagen.make_dataset(truth, 4)
    flat, offs, sides = datagen.pack(ds, np.float32)
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).to(cuda)
    psf = api.psf_table("gaussian", truth.psf_fwhm.astype(np.float32), device=cuda)
    cfg = api.FitConfig(n_chains=4, n_warmup=60, n_samples=40, n_leapfrog=16, seed=6)
    res = {}
    for cpc, regs in ((0, 128), (2, 128), (1, 96), (2, 80)):
        plan = api.FitPlan(t(flat), t(offs), t(sides), psf, torch.ones(12, device=cuda),
                           t(ds.init, np.float32), cfg, registers=regs, chains_per_cta=cpc)
        plan.run()
        torch.cuda.synchronize()
        res[(cpc, regs)] = {k: v.clone() for k, v in plan.result().items() if v is not None}
    for key in ((2, 128), (1, 96), (2, 80)):
        for k, v in res[(0, 128)].items():
            assert torch.equal(v, res[key][k]), (key, k)
