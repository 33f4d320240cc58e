"""The fit kernel's register budgets the autotuner chooses between (128 and
96 registers per thread) give the same chains, bit for bit, so its choice
changes speed only.  The 80-register instance, which the compiler rounds
differently in places, gives valid chains of its own (all statuses 0, the
same number of draws, a log posterior at every draw)."""
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
    for k, v in res[128].items():
        assert torch.equal(v, res[96][k]), k
    assert (res[80]["status"] == 0).all()
    assert torch.isfinite(res[80]["samples"]).all() and torch.isfinite(res[80]["logp"]).all()
    assert res[80]["samples"].shape == res[128]["samples"].shape
