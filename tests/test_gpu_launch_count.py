"""The library's launch counter (bs_kernel_launches), which the benchmark's
gpu_launches figure reads: one per direct launch, the graph's kernels per
replay of a captured plan, nothing for the kernels recorded at capture."""
import numpy as np
import pytest
import torch

import datagen
from paper_2604_22048_gb300 import api, synth

pytestmark = pytest.mark.gpu


def test_direct_launches(cuda):
    rng = np.random.default_rng(3)
    e = rng.normal(0.0, 0.2, (2, 400, 64)).astype(np.float32)
    plan = api.ShearPlan(torch.from_numpy(e[0]).to(cuda), torch.from_numpy(e[1]).to(cuda))
    n0 = api.kernel_launches()
    plan.loglike(0.01, -0.02, 0.25)
    assert api.kernel_launches() - n0 == 2                     # likelihood pass + finalize
    pts = np.column_stack([np.linspace(-0.04, 0.04, 9), np.zeros(9), np.full(9, 0.22)])
    n0 = api.kernel_launches()
    plan.loglike_multi(pts)
    assert api.kernel_launches() - n0 == 3 + 9                 # 4-point passes + one finalize per point


def test_graph_replay_counts_its_kernels(cuda):
    sides = [25, 41, 67, 97]
    truth = synth.draw_ragged(len(sides), seed=11)
    truth.side = np.asarray(sides, dtype=np.int64)
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sd = datagen.pack(ds)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(cuda)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), truth.psf_beta, device=cuda)
    cfg = api.FitConfig(n_chains=2, n_warmup=10, n_samples=10, n_leapfrog=4)
    args = (t(flat), t(offs), t(sd), psf, t(ds.sigma.astype(np.float32)), t(ds.init.astype(np.float32)), cfg)
    n0 = api.kernel_launches()
    plan = api.RaggedFitPlan(*args, capture=True, autotune=False)
    assert api.kernel_launches() == n0                         # captured, not launched
    n_class = len(plan.info())
    assert n_class == 4
    for k in range(1, 3):
        plan.run()
        assert api.kernel_launches() - n0 == k * n_class
    torch.cuda.synchronize()
    direct = api.RaggedFitPlan(*args, capture=False, autotune=False)
    n1 = api.kernel_launches()
    direct.run()
    assert api.kernel_launches() - n1 == n_class
