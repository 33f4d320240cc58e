"""Ragged batches through the captured launch plan (bs_fit_plan_*): stamps of
25..99 px in all column-slot classes with per-galaxy Moffat PSFs.  The oracle
adapts each galaxy's chains; both sides then run the sampling phase from the
same state with the same random stream, so the chains are coupled."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_22048_gb300 import api, synth
from tests import datagen

pytestmark = pytest.mark.gpu

SIDES = [25, 31, 41, 57, 63, 71, 85, 99]


def _oracle_fit(ds, i, **kw):
    N = ds.stamps[i].shape[0]
    st = ds.stamps[i].astype(np.float32).astype(np.float64)[None]
    return O.fit_galaxies(st, 1.0, ds.psf[i], kw.pop("init")[i:i + 1], ids=[i], random_steps=True, seed=kw.pop("seed"),
                          **kw)


def test_ragged_plan_coupled_to_oracle(cuda):
    truth = synth.draw_ragged(len(SIDES), seed=31)
    truth.side = np.array(SIDES, dtype=np.int32)
    ds = datagen.make_dataset(truth, 2)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    init0 = f32(ds.init)
    with ThreadPoolExecutor(8) as ex:
        warm = list(ex.map(lambda i: _oracle_fit(ds, i, init=init0, seed=5, n_warmup=60, n_samples=1,
                                                 n_leapfrog=16), range(len(SIDES))))
    state = np.stack([np.moveaxis(w["samples"][:, 0, :, 0], 0, -1) for w in warm])     # [n, C, 6]
    step = np.stack([w["step_size"][0] for w in warm])
    im = np.stack([w["inv_mass"][0] for w in warm])
    S = 40
    with ThreadPoolExecutor(8) as ex:
        ref = list(ex.map(lambda i: _oracle_fit(ds, i, init=f32(state), seed=9, n_warmup=0, n_samples=S,
                                                n_leapfrog=16, init_step_size=f32(step[i:i + 1]),
                                                init_inv_mass=f32(im[i:i + 1])), range(len(SIDES))))
    flat, offs, sides = datagen.pack(ds, np.float32)
    t = lambda a, dt=np.float32: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(cuda)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), 3.0, device=cuda)
    cfg = api.FitConfig(n_chains=2, n_warmup=0, n_samples=S, n_leapfrog=16, random_steps=True, seed=9)
    plan = api.RaggedFitPlan(t(flat), t(offs, np.int64), t(sides, np.int32), psf, t(np.ones(len(SIDES))), t(state),
                             cfg, init_step_size=t(step), init_inv_mass=t(im),
                             want=("accepted", "status", "n_grad", "step_size"))
    plan.run()
    plan.run()            # the graph replays: the second launch must give the same chains
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in plan.result().items()}
    assert (res["status"] == 0).all()
    coupled = np.array([[np.array_equal(res["accepted"][i, c], ref[i]["accept"][0, c]) for c in range(2)]
                        for i in range(len(SIDES))])
    assert coupled.mean() >= 0.85, coupled
    worst = 0.0
    for i in range(len(SIDES)):
        for c in range(2):
            if not coupled[i, c]:
                continue
            assert res["n_grad"][i, c] == ref[i]["n_grad"][0, c]
            for k in range(6):
                x, y = res["samples"][k, i, c], ref[i]["samples"][k, 0, c]
                mcse = y.std() / np.sqrt(O.ess(y[None, :]))
                worst = max(worst, abs(x.mean() - y.mean()) / mcse)
    assert worst <= 1e-3, worst


def test_autotuned_plan_matches_untuned(cuda):
    """The autotuner only picks the register budget of each class launch: the
    chains must be bit-identical to the untuned plan's, and every class must
    report a budget and the trial times of all three instances."""
    truth = synth.draw_ragged(64, seed=33)
    truth.side = np.array([SIDES[i % len(SIDES)] for i in range(64)], dtype=np.int32)
    ds = datagen.make_dataset(truth, 2)
    flat, offs, sides = datagen.pack(ds, np.float32)
    t = lambda a, dt=np.float32: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(cuda)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), 3.0, device=cuda)
    cfg = api.FitConfig(n_chains=2, n_warmup=30, n_samples=20, n_leapfrog=8, seed=3)
    args = (t(flat), t(offs, np.int64), t(sides, np.int32), psf, t(np.ones(64)), t(ds.init))
    want = ("accepted", "step_size", "n_grad", "status")
    tuned = api.RaggedFitPlan(*args, cfg, capture=True, autotune=True, want=want)
    plain = api.RaggedFitPlan(*args, cfg, capture=False, autotune=False, want=want)
    tuned.run()
    plain.run()
    torch.cuda.synchronize()
    a, b = tuned.result(), plain.result()
    for k in ("samples", "accepted", "step_size", "n_grad", "status"):
        assert torch.equal(a[k], b[k]), k
    info = tuned.info()
    assert sorted(i["slot_class"] for i in info) == [1, 2, 3, 4]
    for i in info:
        t = {128: i["trial_ms_128"], 96: i["trial_ms_96"], 80: i["trial_ms_80"]}
        assert i["registers"] in (128, 96) and all(v > 0 for v in t.values())
        assert t[i["registers"]] <= min(t[128], t[96])     # the 80-register instance is timed, not chosen
    assert all(i["trial_ms_128"] == 0 and i["registers"] == 128 for i in plain.info())
