"""Serving (bs_serve_*): a request's result is the same alone, in a mix with
others, under memory-bound admission, and as part of a batched launch
(bs_fit_plan_* over the same galaxies): the fit of a galaxy depends only on
its stamp, PSF, noise, starts and gal_id."""
import numpy as np
import pytest
import torch

from paper_2604_22048_gb300 import _ffi, api, synth
from tests import datagen

pytestmark = pytest.mark.gpu

SIDES = [25, 31, 33, 41, 53, 57, 63, 65, 71, 85, 95, 97, 101, 45, 29, 61]
CFG = api.FitConfig(n_chains=4, n_warmup=40, n_samples=30, n_leapfrog=8, seed=77)
FIELDS = ("samples", "logp", "accepted", "accept_rate", "step_size", "inv_mass", "n_div", "n_grad")


@pytest.fixture(scope="module")
def data():
    truth = synth.draw_ragged(len(SIDES), seed=41)
    truth.side = np.array(SIDES, dtype=np.int32)
    ds = datagen.make_dataset(truth, CFG.n_chains)
    flat, offs, sides = datagen.pack(ds, np.float32)
    init = np.ascontiguousarray(ds.init, dtype=np.float32)
    gal_id = np.arange(1000, 1000 + len(SIDES), dtype=np.uint64)
    return truth, flat, offs, sides, init, gal_id


@pytest.fixture(scope="module")
def batched(cuda, data):
    truth, flat, offs, sides, init, gal_id = data
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).to(cuda)
    psf = api.psf_table("moffat", truth.psf_fwhm.astype(np.float32), 3.0, device=cuda)
    plan = api.RaggedFitPlan(t(flat), t(offs), t(sides), psf, t(np.ones(len(SIDES), np.float32)), t(init), CFG,
                             gal_id=t(gal_id, np.int64), capture=False,
                             want=("logp", "accepted", "accept_rate", "step_size", "inv_mass", "n_div",
                                   "status", "n_grad"))
    plan.run()
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in plan.result().items() if v is not None}
    r["samples"] = np.moveaxis(r["samples"], 1, 0)     # [n, 6, C, S]
    return r


def _requests(data, idx, tags):
    truth, flat, offs, sides, init, gal_id = data
    # the requests point into `flat` and `init`, which the module fixture keeps alive
    return api.Server.requests(flat, offs[idx], sides[idx], "moffat", truth.psf_fwhm[idx], 3.0,
                               np.ones(len(idx), np.float32), init, gal_id[idx], tags=tags, init_index=idx)


def _collect(srv, n, timeout_s=120.0):
    got = {}
    t_end = srv.now_ns() + int(timeout_s * 1e9)
    while len(got) < n:
        assert srv.now_ns() < t_end, f"only {len(got)} of {n} completions"
        for c in srv.poll(timeout_us=20000):
            got[int(c["tag"])] = (c, srv.result(c))
    return got


def _same(res, ref, i):
    assert res["status"] == ref["status"][i] == 0
    for k in FIELDS:
        a = res[k]
        b = ref[k][i]
        assert np.array_equal(a, b), (k, i)


def test_serve_mixed_equals_batched(cuda, data, batched):
    srv = api.Server(CFG, max_side=101, arena_bytes=64 << 20)
    try:
        idx = np.arange(len(SIDES))
        srv.submit(_requests(data, idx, idx))
        got = _collect(srv, len(SIDES))
        for i in idx:
            c, res = got[i]
            assert c["t_arrival_ns"] <= c["t_submit_ns"] <= c["t_admit_ns"] <= c["t_done_ns"]
            assert c["side"] == SIDES[i]
            _same(res, batched, i)
        st = srv.stats()
        assert st["completed"] == len(SIDES) and st["inflight"] == 0 and st["pending"] == 0
    finally:
        srv.close()


def test_serve_alone_equals_batched(cuda, data, batched):
    srv = api.Server(CFG, max_side=101, arena_bytes=16 << 20)
    try:
        for i in (0, 5, 12, 9):      # one request at a time, classes 1..4
            srv.submit(_requests(data, np.array([i]), np.array([i])))
            got = _collect(srv, 1)
            _same(got[i][1], batched, i)
    finally:
        srv.close()


def test_serve_admission_by_memory(cuda, data, batched):
    """A 1 MiB arena holds about twenty 101-px requests: 64 requests (each
    galaxy four times) must queue for memory and still give the same results."""
    srv = api.Server(CFG, max_side=101, arena_bytes=1 << 20)
    try:
        idx = np.tile(np.arange(len(SIDES)), 4)
        tags = np.arange(len(idx))
        srv.submit(_requests(data, idx, tags))
        got = _collect(srv, len(idx))
        for t in tags:
            _same(got[int(t)][1], batched, idx[t])
        st = srv.stats()
        assert st["waits_memory"] > 0
        assert 0 < st["arena_high_water"] <= 1 << 20
        assert st["arena_used"] == 0 or st["inflight"] == 0
    finally:
        srv.close()


def test_serve_rejects_bad_requests(cuda, data):
    srv = api.Server(CFG, max_side=63, arena_bytes=1 << 20)
    try:
        r = _requests(data, np.array([0]), np.array([0]))
        bad = r.copy()
        bad["side"] = 24
        with pytest.raises(_ffi.BsError, match="side"):
            srv.submit(bad)
        big = _requests(data, np.array([12]), np.array([1]))   # 101 px > max_side 63
        with pytest.raises(_ffi.BsError, match="side"):
            srv.submit(big)
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()


def test_serve_stress_bursts_and_teardown(cuda, data):
    """Random bursts of all four slot classes through a 4 MiB arena with at
    most 24 requests on the GPU: every request completes exactly once with a
    clean status, the counters agree and the arena drains; a server destroyed
    with requests still queued and running shuts down cleanly."""
    rng = np.random.default_rng(3)
    cfg = api.FitConfig(n_chains=4, n_warmup=20, n_samples=10, n_leapfrog=4, seed=5)
    truth, flat, offs, sides, init, gal_id = data
    srv = api.Server(cfg, max_side=101, arena_bytes=4 << 20, max_inflight=24, batch_us=100)
    n_total, sent, got = 600, 0, {}
    try:
        while len(got) < n_total:
            if sent < n_total and rng.uniform() < 0.3:
                k = int(min(rng.integers(1, 40), n_total - sent))
                idx = rng.integers(0, len(SIDES), k)
                srv.submit(api.Server.requests(flat, offs[idx], sides[idx], "moffat", truth.psf_fwhm[idx], 3.0,
                                               np.ones(k, np.float32), init, gal_id[idx],
                                               tags=np.arange(sent, sent + k), init_index=idx))
                sent += k
            for c in srv.poll(timeout_us=2000):
                tag = int(c["tag"])
                assert tag not in got
                assert c["status"] == 0
                got[tag] = int(c["side"])
        srv.poll()           # release the last completions
        st = srv.stats()
        assert st["submitted"] == st["admitted"] == st["completed"] == n_total
        assert st["inflight"] == 0 and st["pending"] == 0 and st["arena_used"] == 0
        assert 0 < st["arena_high_water"] <= 4 << 20
    finally:
        srv.close()
    # teardown with work in flight
    srv = api.Server(cfg, max_side=101, arena_bytes=4 << 20)
    idx = np.arange(len(SIDES)).repeat(20)
    srv.submit(api.Server.requests(flat, offs[idx], sides[idx], "moffat", truth.psf_fwhm[idx], 3.0,
                                   np.ones(len(idx), np.float32), init, gal_id[idx], init_index=idx))
    srv.close()
