"""Multi-rank host logic on CPU: two gloo ranks each evaluate the shear
likelihood of their galaxy shard (with the oracle) and sum the (value,
gradient) vector through the same all-reduce hook the GPU path uses; the sum
equals the unsharded value, and the library's shear estimate run on both
ranks with that all-reduce (bs_shear_estimate_custom) equals the one-process
estimate.  Also the size-balanced galaxy partition."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_22048_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, e1, e2, parts, out):
    import torch.distributed as dist
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = parts[rank]
    ar = sharding.make_allreduce()
    for (g1, g2, a) in [(0.02, 0.0, 0.2), (-0.01, 0.03, 0.25)]:
        v, g = O.shear_loglike(e1[idx], e2[idx], g1, g2, a, family=O.EPRIOR_TRUNC_GAUSS)
        tot = ar(np.array([v, *g]))
        out[rank].append(tot.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_shear_loglike_sums_to_unsharded():
    rng = np.random.default_rng(0)
    n, K = 301, 24
    e = rng.normal(0, 0.2, (n, K, 2))
    e *= np.minimum(1.0, 0.9 / np.hypot(e[..., 0], e[..., 1]))[..., None]
    e1, e2 = e[..., 0].astype(np.float32), e[..., 1].astype(np.float32)
    sides = rng.choice([25, 53, 101], size=n)
    parts = sharding.partition_galaxies(sides, 2)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = [mgr.list(), mgr.list()]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, e1, e2, parts, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    import oracle as O
    for j, (g1, g2, a) in enumerate([(0.02, 0.0, 0.2), (-0.01, 0.03, 0.25)]):
        v, g = O.shear_loglike(e1, e2, g1, g2, a, family=O.EPRIOR_TRUNC_GAUSS)
        want = np.array([v, *g])
        for r in range(2):
            got = np.array(out[r][j])
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def _shard_loglike(e1, e2):
    import oracle as O

    def f(x):
        return np.array([[v, *g] for v, g in (O.shear_loglike(e1, e2, p[0], p[1], p[2],
                                                              family=O.EPRIOR_TRUNC_GAUSS) for p in x)])
    return f


def _estimate_worker(rank, world, port, e1, e2, parts, out):
    import torch.distributed as dist
    from paper_2604_22048_gb300 import api
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = parts[rank]
    mean, cov, nev = api.shear_estimate_custom(_shard_loglike(e1[idx], e2[idx]), free_alpha=True, alpha=0.2,
                                               alpha_lo=0.1, alpha_hi=0.4, allreduce=sharding.make_allreduce())
    out[rank].append([*mean.tolist(), *cov.ravel().tolist(), nev])
    dist.barrier()
    dist.destroy_process_group()


def test_library_estimate_over_gloo_ranks_equals_one_process():
    """Every rank runs the library's Newton and quadrature on the likelihood
    all-reduced over the ranks (each summing its shard with the oracle); the
    ranks agree with each other exactly and with the one-process estimate of
    the same library code on all galaxies to rounding (1e-9)."""
    from paper_2604_22048_gb300 import api
    rng = np.random.default_rng(5)
    n, K = 240, 16
    e = rng.normal(0, 0.2, (n, K, 2)) * 0.6
    e1, e2 = e[..., 0].astype(np.float32), e[..., 1].astype(np.float32)
    parts = sharding.partition_galaxies(rng.choice([25, 53, 101], size=n), 2)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = [mgr.list(), mgr.list()]
    port = _free_port()
    procs = [ctx.Process(target=_estimate_worker, args=(r, 2, port, e1, e2, parts, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    r0, r1 = np.array(out[0][0]), np.array(out[1][0])
    assert np.array_equal(r0, r1)
    mean, cov, nev = api.shear_estimate_custom(_shard_loglike(e1, e2), free_alpha=True, alpha=0.2,
                                               alpha_lo=0.1, alpha_hi=0.4)
    assert np.abs(r0[:3] - mean).max() <= 1e-9, (r0[:3], mean)
    assert np.abs(r0[3:12] - cov.ravel()).max() <= 1e-9 * np.abs(cov).max()


def test_partition_is_complete_and_balanced():
    rng = np.random.default_rng(1)
    sides = rng.choice(np.arange(25, 102, 2), size=5000)
    for world in (1, 2, 3, 8):
        parts = sharding.partition_galaxies(sides, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(sides)))
        loads = [sharding.galaxy_cost(sides[p]).sum() for p in parts]
        assert max(loads) - min(loads) <= sharding.galaxy_cost([101])[0]
