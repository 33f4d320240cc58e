"""bs_shear_loglike_noalloc, the shear likelihood for callers that cannot
allocate device memory (its scratch is a static device array of the
library), called through the C ABI.  It runs the same kernels, grid and
fixed-order finalize as the workspace entry point bs_shear_loglike, so its
results must be bit-identical to it: two calls in a row on one dataset, after
a call on a larger, different dataset has left its own partials in the
static scratch (no slot a call reads may be stale).

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _samples(rng, n, K, cuda):
    e = rng.normal(0, 0.2, (n, K, 2))
    e *= np.minimum(1.0, 0.9 / np.hypot(e[..., 0], e[..., 1]))[..., None]
    return (torch.from_numpy(e[..., 0].astype(np.float32)).to(cuda),
            torch.from_numpy(e[..., 1].astype(np.float32)).to(cuda))


def test_noalloc_matches_workspace_entry_point(cuda):
    from paper_2604_22048_gb300 import _ffi as F
    from paper_2604_22048_gb300 import api
    rng = np.random.default_rng(17)
    n, K = 3000, 120
    plan = api.ShearPlan(*_samples(rng, n, K, cuda))            # workspace entry point
    other = api.ShearPlan(*_samples(rng, 4 * n, K + 8, cuda))   # fills the static scratch first
    out = torch.empty(4, dtype=torch.float64, device=cuda)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    F.check(F.lib().bs_shear_loglike_noalloc(C.byref(other.data), 0.01, 0.0, 0.25, out.data_ptr(), stream))
    first = out.cpu().numpy()
    assert np.isfinite(first).all()
    for (g1, g2, alpha) in [(0.02, -0.01, 0.22), (-0.03, 0.015, 0.18)]:
        want = plan.loglike(g1, g2, alpha, host=True)
        out.fill_(np.nan)
        F.check(F.lib().bs_shear_loglike_noalloc(C.byref(plan.data), g1, g2, alpha, out.data_ptr(), stream))
        got = out.cpu().numpy()
        assert np.array_equal(got, want), (got, want)
