"""bs_shear_loglike_noalloc, the shear likelihood for callers that cannot
allocate device memory (its scratch is a static device array of the
library), called through the C ABI: two calls in a row, each compared with
the workspace entry point bs_shear_loglike on the same inputs, within the
shear tolerances of the parity tests (value 1e-5 relative, gradient 1e-4).

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point(cuda):
    from paper_2604_22048_gb300 import _ffi as F
    from paper_2604_22048_gb300 import api
    rng = np.random.default_rng(17)
    n, K = 3000, 120
    e = rng.normal(0, 0.2, (n, K, 2))
    e *= np.minimum(1.0, 0.9 / np.hypot(e[..., 0], e[..., 1]))[..., None]
    e1 = torch.from_numpy(e[..., 0].astype(np.float32)).to(cuda)
    e2 = torch.from_numpy(e[..., 1].astype(np.float32)).to(cuda)
    plan = api.ShearPlan(e1, e2)                 # workspace entry point
    out = torch.empty(4, dtype=torch.float64, device=cuda)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (g1, g2, alpha) in [(0.02, -0.01, 0.22), (-0.03, 0.015, 0.18)]:
        want = plan.loglike(g1, g2, alpha, host=True)
        out.fill_(np.nan)
        F.check(F.lib().bs_shear_loglike_noalloc(C.byref(plan.data), g1, g2, alpha, out.data_ptr(), stream))
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= 1e-5 * max(abs(want[0]), n), (got, want)
        assert np.abs(got[1:] - want[1:]).max() <= 1e-4 * np.abs(want[1:]).max(), (got, want)
