"""The shear log-likelihood (Eq. likelihood-shear) is smooth in g and alpha
at the scale where estimates are made, at a size where a rounding error
shared by every sample adds up: at 5 x 10^5 galaxies x 300 samples, values
at theta_j + i delta follow a quadratic in i delta to 3e-3 nat, and its
slope is the analytic gradient (samples kept away from the truncation
radius, where the likelihood itself jumps).  A per-call constant rounded
once (1 - |g|^2, or 1/(2 alpha^2) against per-galaxy constants taken at the
unrounded alpha) shifts every sample's exponent alike and makes the total
jump by about 0.01-0.1 nat between neighbouring points; the kernel's own
remaining wander stays below 1e-3 nat at this size."""
import numpy as np
import pytest
import torch

from paper_2604_22048_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("family", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_loglike_smooth(cuda, family, axis):
    n, K = 500_000, 300
    gen = torch.Generator(device=cuda)
    gen.manual_seed(71 + 2 * family + axis)
    # |eps'| <= 0.5, so that no sample's |eps| reaches the truncated family's
    # radius 0.7 at these g: crossing it is a true jump of the likelihood
    e = torch.randn((2, n, K), generator=gen, device=cuda) * 0.2
    r = torch.hypot(e[0], e[1])
    e = torch.where(r < 0.5, e, e * (0.5 / r))
    plan = api.ShearPlan(e[0].contiguous(), e[1].contiguous(), family=family, trunc_r=0.7)
    th0 = np.array([0.013, -0.007, 0.22])
    delta = 5e-6 if axis < 2 else 1e-6
    steps = np.arange(-3, 4)
    vals, grads = [], []
    for i in steps:
        th = th0.copy()
        th[axis] += i * delta
        out = plan.loglike(th[0], th[1], th[2], host=True)
        vals.append(out[0])
        grads.append(out[1 + axis])
    v = np.array(vals) - vals[3]
    x = steps * delta
    coef = np.polyfit(x, v, 2)
    resid = v - np.polyval(coef, x)
    assert np.abs(resid).max() < 3e-3, (resid, coef)
    # the slope of the fit carries the values' noise over the span of the steps
    assert abs(coef[1] - grads[3]) <= 1e-3 * abs(grads[3]) + 3e-4 / delta, (coef, grads[3])
