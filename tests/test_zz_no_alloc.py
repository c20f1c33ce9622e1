"""The allocation-free moments entry point (wke_moments_noalloc).

Callers that cannot allocate device memory where they need mass, momentum
and energy (inside another allocator's budget, or while a stream capture is
open) use this call instead of a plan.  Its partial sums live in a fixed
array inside the library, shared by all calls, so two calls in a row must
each give the same answer as the plan-based wke_moments.  This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest

import wke_inputs as I
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_moments_match_plan_moments_twice(prec):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    code = wke.WKE_FP64 if prec == "fp64" else wke.WKE_FP32
    dtype = torch.float64 if prec == "fp64" else torch.float32
    cases = [(3, 32, I.ring(3, 32, 8.0)), (2, 128, I.two_gaussians(128, 8.0, 3))]
    for d, N, g_np in cases:
        g = torch.tensor(g_np, dtype=dtype, device="cuda")
        with wke.Plan(d, N, 8.0, 2, 4 if d == 2 else 8, 4 if d == 2 else 8, precision=prec) as plan:
            ref = plan.moments(g).cpu().numpy()
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):                                   # two calls in a row share the scratch
            out = torch.full((d + 2,), float("nan"), dtype=torch.float64, device="cuda")
            rc = wke.lib().wke_moments_noalloc(d, N, 8.0, code, g.data_ptr(), out.data_ptr(), stream)
            assert rc == wke.WKE_OK, wke.lib().wke_last_error_string()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    g = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    rc = wke.lib().wke_moments_noalloc(3, 256, 8.0, wke.WKE_FP64, g.data_ptr(), out.data_ptr(), None)
    assert rc == wke.WKE_ERR_INVALID
    assert b"4194304" in wke.lib().wke_last_error_string()
