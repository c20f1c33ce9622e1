"""GPU: plans created by the layout autotuner (wke_plan_create_autotuned)
give the oracle's Q, use one of the candidate pencil layouts, and honour an
explicit layout request.  Tolerances as in test_gpu_parity: FP64 1e-12, FP32
the derived bound of ``gpu_util.fp32_tolerance``."""
import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests.gpu_util import fp32_tolerance, rel_max_err, require_cuda

pytestmark = pytest.mark.gpu

CASES = [
    # name, d, N, n_r, n_s, n_sig, sphere, input
    ("3d_n16 cube", 3, 16, 2, 8, 8, "cube", lambda: I.gaussian_noise(3, 16, 8.0, 21, 0.1)),
    ("2d_n32 midpoint", 2, 32, 4, 4, 4, "midpoint", lambda: I.two_gaussians(32, 8.0, 22)),
]


def _layout_flags(info):
    return "separable" if info.separable else "shared" if info.shared_fields else "per_group"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_autotuned_plan_matches_oracle(case, prec):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    name, d, N, n_r, n_s, n_sig, sph, gen = case
    L = 8.0
    f_np = gen()
    dt = torch.float64 if prec == "fp64" else torch.float32
    f = torch.tensor(f_np, dtype=dt, device="cuda")
    plan, ms = wke.Plan.autotuned(f, d, N, L, n_r, n_s, n_sig, reps=2, sphere=sph, precision=prec)
    try:
        assert ms > 0.0
        candidates = {"separable", "shared", "per_group"} if d == 3 else {"shared", "per_group"}
        assert plan.layout in candidates
        assert _layout_flags(plan.info()) == plan.layout
        Q = plan.collision(f)
        torch.cuda.synchronize()
        quad = O.make_quadrature(d, n_r, n_s, n_sig, O.default_R(L), sph)
        ref, _ = O.collision_fast(f_np, L, quad)
        tol = 1e-12 if prec == "fp64" else fp32_tolerance(f_np, L, quad)
        assert rel_max_err(Q.double().cpu().numpy(), ref) <= tol, name
    finally:
        plan.close()


@pytest.mark.parametrize("layout", ["shared", "per_group"])
def test_explicit_layout_is_kept(layout):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = torch.tensor(I.gaussian_noise(3, 16, 8.0, 23, 0.1), dtype=torch.float32, device="cuda")
    plan, _ = wke.Plan.autotuned(f, 3, 16, 8.0, 2, 8, 8, reps=1, sphere="cube", precision="fp32", layout=layout)
    try:
        assert plan.layout == layout
        assert _layout_flags(plan.info()) == layout
    finally:
        plan.close()


def test_autotuned_rejects_bad_arguments():
    torch = require_cuda()
    import ctypes
    from paper_2503_12805_gb300 import wke
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = 2, 4, 4
    out = ctypes.c_void_p()
    f = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    # reps < 1 and a NULL f are refused before anything is created
    assert wke.lib().wke_plan_create_autotuned(2, 16, 8.0, 32, ctypes.byref(q), f.data_ptr(), f.data_ptr(), None, 0,
                                               ctypes.byref(out), None, None) == wke.WKE_ERR_INVALID
    assert wke.lib().wke_plan_create_autotuned(2, 16, 8.0, 32, ctypes.byref(q), None, f.data_ptr(), None, 1,
                                               ctypes.byref(out), None, None) == wke.WKE_ERR_INVALID
    assert not out.value
    # an invalid plan (M != n_r n_s n_sig) reports plan creation's code
    assert wke.lib().wke_plan_create_autotuned(2, 16, 8.0, 33, ctypes.byref(q), f.data_ptr(), f.data_ptr(), None, 1,
                                               ctypes.byref(out), None, None) == wke.WKE_ERR_INVALID
    assert not out.value
