"""The bounds-checked debug build (libwke_check.so, compiled with -DWKE_CHECK).

Its hot kernels test every index they take from the plan's tables against
the extents of the buffers it addresses and record failing check sites in a
device word instead of accessing memory (nothing traps).  On the small
parity cases below the checked build must give the oracle's result and
record no failure; the 3D N=64 case runs the fused N = 64 kernels.
"""
import os

import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests.gpu_util import gpu_collision, rel_max_err, require_cuda

pytestmark = pytest.mark.gpu

CASES = [
    # d, N, n_r, n_s, n_sig, rule, precision, layout, tolerance
    (2, 16, 8, 4, 1, "midpoint", "fp64", "auto", 1e-12),
    (2, 32, 4, 4, 4, "midpoint", "fp32", "auto", 1e-5),
    (3, 16, 2, 8, 8, "cube", "fp64", "separable", 1e-12),
    (3, 16, 2, 8, 8, "cube", "fp32", "shared", 1e-5),
    (3, 64, 2, 8, 8, "cube", "fp32", "separable", 1e-5),
]


@pytest.fixture(scope="module")
def checked_wke():
    require_cuda()
    from paper_2503_12805_gb300 import wke
    if not os.path.exists(wke.CHECK_LIB_PATH):
        pytest.fail("libwke_check.so is not built (build() compiles it)")
    prev = wke.use_library(wke.CHECK_LIB_PATH)
    try:
        assert b"bounds-checked" in wke.lib().wke_version()
        yield wke
    finally:
        wke.restore_library(prev)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d_n{c[1]}_{c[6]}_{c[7]}" for c in CASES])
def test_checked_build_matches_oracle_without_check_failures(checked_wke, case):
    import torch
    wke = checked_wke
    d, N, n_r, n_s, n_sig, rule, prec, layout, tol = case
    f = I.gaussian_noise(d, N, 8.0, 61, 0.1) if d == 2 else I.ring(3, N, 8.0)
    ref, _ = O.collision_fast(f, 8.0, O.make_quadrature(d, n_r, n_s, n_sig, O.default_R(8.0), rule))
    with wke.Plan(d, N, 8.0, n_r, n_s, n_sig, sphere=rule, precision=prec, layout=layout) as plan:
        Q = gpu_collision(torch, plan, f)
        if prec == "fp32" and d == 3:
            wke.wke_plan_set_tuning(plan.handle, 8, 0, 0)       # the separate axis-0 and product kernels too
            Q2 = gpu_collision(torch, plan, f)
            assert rel_max_err(Q2, ref) <= tol
    assert rel_max_err(Q, ref) <= tol
    assert wke.wke_check_status() == 0
