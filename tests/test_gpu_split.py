"""Split precision (WKE_SPLIT): the axis-0 transforms as TF32 tensor-core
GEMMs with hi/lo operand splitting.  Against the oracle with the FP32
tolerance of ``gpu_util.tolerance``, and on the benchmark workload (3D N=64,
M=2048) against the FP64 plan within the 1e-6 relative target of the split
variant.
"""
import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests.gpu_util import gpu_collision, rel_max_err, require_cuda, tolerance

pytestmark = pytest.mark.gpu

L = 8.0


@pytest.mark.parametrize("N,n_r,gen", [(32, 3, lambda: I.ring(3, 32, L)),
                                       (64, 2, lambda: I.gaussian_noise(3, 64, L, 71, 0.1))],
                         ids=["3d_n32_ring", "3d_n64_noise"])
def test_split_matches_oracle(N, n_r, gen):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = gen()
    quad = O.make_quadrature(3, n_r, 8, 8, O.default_R(L), "cube")
    ref = O.collision_fast(f, L, quad, return_complex=True)
    with wke.Plan(3, N, L, n_r, 8, 8, sphere="cube", precision="split") as plan:
        info = plan.info()
        assert info.precision == wke.WKE_SPLIT and info.shared_fields == 1
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    scale = np.max(np.abs(ref))
    tol = tolerance("fp32", f, L, quad)
    assert rel_max_err(Q, ref.real, scale) <= tol
    assert rel_max_err(Qim, ref.imag, scale) <= tol


def test_split_within_1e6_of_fp64_on_the_benchmark_workload():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["3d_n64_m2048"]
    f = w.initial()
    out = {}
    for prec in ("fp64", "split"):
        with wke.Plan(3, w.N, w.L, w.n_r, w.n_s, w.n_sig, sphere=w.sphere, precision=prec) as plan:
            out[prec] = gpu_collision(torch, plan, f)
    assert rel_max_err(out["split"], out["fp64"]) <= 1e-6
