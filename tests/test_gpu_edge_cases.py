"""Degenerate and boundary cases of the CUDA path against the oracle or exact
identities: f = 0, constant f, a single quadrature node, caller-supplied
(non-symmetric, unequal-weight) direction rules, exact cubic homogeneity, and
a chunk layout whose last chunk holds a lone group.
"""
import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests.gpu_util import gpu_collision, rel_max_err, require_cuda, tolerance

pytestmark = pytest.mark.gpu

L = 8.0
PRECS = ["fp64", "fp32"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_zero_input_gives_exact_zero(d, N, prec):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = np.zeros((N,) * d)
    with wke.Plan(d, N, L, 3, 4 if d == 2 else 8, 4 if d == 2 else 8, precision=prec) as plan:
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    assert not Q.any() and not Qim.any()


@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_constant_input_gives_zero(d, N):
    """Every shifted field of a constant is that constant, so each node's
    bracket c^2 (2c) - c^2 (2c) vanishes."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = np.full((N,) * d, 0.7)
    n_s = 4 if d == 2 else 8
    with wke.Plan(d, N, L, 3, n_s, n_s, precision="fp64") as plan:
        Q = gpu_collision(torch, plan, f)
    quad = O.make_quadrature(d, 3, n_s, n_s, O.default_R(L), "midpoint" if d == 2 else "cube")
    scale = 0.7 ** 3 * sum(abs(n[3]) for n in quad.nodes())
    assert np.max(np.abs(Q)) <= 1e-14 * scale


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("d,N", [(2, 16), (3, 16)])
def test_single_node(d, N, prec):
    """M = 1: one radial node, one direction and one collision angle, given as
    caller rules (a one-point built-in rule would make sigma = qhat, where
    every bracket vanishes); sigma is not antipodal, so nothing is paired."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.gaussian_noise(d, N, L, 51, 0.2) * I.gaussian(d, N, L, 2.0)
    s_row = np.array([[-1.0, 0.0, 2 * np.pi]]) if d == 2 else np.array([[0.0, 0.0, 1.0, 4 * np.pi]])
    g_row = np.array([[0.6, 0.8, 2 * np.pi]]) if d == 2 else np.array([[0.0, 0.6, 0.8, 4 * np.pi]])
    r, w_r = O.radial_gauss_legendre(1, O.default_R(L))
    quad = O.Quadrature(d, O.default_R(L), r, w_r, s_row[:, :d].copy(), s_row[:, d].copy(),
                        g_row[:, :d].copy(), g_row[:, d].copy())
    ref = O.collision_fast(f, L, quad, return_complex=True)
    with wke.Plan(d, N, L, 1, 1, 1, user_s=s_row, user_sig=g_row, precision=prec) as plan:
        info = plan.info()
        assert info.n_groups == 1 and info.products_per_group == 1
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    tol = tolerance(prec, f, L, quad)
    scale = np.max(np.abs(ref))
    assert rel_max_err(Q, ref.real, scale) <= tol
    assert rel_max_err(Qim, ref.imag, scale) <= tol


def _user_rule(d, n, seed):
    """n seeded directions (not normalised: the library normalises them) with
    unequal positive weights, rows (coords, weight)."""
    u = I.splitmix64_uniform(seed, n * (d + 1))
    rows = np.empty((n, d + 1))
    for i in range(n):
        rows[i, :d] = 2.0 * u[i * (d + 1):i * (d + 1) + d] - 1.0 + (0.3 if d == 2 else 0.1)
        rows[i, d] = 0.5 + u[i * (d + 1) + d]
    return rows


@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_user_direction_rules(d, N):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    us, ug = _user_rule(d, 5, 61), _user_rule(d, 3, 62)
    r, w_r = O.radial_gauss_legendre(2, O.default_R(L))
    norm = lambda rows: rows[:, :d] / np.linalg.norm(rows[:, :d], axis=1, keepdims=True)
    quad = O.Quadrature(d, O.default_R(L), r, w_r, norm(us), us[:, d].copy(), norm(ug), ug[:, d].copy())
    f = I.gaussian_noise(d, N, L, 63, 0.2)
    ref = O.collision_fast(f, L, quad, return_complex=True)
    with wke.Plan(d, N, L, 2, 5, 3, user_s=us, user_sig=ug, precision="fp64") as plan:
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    scale = np.max(np.abs(ref))
    assert rel_max_err(Q, ref.real, scale) <= 1e-12
    assert rel_max_err(Qim, ref.imag, scale) <= 1e-12


@pytest.mark.parametrize("prec", PRECS)
def test_cubic_homogeneity_is_bitwise(prec):
    """Scaling f by 2 scales every rounded operation by a power of two, so
    Q(2 f) = 8 Q(f) bit for bit."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = 0.2 + I.ring(3, 32, L)          # no values near the subnormal range
    with wke.Plan(3, 32, L, 3, 8, 8, precision=prec) as plan:
        a = gpu_collision(torch, plan, f)
        b = gpu_collision(torch, plan, 2.0 * f)
    assert np.array_equal(b, 8.0 * a)


def test_lone_group_in_last_chunk():
    """n_r n_s = 9 groups with two groups per chunk: the last chunk holds a
    single group whose C field has no partner in its packed unit."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    d, N = 2, 64
    f = I.two_gaussians(N, L, 8)
    quad = O.make_quadrature(d, 3, 3, 4, O.default_R(L), "midpoint")
    ref = O.collision_fast(f, L, quad, return_complex=True)
    n_fields = 1 + 4                                # C and one field per sigma (paired)
    per_pair_bytes = (2 * 2 + 1) * N * N * 16       # the library's chunk estimate per two groups
    with wke.Plan(d, N, L, 3, 3, 4, precision="fp64", chunk_bytes=per_pair_bytes) as plan:
        info = plan.info()
        assert info.fields_per_group == n_fields
        assert info.groups_per_chunk == 2 and info.n_chunks == 5
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    scale = np.max(np.abs(ref))
    assert rel_max_err(Q, ref.real, scale) <= 1e-12
    assert rel_max_err(Qim, ref.imag, scale) <= 1e-12


DESCRIBE_CASES = [
    (3, 64, (32, 8, 8), dict(sphere="cube", precision="fp32")),
    (3, 32, (4, 8, 8), dict(sphere="cube", precision="fp64", layout="per_group")),
    (3, 32, (4, 8, 8), dict(sphere="cube", precision="split")),
    (2, 64, (6, 4, 4), dict(sphere="midpoint", precision="fp32", nyquist="zero", dealias=True)),
    (3, 16, (2, 12, 20), dict(sphere="icosahedron", sphere_sig="dodecahedron", precision="fp64")),
]


@pytest.mark.parametrize("d,N,n,kw", DESCRIBE_CASES)
def test_describe_matches_created_plan(d, N, n, kw):
    """wke_plan_describe (host work only) gives the created plan's record; its
    device bytes, the admission estimate, cover what the plan allocated."""
    require_cuda()
    from paper_2503_12805_gb300 import wke
    with wke.Plan(d, N, L, *n, **kw) as plan:
        got = plan.info()
        want = wke.wke_plan_describe(d, N, L, plan.M, plan.quad)
    for name, _ in wke.WkePlanInfo._fields_:
        if name != "device_bytes":
            assert getattr(want, name) == getattr(got, name), name
    assert got.device_bytes <= want.device_bytes <= got.device_bytes + 4096
