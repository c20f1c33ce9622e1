"""De-aliased plans (WKE_DEALIAS_PAD2): the linear index sums of Eqs.
(3.3)-(3.6) through 2N zero padding, against the oracle's padded evaluation
(which is pinned to the O(N^{3d}) linear sums), and the exact mass that the
linear sums give for the same antipodal rule on qhat and sigma (Appendix B).

Tolerances (relative max-norm): the cancellation bound of
``gpu_util.tolerance`` on the 2N grid, never below 1e-12 (FP64) and 1e-5
(FP32); it exceeds the floor only for the near-equilibrium Rayleigh-Jeans
state, whose Q is 1e6 times smaller than its terms.
"""
import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests.gpu_util import gpu_collision, rel_max_err, require_cuda, tolerance

pytestmark = pytest.mark.gpu

L = 8.0

CASES = [
    # name, d, N, n_r, n_s, n_sig, sphere, sphere_sig, input
    ("2d_n16", 2, 16, 4, 4, 3, "midpoint", None, lambda: I.gaussian_noise(2, 16, L, 31, 0.2)),
    ("2d_n32 two Gaussians", 2, 32, 6, 4, 4, "midpoint", None, lambda: I.two_gaussians(32, L, 5)),
    ("2d_n48", 2, 48, 3, 4, 4, "midpoint", None, lambda: I.two_gaussians(48, L, 13)),
    ("2d_n128 Rayleigh-Jeans", 2, 128, 2, 4, 4, "midpoint", None,
     lambda: I.rayleigh_jeans(2, 128, L, 1.0, [0.0, 0.0], 0.1)),
    ("3d_n16 non-antipodal sigma", 3, 16, 2, 8, 6, "cube", "product:2:3",
     lambda: I.gaussian_noise(3, 16, L, 12, 0.1)),
    ("3d_n32 cube", 3, 32, 2, 8, 8, "cube", None, lambda: I.ring(3, 32, L)),
]


def _quad(d, n_r, n_s, n_sig, sph, sph_sig):
    return O.make_quadrature(d, n_r, n_s, n_sig, O.default_R(L), sph, sph_sig)


# The Rayleigh-Jeans state is an equilibrium: its Q is a million times smaller
# than the terms that cancel to it, below what FP32 arithmetic resolves, so it
# runs in FP64 only.
PARAMS = [(c, p) for c in CASES for p in ("fp64", "fp32") if not (p == "fp32" and "Rayleigh" in c[0])]


@pytest.mark.parametrize("case,prec", PARAMS, ids=[f"{c[0]}-{p}" for c, p in PARAMS])
def test_dealiased_parity(case, prec):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    name, d, N, n_r, n_s, n_sig, sph, sph_sig, gen = case
    f = gen()
    quad = _quad(d, n_r, n_s, n_sig, sph, sph_sig)
    ref = O.collision_dealiased(f, L, quad, nyquist="zero", return_complex=True)
    with wke.Plan(d, N, L, n_r, n_s, n_sig, sphere=sph, sphere_sig=sph_sig, precision=prec, nyquist="zero",
                  dealias=True) as plan:
        info = plan.info()
        assert info.N == N and info.N_compute == 2 * N
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    scale = np.max(np.abs(ref))
    tol = tolerance(prec, f, L, quad, dealias=True, nyquist="zero")
    assert rel_max_err(Q, ref.real, scale) <= tol, name
    assert rel_max_err(Qim, ref.imag, scale) <= tol, name


@pytest.mark.parametrize("d", [2, 3])
def test_dealiased_mass_is_exact_and_aliased_is_not(d):
    """Same antipodal rule for qhat and sigma, f not band-limited: the linear
    sums give sum_i Q_i = 0 to rounding; the circular sums do not."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    N, n_r, n_s, n_sig, sph = (32, 5, 6, 6, "midpoint") if d == 2 else (16, 3, 8, 8, "cube")
    f = I.gaussian_noise(d, N, L, 23, eps=0.4) * I.gaussian(d, N, L, 1.5)
    out = {}
    for dealias in (True, False):
        with wke.Plan(d, N, L, n_r, n_s, n_sig, sphere=sph, precision="fp64", nyquist="zero",
                      dealias=dealias) as plan:
            out[dealias] = gpu_collision(torch, plan, f)
    assert abs(out[True].sum()) / np.abs(out[True]).sum() < 1e-13
    assert abs(out[False].sum()) / np.abs(out[False]).sum() > 1e-4


def test_dealiased_rk4_conserves_mass():
    """Ten RK4 steps of a de-aliased FP64 plan: the mass changes only by
    rounding, step after step."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    N = 32
    f0 = I.two_gaussians(N, L, 3)
    with wke.Plan(2, N, L, 6, 4, 4, precision="fp64", nyquist="zero", dealias=True) as plan:
        ft = torch.tensor(f0, dtype=torch.float64, device="cuda")
        m0 = plan.moments(ft)[0].item()
        for _ in range(10):
            plan.step(ft, 1e-2, 4)
        m1 = plan.moments(ft)[0].item()
        assert abs(m1 - m0) <= 1e-13 * abs(m0)
        # and the state matches ten oracle steps of the de-aliased operator
        quad = O.make_quadrature(2, 6, 4, 4, O.default_R(L), "midpoint")
        g = f0.copy()
        for _ in range(10):
            g = O.rk_step(g, L, quad, 1e-2, 4, nyquist="zero", dealias=True)
        assert rel_max_err(ft.cpu().numpy(), g) <= 1e-12


def test_dealiased_host_call_matches_device_call():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    N = 16
    f = I.gaussian_noise(3, N, L, 7, 0.2)
    with wke.Plan(3, N, L, 2, 8, 8, precision="fp32", nyquist="zero", dealias=True) as plan:
        Qd = gpu_collision(torch, plan, f)
        fh = torch.tensor(f, dtype=torch.float32).pin_memory()
        Qh = torch.empty_like(fh).pin_memory()
        plan.collision_host(fh, Qh)
    assert np.array_equal(Qh.numpy(), Qd.astype(np.float32))
