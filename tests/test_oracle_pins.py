"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: a different
parametrisation of Eq. (2.3), closed-form integrals, exact identities of the
resonance manifold, or the same quantity by a different algorithm.
"""
import math

import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests import pins

L = 8.0


# ------------------------------------------------------------ components

@pytest.mark.parametrize("d", [2, 3])
def test_fft_matches_eq31_term_by_term(d):
    assert pins.naive_dft(O, d) < 1e-13


@pytest.mark.parametrize("n_r", [1, 3, 8])
def test_gauss_legendre_radial_exact_to_degree(n_r):
    R = 7.25
    r, w = O.radial_gauss_legendre(n_r, R)
    for k in range(2 * n_r):
        assert abs(np.sum(w * r ** k) - R ** (k + 1) / (k + 1)) <= 1e-13 * R ** (k + 1)


@pytest.mark.parametrize("n", [2, 4, 6, 12])
def test_circle_midpoint_exact_below_n(n):
    dirs, w = O.circle_midpoint(n)
    th = np.arctan2(dirs[:, 1], dirs[:, 0])
    assert abs(np.sum(w) - 2 * math.pi) < 1e-13
    for m in range(1, n):
        assert abs(np.sum(w * np.cos(m * th))) < 1e-12
        assert abs(np.sum(w * np.sin(m * th))) < 1e-12


def _sphere_monomial(a, b, c):
    """Exact int_{S^2} x^a y^b z^c."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


@pytest.mark.parametrize("kind,n,t", [("octahedron", 6, 3), ("cube", 8, 3), ("icosahedron", 12, 5),
                                      ("dodecahedron", 20, 5), ("product:3:6", 18, 5)])
def test_sphere_designs_exact_to_strength(kind, n, t):
    pts, w = O.sphere_rule(3, n, kind)
    assert np.allclose(np.linalg.norm(pts, axis=1), 1.0, atol=1e-15)
    for a in range(t + 1):
        for b in range(t + 1 - a):
            for c in range(t + 1 - a - b):
                got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(got - _sphere_monomial(a, b, c)) < 1e-12, (a, b, c)


@pytest.mark.parametrize("d", [2, 3])
def test_total_node_weight_closed_form(d):
    assert pins.weight_total(O, d) < 1e-13


# ------------------------------------------------------------ the operator

@pytest.mark.parametrize("d", [2, 3])
def test_spherical_form_matches_bruteforce_eq23(d):
    """Eq. (2.7) as the oracle evaluates it equals the resonant-manifold
    integral of Eq. (2.3) computed by an independent route: this fixes the
    2^{1-d} prefactor, |q|^{d-2}, the r^{2d-3} radial weight, the four signs
    and the post-collision points k', k2'."""
    assert pins.operator_vs_bruteforce(O, d) < 1e-10


@pytest.mark.parametrize("d", [2, 3])
def test_rayleigh_jeans_integrand_vanishes(d):
    """Eq. (2.6): K(f_eq) = 0.  Momentum and energy are conserved by every
    node (a + b = q and |a|^2 + |b|^2 = |q|^2), so the real-space form is zero
    to rounding for any quadrature."""
    assert pins.rj_zero(O, d) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_fast_equals_realspace_on_bandlimited_f(d):
    assert pins.fast_vs_realspace(O, d) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_algorithm1_equals_grid_accumulation(d):
    assert pins.alg1_vs_fast(O, d) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_fast_equals_direct_circular_sums(d):
    assert pins.fast_vs_direct(O, d) < 1e-12


@pytest.mark.slow
def test_fast_equals_direct_on_2d_n16_m32_workload():
    """The 2D N=16, M=32 workload: fast form against the O(N^6) sums, and the
    Rayleigh-Jeans check state 1/(1 + 0.1|k|^2)."""
    w = I.WORKLOADS["2d_n16_m32"]
    quad = O.make_quadrature(2, w.n_r, w.n_s, w.n_sig, O.default_R(w.L), "midpoint")
    for f in (w.initial(), I.rayleigh_jeans(2, w.N, w.L, 1.0, [0.0, 0.0], 0.1)):
        assert pins.fast_vs_direct(O, 2, w.N, quad, f) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_mass_identity_bandlimited(d):
    """Appendix B: with the same rule for qhat and sigma the terms pair up
    (K1 <-> K2 and K3 <-> K4 under qhat <-> sigma), so the grid sum of Q
    vanishes when the cubic products do not alias (|j_c| <= N/3 - 1)."""
    assert pins.mass_bandlimited(O, d) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("nyquist", ["keep", "zero"])
def test_dealiased_equals_linear_sums(d, nyquist):
    """2N padding gives the linear index sums of Eqs. (3.3)-(3.6) exactly."""
    assert pins.dealiased_vs_linear(O, d, nyquist) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_dealiased_mass_for_any_band(d):
    """Appendix B for the linear sums with quadrature weights: the mass of Q
    vanishes for f that is not band-limited (the circular sums do not)."""
    assert pins.dealiased_mass(O, d) < 1e-13
    N, quad = (16, O.make_quadrature(2, 5, 6, 6, O.default_R(L), "midpoint")) if d == 2 else \
        (8, O.make_quadrature(3, 3, 8, 8, O.default_R(L), "cube"))
    f = I.gaussian_noise(d, N, L, 23, eps=0.4) * I.gaussian(d, N, L, 1.5)
    qc = O.collision_fast(f, L, quad, return_complex=True)
    assert abs(np.sum(qc)) / np.sum(np.abs(qc)) > 1e-3       # the check can tell the two apart


@pytest.mark.parametrize("d", [2, 3])
def test_dealiased_equals_aliased_for_narrow_band(d):
    assert pins.dealiased_vs_aliased_bandlimited(O, d) < 1e-12


def test_mass_appendix_b_linear_exact_weights():
    """Appendix B: the non-fast system (linear sums, exact weights) has
    hat K_0 = 0 for any f."""
    N = 8
    quad = O.make_quadrature(2, 4, 4, 4, O.default_R(L), "midpoint")
    f = I.gaussian_noise(2, N, L, 23, eps=0.4) * I.gaussian(2, N, L, 1.5)
    Kh = O.collision_direct(f, L, quad, wrap=False, weights="exact", return_hat=True)
    assert abs(Kh[0, 0]) < 1e-13 * np.max(np.abs(Kh))


def test_exact_weight_radial_integral_closed_forms():
    """psi_exact against the closed forms: 2D Lommel integral
    int_0^R r J0(ar) J0(br) dr = R [a J1(aR) J0(bR) - b J0(aR) J1(bR)]/(a^2-b^2),
    and the 3D elementary integral 16 pi^2/(ab) int_0^R r sin(ar) sin(br) dr."""
    from scipy.special import j0, j1
    R = 7.0
    a = np.array([0.3, 1.7, 4.1, 9.0])
    b = np.array([1.1, 0.2, 2.5, 8.3])
    lommel = R * (a * j1(a * R) * j0(b * R) - b * j0(a * R) * j1(b * R)) / (a * a - b * b)
    assert np.allclose(O.psi_exact(2, R, a, b), 4 * math.pi ** 2 * lommel, rtol=1e-12, atol=1e-12)

    def I_cos(c):
        return R * np.sin(c * R) / c + (np.cos(c * R) - 1.0) / (c * c)
    three = 16 * math.pi ** 2 / (a * b) * 0.5 * (I_cos(a - b) - I_cos(a + b))
    assert np.allclose(O.psi_exact(3, R, a, b), three, rtol=1e-11, atol=1e-11)


def test_quadrature_weights_converge_to_exact():
    """The separated quadrature of Eq. (3.8) converges to the exact weights
    as N_r, N_s = N_sig grow (Sec. 3.4 remark)."""
    N = 8
    f = I.gaussian(2, N, L, 1.5)
    ref = O.collision_direct(f, L, O.make_quadrature(2, 4, 4, 4, O.default_R(L)), wrap=False,
                             weights="exact", return_hat=True)
    errs = []
    for n_r, n_s in [(4, 4), (8, 8), (16, 16), (32, 32), (48, 64)]:
        quad = O.make_quadrature(2, n_r, n_s, n_s, O.default_R(L), "midpoint")
        Kh = O.collision_direct(f, L, quad, wrap=False, return_hat=True)
        errs.append(float(np.max(np.abs(Kh - ref)) / np.max(np.abs(ref))))
    assert errs[-1] < 1e-12
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs


# ------------------------------------------------------------ invariants

def test_cubic_homogeneity_and_grid_shift():
    N = 16
    quad = O.make_quadrature(2, 5, 4, 4, O.default_R(L), "midpoint")
    f = I.two_gaussians(N, L, 7)
    q, _ = O.collision_fast(f, L, quad)
    q3, _ = O.collision_fast(1.7 * f, L, quad)
    assert np.max(np.abs(q3 - 1.7 ** 3 * q)) < 1e-13 * np.max(np.abs(q3))
    qs, _ = O.collision_fast(np.roll(f, (3, -5), axis=(0, 1)), L, quad)
    assert np.max(np.abs(qs - np.roll(q, (3, -5), axis=(0, 1)))) < 1e-13 * np.max(np.abs(q))


def test_coordinate_symmetry_3d_cube():
    """The cube rule is invariant under coordinate permutations and
    reflections, so Q inherits the symmetry of f."""
    N = 8
    quad = O.make_quadrature(3, 3, 8, 8, O.default_R(L), "cube")
    f = I.gaussian(3, N, L, 1.2)
    f = f + np.transpose(f, (1, 0, 2))     # symmetric under k1 <-> k2
    q, _ = O.collision_fast(f, L, quad)
    assert np.max(np.abs(q - np.transpose(q, (1, 0, 2)))) < 1e-13 * np.max(np.abs(q))


def test_spectral_convergence_on_gaussian():
    """Q on a resolved Gaussian converges spectrally in N at common points."""
    quad = O.make_quadrature(2, 6, 4, 4, O.default_R(L), "midpoint")
    Q = {}
    for N in (16, 32, 64):
        Q[N], _ = O.collision_fast(I.gaussian(2, N, L), L, quad)
    e1 = np.max(np.abs(Q[16] - Q[32][::2, ::2]))
    e2 = np.max(np.abs(Q[32] - Q[64][::2, ::2]))
    assert e2 < 1e-8 * np.max(np.abs(Q[64]))
    assert e2 < 1e-3 * e1


def test_momentum_and_energy_nearly_conserved():
    """Momentum and energy are exact per collision; on the grid the error comes
    from interpolation, wrap and truncation, small for a localised f."""
    N = 32
    quad = O.make_quadrature(2, 12, 8, 8, O.default_R(L), "midpoint")
    f = I.two_gaussians(N, L, 4, width=0.9, centre=1.0)
    q, _ = O.collision_fast(f, L, quad)
    h = 2 * L / N
    k = O.grid_points(2, N, L)
    m = O.moments(q, L)
    scale_p = h * h * np.sum(np.abs(q) * np.linalg.norm(k, axis=-1))
    scale_e = h * h * np.sum(np.abs(q) * np.sum(k * k, axis=-1))
    assert np.max(np.abs(m[1:3])) < 1e-6 * scale_p
    assert abs(m[3]) < 1e-6 * scale_e


def _paper_table(name):
    import os
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_rj_residuals.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t, d, N, ns, linf, l2 = line.split()
        if t == name:
            rows.append((int(N), int(ns), float(linf)))
    return rows


@pytest.mark.slow
def test_rj_residual_trend_matches_paper_table():
    """Sec. 4.1.1, Example 1 (Table "table-2D-Keq"): the Rayleigh-Jeans residual
    of the fast method decreases with N.  The paper does not state L, so only
    the trend and the order of magnitude at the finest common N are pinned
    (L = (3 + sqrt 2) S / 2 here)."""
    S = 5.0
    Lp = (3.0 + math.sqrt(2.0)) / 2.0 * S
    rows = _paper_table("2D-Keq")
    ours = {}
    for N, ns, _ in rows:
        if N > 64:
            continue
        quad = O.make_quadrature(2, N, ns, ns, 2 * S, "midpoint")
        q, _ = O.collision_fast(I.rayleigh_jeans(2, N, Lp, 50.0, [5.0, 5.0], 100.0), Lp, quad)
        ours[N] = float(np.max(np.abs(q)))
    Ns = sorted(ours)
    assert all(ours[Ns[i + 1]] < ours[Ns[i]] for i in range(len(Ns) - 1)), ours
    paper64 = [v for N, ns, v in rows if N == 64][0]
    assert 0.1 < ours[64] / paper64 < 10.0, (ours[64], paper64)


# ------------------------------------------------------------ evaluators used as GPU references

@pytest.mark.parametrize("d", [2, 3])
def test_collision_at_points_matches_fast_form(d):
    """The point evaluator (the reference of the full-size sampled GPU
    checks) equals the FFT route at random grid points to rounding."""
    assert pins.at_points_vs_fast(O, d) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_moments_match_gaussian_closed_forms(d):
    """Mass, momentum and energy of a shifted Gaussian (Sec. 2 definitions)."""
    assert pins.moments_gaussian(O, d) < 1e-11


@pytest.mark.parametrize("d", [2, 3])
def test_rk_step_orders_of_accuracy(d):
    """Euler, Heun and classical RK4 converge at orders 1, 2 and 4 against an
    independent ODE solution: a wrong stage weight or stage argument lowers
    the observed order."""
    orders = pins.rk_orders(O, d)
    for p in (1, 2, 4):
        assert abs(orders[p] - p) < 0.3, orders


def test_pooled_fast_form_equals_single_call():
    """The process-parallel driver (node ranges of whole groups, partial sums
    added in node order) gives the single-call fast form to rounding."""
    from oracle.pool import OraclePool, node_ranges
    assert node_ranges(2048, 8, 16)[0] == (0, 128) and node_ranges(2048, 8, 16)[-1][1] == 2048
    assert node_ranges(12, 4, 5) == [(0, 4), (4, 8), (8, 12)]
    quad_args = (3, 3, 8, 6, O.default_R(L), "cube", "octahedron")
    f = I.gaussian_noise(3, 8, L, 3, eps=0.2)
    ref = O.collision_fast(f, L, O.make_quadrature(*quad_args), return_complex=True)
    with OraclePool(2) as pool:
        got, _, _ = pool.collision_fast(f, L, quad_args, parts=5)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
