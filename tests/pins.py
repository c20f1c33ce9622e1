"""Pins of the oracle: each returns a discrepancy that is at rounding level
for a correct oracle.  They take the oracle module as an argument so that a
test can plant a mistake in it (on the CPU) and check the pin catches it.

What each pin rests on (none of them re-types the oracle's formulas):
  operator_vs_bruteforce  Eq. (2.3) integrated in a different parametrisation
  rj_zero                 Eq. (2.6): the bracket vanishes on Rayleigh-Jeans states
  weight_total            sum_p W_p = |S^{d-1}|^2 R^{2d-2}/(2d-2), closed form
  fast_vs_realspace       band-limited f: spectral interpolation is exact
  fast_vs_direct          the FFT route equals the O(N^{3d}) sums (3.3)-(3.6)
  alg1_vs_fast            Algorithm 1 literally vs its linearity-reduced form
  mass_bandlimited        Appendix B's symmetry argument (sum_i Q_i = 0)
  naive_dft               Eq. (3.1) summed term by term
"""
import math

import numpy as np

import wke_inputs as I
from tests import bruteforce_eq23 as BF

L = 8.0


def _gauss(k):
    return np.exp(-0.5 * np.sum(np.asarray(k) ** 2, axis=-1))


def operator_vs_bruteforce(O, d):
    """Relative difference between the oracle's Eq. (2.7) quadrature (many
    nodes, R large enough that truncation is negligible) and the direct
    integral of Eq. (2.3), for a Gaussian f at a few points."""
    if d == 2:
        quad = O.make_quadrature(2, 64, 64, 64, 14.0, "midpoint")
        pts = [[0.3, -0.5], [1.2, 0.4]]
        ref = [BF.collision_2d(_gauss, p) for p in pts]
    else:
        quad = O.make_quadrature(3, 40, 128, 128, 14.0, "product:8:16")
        pts = [[0.3, -0.5, 0.2]]
        ref = [BF.collision_3d(_gauss, p) for p in pts]
    got = O.collision_realspace(_gauss, np.array(pts), quad)
    ref = np.array(ref)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def rj_zero(O, d):
    """max |Q| / max |K1| on Rayleigh-Jeans states for the real-space form
    (any quadrature): the per-node bracket is identically zero."""
    worst = 0.0
    for mu, nu, xi in [(1.0, [0.3, -0.2, 0.1], 0.1), (50.0, [5.0, 5.0, 0.0], 100.0)]:
        if d == 2:
            quad = O.make_quadrature(2, 6, 5, 5, O.default_R(L), "midpoint")
        else:
            quad = O.make_quadrature(3, 4, 8, 6, O.default_R(L), "cube", "octahedron")
        fn = I.rayleigh_jeans_fn(d, mu, nu[:d], xi)
        k = O.grid_points(d, 6, L).reshape(-1, d)
        q = O.collision_realspace(fn, k, quad)
        gain = np.zeros(len(k))
        F = fn(k)
        for _p1, _p2, _p3, W, c, a, b in quad.nodes():
            gain += W * np.abs(fn(k - a) * fn(k - b) * fn(k - c))
        worst = max(worst, float(np.max(np.abs(q)) / np.max(gain * 2.0 ** (1 - d))))
        del F
    return worst


def weight_total(O, d):
    """Relative error of sum_p W_p against |S^{d-1}|^2 R^{2d-2}/(2d-2)."""
    R = 5.5
    if d == 2:
        quad = O.make_quadrature(2, 5, 7, 3, R, "midpoint")
        area = 2.0 * math.pi
    else:
        quad = O.make_quadrature(3, 5, 12, 20, R, "icosahedron", "dodecahedron")
        area = 4.0 * math.pi
    tot = sum(n[3] for n in quad.nodes())
    exact = area * area * R ** (2 * d - 2) / (2 * d - 2)
    return abs(tot - exact) / exact


def fast_vs_realspace(O, d):
    """Band-limited f (|j_c| <= 3 < N/2): the fast form on the grid equals
    the real-space form with the exact f.  The rules are neither antipodal
    nor symmetric under coordinate swaps, so a sign or axis mix-up in the
    shifts cannot cancel between nodes."""
    if d == 2:
        N, quad = 16, O.make_quadrature(2, 6, 3, 5, O.default_R(L), "midpoint")
    else:
        N, quad = 8, O.make_quadrature(3, 3, 6, 6, O.default_R(L), "product:2:3", "octahedron")
    tp = I.trig_poly(d, L, 3, 6, 11)
    qf, _ = O.collision_fast(tp.on_grid(N), L, quad)
    qr = O.collision_realspace(tp, O.grid_points(d, N, L), quad)
    return float(np.max(np.abs(qf - qr)) / np.max(np.abs(qr)))


def fast_vs_direct(O, d, N=None, quad=None, f=None):
    """The FFT route against the classical sums with quadrature weights and
    circular index wrap (the sums N-point transforms compute).  Default rules
    are not antipodal, so A and B (k' and k2') cannot trade places unseen."""
    if quad is None:
        if d == 2:
            N, quad = 8, O.make_quadrature(2, 4, 4, 3, O.default_R(L), "midpoint")
        else:
            N, quad = 4, O.make_quadrature(3, 2, 8, 6, O.default_R(L), "cube", "product:2:3")
    if f is None:
        f = I.gaussian_noise(d, N, L, 99, eps=0.2) * I.gaussian(d, N, L, 1.3)
    qf, imf = O.collision_fast(f, L, quad)
    qd, imd = O.collision_direct(f, L, quad, wrap=True)
    return float(np.max(np.abs(qf - qd)) / np.max(np.abs(qd)))


def alg1_vs_fast(O, d):
    if d == 2:
        N, quad = 8, O.make_quadrature(2, 3, 4, 4, O.default_R(L), "midpoint")
    else:
        N, quad = 4, O.make_quadrature(3, 2, 6, 8, O.default_R(L), "octahedron", "cube")
    f = I.gaussian_noise(d, N, L, 5, eps=0.3)
    qa, _ = O.collision_alg1(f, L, quad)
    qf, _ = O.collision_fast(f, L, quad)
    return float(np.max(np.abs(qa - qf)) / np.max(np.abs(qf)))


def mass_bandlimited(O, d):
    """|sum_i Q_i| / sum_i |Q_i| for f with |j_c| <= N/3 - 1 and the same
    antipodal rule for qhat and sigma (Appendix B's symmetry argument)."""
    if d == 2:
        N, quad = 18, O.make_quadrature(2, 5, 6, 6, O.default_R(L), "midpoint")
    else:
        N, quad = 12, O.make_quadrature(3, 3, 8, 8, O.default_R(L), "cube")
    tp = I.trig_poly(d, L, N // 3 - 1, 8, 3)
    q, _ = O.collision_fast(tp.on_grid(N), L, quad)
    return float(abs(np.sum(q)) / np.sum(np.abs(q)))


def dealiased_vs_linear(O, d, nyquist="keep"):
    """The padded (de-aliased) evaluation against the classical sums of Eqs.
    (3.3)-(3.6) with linear index sums l + m + n = j and quadrature weights.
    The rules are not antipodal, so k' and k2' cannot trade places unseen."""
    if d == 2:
        N, quad = 8, O.make_quadrature(2, 4, 4, 3, O.default_R(L), "midpoint")
    else:
        N, quad = 4, O.make_quadrature(3, 2, 8, 6, O.default_R(L), "cube", "product:2:3")
    f = I.gaussian_noise(d, N, L, 99, eps=0.2) * I.gaussian(d, N, L, 1.3)
    qa = O.collision_dealiased(f, L, quad, nyquist=nyquist, return_complex=True)
    qd = O.iFFT(O.collision_direct(f, L, quad, wrap=False, nyquist=nyquist, return_hat=True), L)
    return float(np.max(np.abs(qa - qd)) / np.max(np.abs(qd)))


def dealiased_mass(O, d):
    """|sum_i Q_i| / sum_i |Q_i| of the de-aliased operator for an f that is
    not band-limited, with the same antipodal rule for qhat and sigma: the
    linear sums have hat K_0 = 0 (Appendix B), whatever the band of f."""
    if d == 2:
        N, quad = 16, O.make_quadrature(2, 5, 6, 6, O.default_R(L), "midpoint")
    else:
        N, quad = 8, O.make_quadrature(3, 3, 8, 8, O.default_R(L), "cube")
    f = I.gaussian_noise(d, N, L, 23, eps=0.4) * I.gaussian(d, N, L, 1.5)
    q = O.collision_dealiased(f, L, quad, return_complex=True)
    return float(abs(np.sum(q)) / np.sum(np.abs(q)))


def dealiased_vs_aliased_bandlimited(O, d):
    """For a trigonometric polynomial with |j_c| < N/6 the cubic products have
    modes in (-N/2, N/2) and wrap on the N grid as little as on the 2N grid,
    so the circular and the linear sums coincide."""
    N = 18 if d == 2 else 12
    quad = O.make_quadrature(d, 3, 6 if d == 2 else 8, 5 if d == 2 else 6, O.default_R(L),
                             "midpoint" if d == 2 else "cube", None if d == 2 else "product:2:3")
    f = I.trig_poly(d, L, (N - 1) // 6, 8, 3).on_grid(N)
    qa = O.collision_dealiased(f, L, quad, return_complex=True)
    qc = O.collision_fast(f, L, quad, return_complex=True)
    return float(np.max(np.abs(qa - qc)) / np.max(np.abs(qc)))


def naive_dft(O, d):
    """FFT/iFFT against Eq. (3.1) summed term by term."""
    N = 6 if d == 2 else 4
    g = I.gaussian_noise(d, N, L, 17, eps=0.5)
    k = O.grid_points(d, N, L).reshape(-1, d)
    j = O.mode_vectors(d, N).reshape(-1, d)
    E = np.exp(-1j * math.pi / L * (j @ k.T))              # (modes, points)
    ref_hat = (E @ g.reshape(-1)) / N ** d
    got_hat = O.FFT(g, L).reshape(-1)
    back = O.iFFT(O.FFT(g, L), L).reshape(-1)
    ref_back = np.conj(E).T @ ref_hat
    return float(max(np.max(np.abs(got_hat - ref_hat)), np.max(np.abs(back - ref_back)),
                     np.max(np.abs(ref_back - g.reshape(-1)))))


def at_points_vs_fast(O, d):
    """The direct series evaluation at chosen points (no FFT) against the
    FFT route over the whole grid, complex Q, at random grid points.  The
    rules are neither antipodal nor symmetric under coordinate swaps, so a
    sign slip in the per-axis phases exp(i pi j (k - x)/L) or an axis-order
    mix-up in the contraction cannot cancel between nodes."""
    if d == 2:
        N, quad = 12, O.make_quadrature(2, 3, 3, 5, O.default_R(L), "midpoint")
    else:
        N, quad = 8, O.make_quadrature(3, 2, 6, 6, O.default_R(L), "product:2:3", "octahedron")
    f = I.gaussian_noise(d, N, L, 41, eps=0.3) * I.gaussian(d, N, L, 1.4)
    full = O.collision_fast(f, L, quad, return_complex=True)
    u = I.splitmix64_uniform(977 + d, 12 * d).reshape(12, d)
    pts = [tuple(int(v) for v in row) for row in np.floor(u * N).astype(np.int64)]
    got = O.collision_at_points(f, L, quad, pts, chunk=7)
    ref = np.array([full[p] for p in pts])
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(full)))


def moments_gaussian(O, d):
    """Moments of a shifted anisotropic-centre Gaussian A exp(-|k - c|^2/(2 s^2))
    against their closed forms (Sec. 2: rho = int f, E = int f |k|^2):
    mass A (2 pi s^2)^{d/2}, momentum c * mass, energy (d s^2 + |c|^2) * mass.
    With s = 0.9 at L = 8 the tails beyond the box are below 1e-12 of the
    mass and the rectangle rule at h = 0.5 is exact to rounding for a
    Gaussian (its error decays like exp(-2 pi^2 s^2 / h^2))."""
    N, s, A = 32, 0.9, 1.7
    c = np.array([0.7, -1.1, 0.4][:d])
    ks = I.grid_axes(d, N, L)
    r2 = sum((ks[a] - c[a]) ** 2 for a in range(d))
    g = A * np.exp(-r2 / (2.0 * s * s))
    mass = A * (2.0 * math.pi * s * s) ** (d / 2.0)
    exact = np.concatenate([[mass], c * mass, [(d * s * s + float(c @ c)) * mass]])
    got = O.moments(g, L)
    return float(np.max(np.abs(got - exact)) / mass)


def _rk_problem(O, d):
    """A small smooth system df/dt = Re Q(f) and its time span."""
    if d == 2:
        N, quad = 8, O.make_quadrature(2, 3, 4, 3, O.default_R(L), "midpoint")
    else:
        N, quad = 4, O.make_quadrature(3, 2, 6, 6, O.default_R(L), "octahedron", "product:2:3")
    f0 = I.gaussian_noise(d, N, L, 7, eps=0.3) * I.gaussian(d, N, L, 1.6)
    q0, _ = O.collision_fast(f0, L, quad)
    T = 0.15 * float(np.max(np.abs(f0))) / float(np.max(np.abs(q0)))
    return f0, quad, T


def rk_orders(O, d):
    """Observed convergence orders of rk_step (Euler, Heun, classical RK4,
    the paper's integrator in Sec. 4) against an independent high-accuracy
    solution of the same ODE system (scipy's DOP853 at rtol 1e-13 on the
    pinned operator).  Returns {stages: order} from the errors at n and 2n
    steps over the same span."""
    from scipy.integrate import solve_ivp
    f0, quad, T = _rk_problem(O, d)
    shape = f0.shape

    def rhs(_t, y):
        return O.collision_fast(y.reshape(shape), L, quad)[0].reshape(-1)

    sol = solve_ivp(rhs, (0.0, T), f0.reshape(-1), method="DOP853", rtol=1e-13, atol=1e-15)
    ref = sol.y[:, -1].reshape(shape)
    orders = {}
    for stages, n in ((1, 8), (2, 4), (4, 2)):
        errs = []
        for steps in (n, 2 * n):
            f = f0.copy()
            for _ in range(steps):
                f = O.rk_step(f, L, quad, T / steps, stages)
            errs.append(float(np.max(np.abs(f - ref))))
        orders[stages] = math.log2(errs[0] / errs[1])
    return orders


def rk_order_defect(O, d):
    """max over the three schemes of |observed order - design order|."""
    orders = rk_orders(O, d)
    return max(abs(orders[p] - p) for p in (1, 2, 4))
