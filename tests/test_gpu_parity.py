"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (relative max-norm against the oracle's max |Q|): FP64 1e-12;
FP32 1e-5 on the benchmark workloads, and on the other full-field cases the
larger of 1e-5 and the bound eps32 log2(N^d) kappa derived from the
cancellation kappa of the four cubic terms (``gpu_util.fp32_tolerance``).
Inputs are the seeded generators of ``wke_inputs``.
"""
import math

import numpy as np
import pytest

import wke_inputs as I
from oracle import wke_oracle as O
from tests.gpu_util import fp32_tolerance, gpu_collision, rel_max_err, require_cuda

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _plan(wke, d, N, L, n_r, n_s, n_sig, sphere=None, sphere_sig=None, **kw):
    return wke.Plan(d, N, L, n_r, n_s, n_sig, sphere=sphere, sphere_sig=sphere_sig, **kw)


def _oracle_quad(d, L, n_r, n_s, n_sig, sphere, sphere_sig=None, R=None):
    return O.make_quadrature(d, n_r, n_s, n_sig, R or O.default_R(L), sphere, sphere_sig)


CASES = [
    # name, d, N, n_r, n_s, n_sig, sphere, sphere_sig, input
    ("2d_n16_m32 workload", 2, 16, 8, 4, 1, "midpoint", None, lambda: I.WORKLOADS["2d_n16_m32"].initial()),
    ("2d_n16 Rayleigh-Jeans", 2, 16, 8, 4, 1, "midpoint", None,
     lambda: I.rayleigh_jeans(2, 16, 8.0, 1.0, [0.0, 0.0], 0.1)),
    ("2d_n32 paired", 2, 32, 6, 4, 4, "midpoint", None, lambda: I.two_gaussians(32, 8.0, 5)),
    ("2d_n32 odd sigma rule", 2, 32, 5, 5, 3, "midpoint", None, lambda: I.gaussian_noise(2, 32, 8.0, 9, 0.2)),
    ("2d_n64", 2, 64, 4, 6, 6, "midpoint", None, lambda: I.two_gaussians(64, 8.0, 6)),
    ("2d_n256", 2, 256, 3, 4, 4, "midpoint", None, lambda: I.two_gaussians(256, 8.0, 7)),
    ("3d_n16 cube", 3, 16, 3, 8, 8, "cube", None, lambda: I.gaussian_noise(3, 16, 8.0, 11, 0.1)),
    ("3d_n16 non-antipodal sigma", 3, 16, 2, 8, 6, "cube", "product:2:3",
     lambda: I.gaussian_noise(3, 16, 8.0, 12, 0.1)),
    ("3d_n32 icosahedron/dodecahedron", 3, 32, 2, 12, 20, "icosahedron", "dodecahedron",
     lambda: I.ring(3, 32, 8.0)),
    # lengths 3 * 2^a (radix-12 stages)
    ("2d_n48", 2, 48, 4, 4, 4, "midpoint", None, lambda: I.two_gaussians(48, 8.0, 13)),
    ("2d_n96 odd sigma rule", 2, 96, 3, 4, 3, "midpoint", None, lambda: I.gaussian_noise(2, 96, 8.0, 14, 0.2)),
    ("3d_n48 cube", 3, 48, 2, 8, 8, "cube", None, lambda: I.ring(3, 48, 8.0)),
    ("3d_n48 non-antipodal sigma", 3, 48, 2, 6, 6, "octahedron", "product:2:3",
     lambda: I.gaussian_noise(3, 48, 8.0, 15, 0.1)),
]


@pytest.mark.parametrize("layout", ["per_group", "shared"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_full_field_parity(case, prec, layout):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    name, d, N, n_r, n_s, n_sig, sph, sph_sig, gen = case
    L = 8.0
    f = gen()
    quad = _oracle_quad(d, L, n_r, n_s, n_sig, sph, sph_sig)
    ref = O.collision_fast(f, L, quad, return_complex=True)
    with _plan(wke, d, N, L, n_r, n_s, n_sig, sph, sph_sig, precision=prec, layout=layout) as plan:
        assert plan.info().shared_fields == (layout == "shared")
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    scale = np.max(np.abs(ref))
    tol = TOL[prec] if prec == "fp64" else fp32_tolerance(f, L, quad)
    assert rel_max_err(Q, ref.real, scale) <= tol, name
    assert rel_max_err(Qim, ref.imag, scale) <= tol, name


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload_3d_n32_m1024(prec):
    """3D N=32, M=1024 (16 radial x 8 x 8 cube directions), Gaussian with 1%
    seeded noise: full field."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["3d_n32_m1024"]
    f = w.initial()
    ref, _ = O.collision_fast(f, w.L, _oracle_quad(3, w.L, w.n_r, w.n_s, w.n_sig, w.sphere))
    with _plan(wke, 3, w.N, w.L, w.n_r, w.n_s, w.n_sig, w.sphere, precision=prec) as plan:
        Q = gpu_collision(torch, plan, f)
    assert rel_max_err(Q, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload_2d_n128_m512(prec):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["2d_n128_m512"]
    f = w.initial()
    ref, _ = O.collision_fast(f, w.L, _oracle_quad(2, w.L, w.n_r, w.n_s, w.n_sig, w.sphere))
    with _plan(wke, 2, w.N, w.L, w.n_r, w.n_s, w.n_sig, w.sphere, precision=prec) as plan:
        Q = gpu_collision(torch, plan, f)
    assert rel_max_err(Q, ref) <= TOL[prec]


def _ring_sample_points(N, L, count, seed):
    """Grid indices on and near the ring |k| = 3 (where Q is large), plus
    seeded random points."""
    k = O.grid_1d(N, L)
    pts = []
    u = I.splitmix64_uniform(seed, 4 * count)
    for i in range(count):
        th, ph = math.pi * u[4 * i], 2 * math.pi * u[4 * i + 1]
        rad = 2.5 + 1.0 * u[4 * i + 2]
        x = rad * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        pts.append(tuple(int(np.argmin(np.abs(k - xa))) for xa in x))
    pts.append(tuple(int(v) for v in np.floor(u[:3] * N)))
    return pts


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_workload_3d_n64_m2048_sampled(prec):
    """The headline size, in the configuration the benchmark times (default
    chunking): sampled points against the oracle's direct series evaluation."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["3d_n64_m2048"]
    f = w.initial()
    pts = _ring_sample_points(w.N, w.L, 5, 4242)
    ref = O.collision_at_points(f, w.L, _oracle_quad(3, w.L, w.n_r, w.n_s, w.n_sig, w.sphere), pts)
    with _plan(wke, 3, w.N, w.L, w.n_r, w.n_s, w.n_sig, w.sphere, precision=prec) as plan:
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    got = np.array([Q[p] for p in pts])
    goti = np.array([Qim[p] for p in pts])
    scale = np.max(np.abs(ref))
    assert rel_max_err(got, ref.real, scale) <= TOL[prec]
    assert rel_max_err(goti, ref.imag, scale) <= TOL[prec]


@pytest.fixture(scope="module")
def headline_reference():
    """The oracle's fast form of the 3D N=64, M=2048 workload over the whole
    grid, evaluated over node ranges on every host core (spawn pool) and
    summed in node order."""
    from oracle.pool import OraclePool
    w = I.WORKLOADS["3d_n64_m2048"]
    f = w.initial()
    with OraclePool() as pool:
        ref, wall, _ = pool.collision_fast(f, w.L, (3, w.n_r, w.n_s, w.n_sig, O.default_R(w.L), w.sphere))
    return f, ref


# The headline workload is held to its target tolerances over the whole grid:
# FP64 1e-12, and 1e-6 for both the FP32 path and the split-precision path.
HEADLINE_TOL = {"fp64": 1e-12, "fp32": 1e-6, "split": 1e-6}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "split"])
def test_workload_3d_n64_m2048_full_field(headline_reference, prec):
    """3D N=64, M=2048 (32 radial x 8 x 8 cube, ring f), in the configuration
    the benchmark times, against the oracle at every grid point: Re Q and
    Im Q, relative max-norm against max |Q|."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["3d_n64_m2048"]
    f, ref = headline_reference
    scale = np.max(np.abs(ref))
    with _plan(wke, 3, w.N, w.L, w.n_r, w.n_s, w.n_sig, w.sphere, precision=prec) as plan:
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
        assert rel_max_err(Q, ref.real, scale) <= HEADLINE_TOL[prec]
        assert rel_max_err(Qim, ref.imag, scale) <= HEADLINE_TOL[prec]
        if prec == "fp32":
            # the benchmark's call (Re Q only), with the cube rule's own product
            # schedule (the default) and with the generic one
            assert plan.info().rule_products_available == 1
            for rp in (1, 0):
                wke.wke_plan_set_tuning(plan.handle, 8, 0, 1, 0, rp)
                assert wke.wke_plan_get_tuning(plan.handle).rule_products == rp
                assert rel_max_err(gpu_collision(torch, plan, f), ref.real, scale) <= HEADLINE_TOL[prec], rp


def test_3d_n64_full_field_small_quadrature():
    """N = 64 in 3D over the whole grid (fewer nodes so the oracle stays fast)."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.ring(3, 64, 8.0)
    ref, _ = O.collision_fast(f, 8.0, _oracle_quad(3, 8.0, 2, 8, 8, "cube"))
    for prec in ("fp64", "fp32"):
        with _plan(wke, 3, 64, 8.0, 2, 8, 8, "cube", precision=prec) as plan:
            Q = gpu_collision(torch, plan, f)
        assert rel_max_err(Q, ref) <= TOL[prec], prec


@pytest.mark.parametrize("dealias", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("d,N", [(2, 32), (3, 16), (3, 64)])
def test_collision_spectrum(d, N, prec, dealias):
    """Q-hat (Algorithm 1's coefficients before the final inverse transform):
    the GPU's Q-hat against the oracle's Eq. (3.1) transform of the oracle's
    Q, elementwise, relative to max |Q| (each coefficient is a mean of Q times
    unit phases, so an error e max |Q| in Q moves it by at most that); Q
    itself as wke_collision gives it; and the mode-0 coefficient equals the
    grid mean of the GPU's own Q (to the output precision)."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    if dealias and (d, N) == (3, 64):
        pytest.skip("the de-aliased plan of this case transforms on 128^3, outside the 3D lengths")
    sph = "midpoint" if d == 2 else "cube"
    n_r = 2 if N == 64 else 3
    f = I.gaussian_noise(d, N, 8.0, 77, 0.2)
    quad = _oracle_quad(d, 8.0, n_r, 4 if d == 2 else 8, 4 if d == 2 else 8, sph)
    nyq = "zero" if dealias else "keep"
    if dealias:
        ref = O.collision_dealiased(f, 8.0, quad, nyquist=nyq)
    else:
        ref = O.collision_fast(f, 8.0, quad, nyquist=nyq)
    ref = ref[0] if isinstance(ref, tuple) else ref
    ref_hat = O.FFT(ref, 8.0)
    kw = {"nyquist": nyq, "dealias": dealias}
    with _plan(wke, d, N, 8.0, quad.n_r, quad.n_s, quad.n_sig, sph, precision=prec, **kw) as plan:
        ft = torch.tensor(f, dtype=plan.dtype, device="cuda")
        Q, Qhat = plan.spectrum(ft)
        torch.cuda.synchronize()
        Q, Qhat = Q.double().cpu().numpy(), Qhat.cpu().numpy().astype(np.complex128)
        with pytest.raises(wke.WkeError):
            plan.spectrum(ft, Q=ft)                    # Q may not overlap f
    tol = TOL[prec] if prec == "fp64" else max(TOL[prec], fp32_tolerance(f, 8.0, quad, dealias=dealias,
                                                                           nyquist=nyq))
    scale = np.max(np.abs(ref))
    assert rel_max_err(Q, ref) <= tol
    assert np.max(np.abs(Qhat - ref_hat)) / scale <= tol
    assert abs(Qhat.flat[0] - Q.mean()) <= (1e-12 if prec == "fp64" else 1e-6) * np.max(np.abs(Q))


@pytest.mark.parametrize("d,N", [(2, 32), (3, 16)])
def test_nyquist_zero_mode(d, N):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    sph = "midpoint" if d == 2 else "cube"
    f = I.gaussian_noise(d, N, 8.0, 31, 0.3)
    quad = _oracle_quad(d, 8.0, 3, 4 if d == 2 else 8, 4 if d == 2 else 8, sph)
    ref = O.collision_fast(f, 8.0, quad, nyquist="zero", return_complex=True)
    with _plan(wke, d, N, 8.0, quad.n_r, quad.n_s, quad.n_sig, sph, nyquist="zero") as plan:
        Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
    assert rel_max_err(Q, ref.real) <= 1e-12
    assert np.max(np.abs(Qim)) <= 1e-12 * np.max(np.abs(ref))


def test_pairing_and_chunking_do_not_change_the_sum():
    """Antipodal pairing (shared fields and products) and the chunk size only
    reorder the same sum."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.gaussian_noise(3, 32, 8.0, 41, 0.05)
    res = []
    for pair, chunk in ((True, 0), (False, 0), (True, 1), (False, 3 << 20)):
        with _plan(wke, 3, 32, 8.0, 5, 8, 8, "cube", pair_antipodal=pair, chunk_bytes=chunk) as plan:
            info = plan.info()
            assert info.fields_per_group == (9 if pair else 17)
            assert info.products_per_group == (3 if pair else 8)
            res.append(gpu_collision(torch, plan, f))
    for r in res[1:]:
        assert rel_max_err(r, res[0]) <= 1e-13


def test_vanishing_nodes_dropped_only_where_exactly_zero():
    """sigma = +-qhat makes {k', k2'} = {k, k - q}: the bracket vanishes when
    F equals the interpolant on the transform grid.  The cube rule pairs into
    4 products per group, one of them (qhat, -qhat); it is dropped with the
    Nyquist modes kept and in a de-aliased plan, kept when F = f(k) differs
    from the zeroed interpolant, and every node stays without pairing."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.gaussian_noise(3, 16, 8.0, 43, 0.1)
    quad = _oracle_quad(3, 8.0, 2, 8, 8, "cube")
    for kw, ppg, oracle in (
            (dict(), 3, lambda: O.collision_fast(f, 8.0, quad, return_complex=True)),
            (dict(nyquist="zero"), 4, lambda: O.collision_fast(f, 8.0, quad, nyquist="zero", return_complex=True)),
            (dict(nyquist="zero", dealias=True), 3,
             lambda: O.collision_dealiased(f, 8.0, quad, nyquist="zero", return_complex=True)),
            (dict(pair_antipodal=False), 8, lambda: O.collision_fast(f, 8.0, quad, return_complex=True))):
        with _plan(wke, 3, 16, 8.0, 2, 8, 8, "cube", **kw) as plan:
            assert plan.info().products_per_group == ppg, kw
            Q, Qim = gpu_collision(torch, plan, f, want_imag=True)
        ref = oracle()
        scale = np.max(np.abs(ref))
        assert rel_max_err(Q, ref.real, scale) <= 1e-12, kw
        assert rel_max_err(Qim, ref.imag, scale) <= 1e-12, kw


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shared_and_per_group_layouts_agree_at_3d_n64(prec):
    """The benchmark's rule at 3D N=64 on two radii: each distinct shifted
    field transformed once per chunk (26 of the 56 the per-group layout
    transforms per radius) gives the same Q."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.ring(3, 64, 8.0)
    out = {}
    for layout in ("shared", "per_group"):
        with _plan(wke, 3, 64, 8.0, 2, 8, 8, "cube", precision=prec, layout=layout) as plan:
            info = plan.info()
            out[layout] = (gpu_collision(torch, plan, f), info.units_per_collision)
    assert out["per_group"][1] == 2 * (4 + 8 * 3)
    assert out["shared"][1] == 2 * 13          # one radius per chunk: 26 fields in 13 units
    assert rel_max_err(out["shared"][0], out["per_group"][0]) <= TOL[prec]


def test_deterministic_repeat():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.ring(3, 32, 8.0)
    with _plan(wke, 3, 32, 8.0, 4, 8, 8, "cube", precision="fp32") as plan:
        a = gpu_collision(torch, plan, f)
        b = gpu_collision(torch, plan, f)
    assert np.array_equal(a, b)


def test_dispersion_k2_halves_q():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.two_gaussians(32, 8.0, 3)
    with _plan(wke, 2, 32, 8.0, 4, 4, 4, "midpoint") as p1, \
            _plan(wke, 2, 32, 8.0, 4, 4, 4, "midpoint", dispersion="k2") as p2:
        a = gpu_collision(torch, p1, f)
        b = gpu_collision(torch, p2, f)
    assert rel_max_err(b, 0.5 * a) <= 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_moments_match_oracle(prec):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    for d, N in ((2, 64), (3, 32)):
        g = I.two_gaussians(N, 8.0, 2) if d == 2 else I.ring(3, N, 8.0)
        with _plan(wke, d, N, 8.0, 2, 4 if d == 2 else 8, 4 if d == 2 else 8, precision=prec) as plan:
            gt = torch.tensor(g, dtype=plan.dtype, device="cuda")
            m = plan.moments(gt).cpu().numpy()
        ref = O.moments(gt.double().cpu().numpy(), 8.0)
        scale = np.abs(ref).max()
        assert np.max(np.abs(m - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("stages", [1, 2, 4])
def test_rk_step_matches_oracle(stages):
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    N, L, dt = 32, 8.0, 0.05
    f0 = I.two_gaussians(N, L, 8)
    quad = _oracle_quad(2, L, 6, 4, 4, "midpoint")
    ref = f0.copy()
    for _ in range(2):
        ref = O.rk_step(ref, L, quad, dt, stages)
    with _plan(wke, 2, N, L, 6, 4, 4, "midpoint") as plan:
        ft = torch.tensor(f0, dtype=torch.float64, device="cuda")
        for _ in range(2):
            plan.step(ft, dt, stages)
        torch.cuda.synchronize()
        got = ft.cpu().numpy()
    change = np.max(np.abs(ref - f0))
    assert np.max(np.abs(got - ref)) <= 1e-12 * change


def test_host_buffer_call_matches_device_call():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.ring(3, 32, 8.0).astype(np.float32)
    with _plan(wke, 3, 32, 8.0, 3, 8, 8, "cube", precision="fp32") as plan:
        dev = gpu_collision(torch, plan, f)
        fh = torch.tensor(f).pin_memory()
        qh = torch.empty_like(fh).pin_memory()
        plan.collision_host(fh, qh)
    assert np.array_equal(qh.double().numpy(), dev)


def test_graph_replay_matches_direct_launches():
    """The cached CUDA graph of an evaluation replays exactly the kernels the
    direct path launches; several pointer sets share one plan."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    fs = [I.ring(3, 32, 8.0), I.gaussian_noise(3, 32, 8.0, 77, 0.1)]
    with _plan(wke, 3, 32, 8.0, 4, 8, 8, "cube", precision="fp32", chunk_bytes=2 << 20) as plan:
        assert plan.info().n_chunks > 2            # exercises both intermediate buffers
        ft = [torch.tensor(f, dtype=torch.float32, device="cuda") for f in fs]
        graph = [[plan.collision(f) for f in ft] for _ in range(2)]
        wke.wke_plan_use_graphs(plan.handle, False)
        direct = [plan.collision(f) for f in ft]
        torch.cuda.synchronize()
    for g_rep in graph:
        for a, b in zip(g_rep, direct):
            assert torch.equal(a, b)


@pytest.mark.parametrize("layout", ["shared", "separable"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_launch_layout_matches_oracle(prec, layout):
    """Each layout the autotuner may pick computes the same Q (to rounding):
    axis-0 points per thread, pass-1 units per block and, in FP32, the fused
    or separate axis-0 and product kernels; the autotuner returns one of
    them."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f = I.gaussian_noise(3, 32, 8.0, 55, 0.1)
    ref, _ = O.collision_fast(f, 8.0, _oracle_quad(3, 8.0, 3, 8, 8, "cube"))
    with _plan(wke, 3, 32, 8.0, 3, 8, 8, "cube", precision=prec, layout=layout) as plan:
        assert plan.info().separable == (layout == "separable")
        assert plan.info().fused_products == (prec == "fp32")
        for fwd32 in ((0, 1) if prec == "fp32" else (0,)):
            for fuse in ((1, 0) if prec == "fp32" else (0,)):
                for p2 in (4, 8):
                    for p1 in (0, 1, 2, 3):
                        wke.wke_plan_set_tuning(plan.handle, p2, p1, fuse, fwd32)
                        assert plan.info().fused_products == fuse
                        Q = gpu_collision(torch, plan, f)
                        assert rel_max_err(Q, ref) <= TOL[prec], (fwd32, fuse, p2, p1)
        wke.wke_plan_set_tuning(plan.handle, 8, 0, int(prec == "fp32"), 0)
        ft = torch.tensor(f, dtype=plan.dtype, device="cuda")
        tuning, ms = plan.autotune(ft, reps=2)
        assert tuning.pass2_points_per_thread in (4, 8) and ms > 0
        Q = gpu_collision(torch, plan, f)
        assert rel_max_err(Q, ref) <= TOL[prec]
        with pytest.raises(wke.WkeError):
            wke.wke_plan_set_tuning(plan.handle, 6, 0)
        if prec == "fp64":
            with pytest.raises(wke.WkeError):
                wke.wke_plan_set_tuning(plan.handle, 8, 0, 1)
            with pytest.raises(wke.WkeError):
                wke.wke_plan_set_tuning(plan.handle, 8, 0, 0, 1)


def test_step_graph_matches_direct_launches():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    f0 = I.two_gaussians(64, 8.0, 21).astype(np.float32)
    out = []
    for graphs in (True, False):
        with _plan(wke, 2, 64, 8.0, 8, 4, 4, "midpoint", precision="fp32") as plan:
            wke.wke_plan_use_graphs(plan.handle, graphs)
            ft = torch.tensor(f0, device="cuda")
            for _ in range(3):
                plan.step(ft, 1e-3, 4)
            torch.cuda.synchronize()
            out.append(ft.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_workload_2d_n128_rk4_fp32_vs_fp64_and_conservation():
    """2D N=128, M=512, RK4, dt = 1e-3, the workload's full 200 steps (Sec. 4
    integrates with RK4): the FP64 trajectory equals the oracle's rk_step
    after steps 1 and 2, the FP32 trajectory stays within 1e-5 of the FP64
    one after 200 steps, and mass and energy drift stay small next to their
    values."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["2d_n128_m512"]
    f0 = w.initial()
    quad = _oracle_quad(2, w.L, w.n_r, w.n_s, w.n_sig, w.sphere)
    oracle_steps = [f0]
    for _ in range(2):
        oracle_steps.append(O.rk_step(oracle_steps[-1], w.L, quad, 1e-3, 4))
    finals, moms, early = {}, {}, {}
    for prec in ("fp64", "fp32"):
        with _plan(wke, 2, w.N, w.L, w.n_r, w.n_s, w.n_sig, w.sphere, precision=prec) as plan:
            ft = torch.tensor(f0, dtype=plan.dtype, device="cuda")
            m0 = plan.moments(ft).cpu().numpy()
            for k in range(200):
                plan.step(ft, 1e-3, 4)
                if k < 2:
                    torch.cuda.synchronize()
                    early.setdefault(prec, []).append(ft.double().cpu().numpy())
            m1 = plan.moments(ft).cpu().numpy()
            torch.cuda.synchronize()
            finals[prec] = ft.double().cpu().numpy()
            moms[prec] = (m0, m1)
    for k in range(2):
        change = np.max(np.abs(oracle_steps[k + 1] - f0))
        assert np.max(np.abs(early["fp64"][k] - oracle_steps[k + 1])) <= 1e-12 * change, k
    assert rel_max_err(finals["fp32"], finals["fp64"]) <= 1e-5
    m0, m1 = moms["fp64"]
    assert abs(m1[0] - m0[0]) <= 1e-6 * abs(m0[0])       # mass
    assert abs(m1[3] - m0[3]) <= 1e-6 * abs(m0[3])       # energy
    assert not np.allclose(finals["fp64"], f0)


def test_workload_3d_n64_rk2_50_steps_fp32_vs_fp64():
    """3D N=64, M=2048, ring f, RK2 (Heun) for the workload's 50 steps in both
    precisions (dt = 1e-5: the ring's |Q| reaches about 770, so explicit
    steps of 1e-3 are unstable); the FP32 trajectory stays within 1e-5 of the
    FP64 one at the same step count, and both conserve mass to 1e-6."""
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    w = I.WORKLOADS["3d_n64_m2048"]
    f0 = w.initial()
    finals, mass = {}, {}
    for prec in ("fp64", "fp32"):
        with _plan(wke, 3, w.N, w.L, w.n_r, w.n_s, w.n_sig, w.sphere, precision=prec) as plan:
            ft = torch.tensor(f0, dtype=plan.dtype, device="cuda")
            m0 = plan.moments(ft).cpu().numpy()
            for _ in range(50):
                plan.step(ft, 1e-5, 2)
            m1 = plan.moments(ft).cpu().numpy()
            torch.cuda.synchronize()
            finals[prec] = ft.double().cpu().numpy()
            mass[prec] = abs(m1[0] - m0[0]) / abs(m0[0])
    assert rel_max_err(finals["fp32"], finals["fp64"]) <= 1e-5
    assert mass["fp64"] <= 1e-6 and mass["fp32"] <= 1e-6
    assert not np.allclose(finals["fp64"], f0)
