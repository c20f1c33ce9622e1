"""The C-ABI library loads, exports every function include/wke.h declares,
and rejects bad arguments with error codes (no GPU work involved)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wke():
    from paper_2503_12805_gb300 import build, wke as w
    build()
    w.lib()
    return w


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(wke_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(wke):
    names = _declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(wke.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(wke.EXPORTED) <= set(names)


def test_version_and_defaults(wke):
    assert b"sm_103a" in wke.lib().wke_version()
    q = wke.wke_quadrature_default()
    assert q.precision == wke.WKE_FP64 and q.pair_antipodal == 1 and q.sphere_rule == -1


@pytest.mark.parametrize("d,N,L,M,nr,ns,nsig,code", [
    (4, 32, 8.0, 8, 2, 2, 2, -1),        # bad dimension
    (2, 32, -1.0, 8, 2, 2, 2, -1),       # bad L
    (2, 32, 8.0, 9, 2, 2, 2, -1),        # M != n_r n_s n_sig
    (2, 33, 8.0, 8, 2, 2, 2, -1),        # odd N
    (2, 80, 8.0, 8, 2, 2, 2, -4),        # valid N, no kernel built
    (2, 24, 8.0, 8, 2, 2, 2, -4),        # 3 * 2^3: no kernel built
    (3, 96, 8.0, 64, 1, 8, 8, -4),       # 96 is built for 2D only
    (3, 128, 8.0, 64, 1, 8, 8, -4),      # 3D N=128 not built
    (3, 32, 8.0, 2 * 7 * 8, 2, 7, 8, -1),  # no Platonic design with 7 points
])
def test_invalid_arguments_return_codes(wke, d, N, L, M, nr, ns, nsig, code):
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = nr, ns, nsig
    size = ctypes.c_size_t()
    rc = wke.lib().wke_plan_footprint_bytes(d, N, L, M, ctypes.byref(q), ctypes.byref(size))
    assert rc == code
    assert wke.lib().wke_last_error_string()
    out = ctypes.c_void_p(123)
    assert wke.lib().wke_plan_create(d, N, L, M, ctypes.byref(q), ctypes.byref(out)) == code
    assert out.value is None


def test_null_arguments(wke):
    lib = wke.lib()
    assert lib.wke_quadrature_default(None) == wke.WKE_ERR_INVALID
    assert lib.wke_collision(None, None, None, None) == wke.WKE_ERR_INVALID
    assert lib.wke_step(None, None, 0.1, 4) == wke.WKE_ERR_INVALID
    assert lib.wke_plan_destroy(None) == wke.WKE_OK


def test_footprint_scales_with_precision_and_chunk(wke):
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = 32, 8, 8
    b64 = wke.wke_plan_footprint_bytes(3, 64, 8.0, 2048, q)
    q.precision = wke.WKE_FP32
    b32 = wke.wke_plan_footprint_bytes(3, 64, 8.0, 2048, q)
    q.chunk_bytes = 8 << 20
    b32s = wke.wke_plan_footprint_bytes(3, 64, 8.0, 2048, q)
    assert b32s < b32 < b64


def test_dealias_argument_checks_and_footprint(wke):
    """De-aliased plans need the Nyquist modes zeroed and 2N among the compiled
    lengths; they hold more memory than the circular plan of the same N."""
    size = ctypes.c_size_t()
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = 4, 4, 4
    q.alias = wke.WKE_DEALIAS_PAD2
    lib = wke.lib()
    assert lib.wke_plan_footprint_bytes(2, 32, 8.0, 64, ctypes.byref(q), ctypes.byref(size)) == wke.WKE_ERR_INVALID
    assert b"NYQ_ZERO" in lib.wke_last_error_string()
    q.nyquist = wke.WKE_NYQ_ZERO
    assert lib.wke_plan_footprint_bytes(2, 256, 8.0, 64, ctypes.byref(q), ctypes.byref(size)) == -4
    q.n_s, q.n_sig = 8, 8
    assert lib.wke_plan_footprint_bytes(3, 64, 8.0, 256, ctypes.byref(q), ctypes.byref(size)) == -4
    q.alias = 7
    assert lib.wke_plan_footprint_bytes(3, 32, 8.0, 256, ctypes.byref(q), ctypes.byref(size)) == wke.WKE_ERR_INVALID
    q.alias = wke.WKE_DEALIAS_PAD2
    q.chunk_bytes = 1 << 20            # one group per chunk: buffers scale with the grid
    dealiased = wke.wke_plan_footprint_bytes(3, 32, 8.0, 256, q)
    q.alias = wke.WKE_ALIAS_CIRCULAR
    circular = wke.wke_plan_footprint_bytes(3, 32, 8.0, 256, q)
    assert dealiased > 4 * circular


def test_split_precision_argument_checks(wke):
    """WKE_SPLIT runs on the shared-field layout with a 3D grid of N = 32 or 64."""
    size = ctypes.c_size_t()
    lib = wke.lib()
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = 2, 8, 8
    q.precision = wke.WKE_SPLIT
    assert lib.wke_plan_footprint_bytes(3, 64, 8.0, 128, ctypes.byref(q), ctypes.byref(size)) == wke.WKE_OK
    assert lib.wke_plan_footprint_bytes(3, 48, 8.0, 128, ctypes.byref(q), ctypes.byref(size)) == -4
    q.n_s, q.n_sig = 4, 4
    assert lib.wke_plan_footprint_bytes(2, 64, 8.0, 32, ctypes.byref(q), ctypes.byref(size)) == -4
    q.n_s, q.n_sig = 8, 8
    q.layout = wke.WKE_LAYOUT_PER_GROUP
    assert lib.wke_plan_footprint_bytes(3, 64, 8.0, 128, ctypes.byref(q), ctypes.byref(size)) == wke.WKE_ERR_INVALID


def _describe(wke, d, N, nr, ns, nsig, **fields):
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = nr, ns, nsig
    for k, v in fields.items():
        setattr(q, k, v)
    return wke.wke_plan_describe(d, N, 8.0, nr * ns * nsig, q)


def test_shared_field_layout_counts(wke):
    """The shared-field layout on the benchmark rule (3D N=64, 32 x 8 x 8 cube):
    per radius 26 distinct shifted fields (8 C fields r qhat, 6 edge and 12
    face-diagonal differences r (qhat - sigma)/2) in 13 units, one radius per
    chunk, 3 products per group after the vanishing sigma = +-qhat pair;
    the per-group layout transforms 896 units.  No device work is done."""
    info = _describe(wke, 3, 64, 32, 8, 8, precision=wke.WKE_FP32)
    assert info.shared_fields == 1 and info.products_per_group == 3
    assert info.n_chunks == 32 and info.units_per_collision == 32 * 13
    # separable transforms: the 26 shifts are the nonzero points of {-1,0,1}^3 times r/sqrt 3,
    # so 3 distinct x2 values and 9 distinct (x1, x2) pairs per radius
    assert info.separable == 1 and info.pair_planes_per_collision == 32 * 9
    # FP32: the axis-0 transform runs inside the product kernel; per chunk Nyquist
    # tables, the trailing-axis pass and the fused pass
    assert info.fused_products == 1
    # (no finalize launch: the last chunk's product kernel writes Q)
    assert info.launches_per_collision == 3 + 3 * 32         # forward: rows, axis 1, axis 0
    # every radius has the cube rule's structure: 6 edge, 12 face and 8 vertex shifts, each
    # group pairing its vertex's edge and face fields axis by axis
    assert info.rule_products_available == 1
    fp64 = _describe(wke, 3, 64, 32, 8, 8, precision=wke.WKE_FP64)
    assert fp64.units_per_collision == 32 * 13            # a whole radius fits the FP64 budget
    assert fp64.separable == 1 and fp64.fused_products == 0
    assert fp64.launches_per_collision == 3 + 4 * 32 + 1
    assert fp64.rule_products_available == 0             # no fused kernel in FP64
    unsep = _describe(wke, 3, 64, 32, 8, 8, precision=wke.WKE_FP32, layout=wke.WKE_LAYOUT_SHARED)
    assert unsep.separable == 0 and unsep.fused_products == 1 and unsep.pair_planes_per_collision == 0
    assert unsep.units_per_collision == 32 * 13
    per_group = _describe(wke, 3, 64, 32, 8, 8, precision=wke.WKE_FP32, layout=wke.WKE_LAYOUT_PER_GROUP)
    assert per_group.shared_fields == 0 and per_group.units_per_collision == 256 * 3 + 128
    # with the Nyquist modes zeroed F is not the grid interpolant: no product vanishes
    zero = _describe(wke, 3, 64, 32, 8, 8, precision=wke.WKE_FP32, nyquist=wke.WKE_NYQ_ZERO)
    assert zero.products_per_group == 4 and zero.rule_products_available == 0
    ico = _describe(wke, 3, 64, 2, 12, 20, precision=wke.WKE_FP32)   # icosahedron / dodecahedron
    assert ico.rule_products_available == 0
    n32 = _describe(wke, 3, 32, 4, 8, 8, precision=wke.WKE_FP32)
    assert n32.fused_products == 1 and n32.rule_products_available == 0   # the N = 64 kernel only
    # 2D mid-point 4 x 4: 8 distinct fields per radius, 1 product per group
    two_d = _describe(wke, 2, 128, 32, 4, 4, precision=wke.WKE_FP32)
    assert two_d.shared_fields == 1 and two_d.products_per_group == 1 and two_d.units_per_collision == 32 * 4


def test_fp32_chunks_fit_the_fused_kernel(wke):
    """3D FP32 plans chunk so that the fused axis-0 + product kernel holds a
    chunk's fields: at N = 48 (the 24 x 8 x 8 cube rule of the serving mix)
    two radii per chunk (52 fields) instead of three (78 fields, more shared
    memory than a block has), so the plan fuses; N = 32 keeps three radii and
    N = 64 one, and FP64 plans (no fused kernel) keep their own chunking."""
    n48 = _describe(wke, 3, 48, 24, 8, 8, precision=wke.WKE_FP32)
    assert n48.fused_products == 1 and n48.n_chunks == 12 and n48.groups_per_chunk == 16
    n32 = _describe(wke, 3, 32, 16, 8, 8, precision=wke.WKE_FP32)
    assert n32.fused_products == 1 and n32.n_chunks == 6 and n32.groups_per_chunk == 24
    n64 = _describe(wke, 3, 64, 32, 8, 8, precision=wke.WKE_FP32)
    assert n64.fused_products == 1 and n64.n_chunks == 32
    f64 = _describe(wke, 3, 48, 24, 8, 8, precision=wke.WKE_FP64)
    assert f64.fused_products == 0 and f64.n_chunks == 24


def test_autotuned_creation_checks_arguments_before_device_work(wke):
    """wke_plan_create_autotuned refuses a NULL out, a NULL f or Q, reps < 1
    and an invalid plan (M != n_r n_s n_sig) with WKE_ERR_INVALID before it
    creates any plan or touches a device; *out stays NULL."""
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = 2, 4, 4
    out = ctypes.c_void_p(1)
    fake = ctypes.c_void_p(16)        # never dereferenced on these paths
    lib = wke.lib()
    assert lib.wke_plan_create_autotuned(2, 16, 8.0, 32, ctypes.byref(q), fake, fake, None, 1, None, None,
                                         None) == wke.WKE_ERR_INVALID
    for f_ptr, q_ptr, reps, M in ((None, fake, 1, 32), (fake, None, 1, 32), (fake, fake, 0, 32),
                                  (fake, fake, 1, 33)):
        out.value = 1
        rc = lib.wke_plan_create_autotuned(2, 16, 8.0, M, ctypes.byref(q), f_ptr, q_ptr, None, reps,
                                           ctypes.byref(out), None, None)
        assert rc == wke.WKE_ERR_INVALID and not out.value
        assert lib.wke_last_error_string()


def test_describe_matches_footprint_and_rejects_like_create(wke):
    q = wke.wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = 4, 8, 8
    info = wke.wke_plan_describe(3, 32, 8.0, 256, q)
    assert info.device_bytes == wke.wke_plan_footprint_bytes(3, 32, 8.0, 256, q)
    info2 = wke.WkePlanInfo()
    assert wke.lib().wke_plan_describe(3, 128, 8.0, 256, ctypes.byref(q), ctypes.byref(info2)) == -4


LAYOUT_CASES = [
    # d, N, (n_r, n_s, n_sig), q-hat rule, sigma rule, precision, Nyquist modes
    (2, 128, (32, 4, 4), "midpoint", None, "fp32", "keep"),
    (2, 64, (6, 6, 6), "midpoint", None, "fp32", "zero"),
    (2, 32, (5, 5, 3), "midpoint", None, "fp64", "keep"),
    (3, 64, (32, 8, 8), "cube", None, "fp32", "keep"),
    (3, 32, (16, 8, 8), "cube", None, "fp64", "keep"),
    (3, 32, (2, 12, 20), "icosahedron", "dodecahedron", "fp32", "keep"),
    (3, 48, (6, 8, 8), "cube", None, "fp32", "zero"),
    (3, 16, (3, 8, 6), "cube", "product:2:3", "fp64", "keep"),
]


@pytest.mark.parametrize("d,N,n,sph,sph_sig,prec,nyq", LAYOUT_CASES)
def test_layout_invariants(wke, d, N, n, sph, sph_sig, prec, nyq):
    """Plan records from wke_plan_describe (host work only): shapes, the launch
    count of each layout, and the automatic choice of the shared-field layout
    exactly when it transforms at most 85% of the per-group layout's units."""
    M = n[0] * n[1] * n[2]

    def describe(layout):
        q = wke.wke_quadrature_default()
        q.n_r, q.n_s, q.n_sig = n
        q.sphere_rule, q.sphere_param = wke._rule(sph)
        if sph_sig is not None:
            q.sphere_rule_sig, q.sphere_param_sig = wke._rule(sph_sig)
        q.precision = {"fp64": wke.WKE_FP64, "fp32": wke.WKE_FP32}[prec]
        q.nyquist = {"keep": wke.WKE_NYQ_KEEP, "zero": wke.WKE_NYQ_ZERO}[nyq]
        q.layout = layout
        info = wke.WkePlanInfo()
        rc = wke.lib().wke_plan_describe(d, N, 8.0, M, ctypes.byref(q), ctypes.byref(info))
        return rc, info

    rc, per_group = describe(wke.WKE_LAYOUT_PER_GROUP)
    assert rc == 0
    rc, auto = describe(wke.WKE_LAYOUT_AUTO)
    assert rc == 0
    rc_shared, shared = describe(wke.WKE_LAYOUT_SHARED)
    for info in (per_group, auto) + ((shared,) if rc_shared == 0 else ()):
        assert (info.d, info.N, info.M) == (d, N, M)
        assert info.n_groups == n[0] * n[1]
        assert info.n_chunks >= 1 and info.units_per_collision >= 1 and info.device_bytes > 0
        # forward (one kernel per axis), per chunk pass 1 (+ Nyquist tables) and
        # pass 2, or axis 0 + products in the shared layout (one fused kernel in
        # 3D FP32), then finalize
        per_chunk = (3 if nyq == "keep" else 2) + (info.shared_fields and not info.fused_products)
        finalize = 0 if info.fused_products else 1
        assert info.launches_per_collision == d + per_chunk * info.n_chunks + finalize
        # fused only where it applies (3D FP32 shared); it may be declined when
        # the chunk's fields do not fit the kernel's shared memory
        assert not info.fused_products or (info.shared_fields and d == 3 and prec == "fp32")
        assert info.separable == 0 or (info.shared_fields and d == 3)
    assert per_group.shared_fields == 0
    rc_sep, sep = describe(wke.WKE_LAYOUT_SEPARABLE)
    if d == 2:
        assert rc_sep == wke.WKE_ERR_INVALID
    elif rc_sep == 0:
        # the same fields and units; the trailing axes once per row value and pair
        assert sep.separable == 1 and sep.shared_fields == 1
        assert sep.units_per_collision == shared.units_per_collision
        assert auto.separable == int(auto.shared_fields == 1 and sep.pair_planes_per_collision
                                     <= 0.85 * 2 * sep.units_per_collision)
    if rc_shared == 0:
        assert shared.shared_fields == 1
        pick = shared.units_per_collision <= 0.85 * per_group.units_per_collision
        assert auto.shared_fields == int(pick)
        chosen = shared if pick else per_group
        assert auto.units_per_collision == chosen.units_per_collision
        assert auto.n_chunks == chosen.n_chunks
    else:
        assert auto.shared_fields == 0


def test_checked_build_exports_every_symbol(wke):
    """The bounds-checked debug build (built beside the library) exports the
    same calls and says so in its version string."""
    if not os.path.exists(wke.CHECK_LIB_PATH):
        pytest.skip("checked build not present")
    lib = ctypes.CDLL(wke.CHECK_LIB_PATH)
    for name in wke.EXPORTED:
        assert hasattr(lib, name), name
    lib.wke_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in lib.wke_version()
    flags = ctypes.c_uint(7)
    # without a device the call either reports no failure or a CUDA error; it never aborts
    rc = lib.wke_check_status(ctypes.byref(flags))
    assert rc in (0, -3)
