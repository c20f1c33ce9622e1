"""Python binding of the C-ABI library ``libwke.so`` (ctypes).

Argument marshalling only: every step of the collision operator runs in the
library's CUDA kernels.  The functions keep the C names; ``Plan`` is a small
convenience wrapper that passes torch CUDA tensors' pointers and streams.
Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwke.so")

WKE_OK = 0
WKE_ERR_INVALID = -1
WKE_ERR_OOM = -2
WKE_ERR_CUDA = -3
WKE_ERR_UNSUPPORTED = -4
WKE_CANCELLED = -5

WKE_SPHERE_DEFAULT = -1
WKE_SPHERE_MIDPOINT_2D = 0
WKE_SPHERE_PLATONIC_3D = 1
WKE_SPHERE_PRODUCT_3D = 2
WKE_SPHERE_USER = 3

WKE_FP64 = 0
WKE_FP32 = 1
WKE_SPLIT = 2
WKE_NYQ_KEEP = 0
WKE_NYQ_ZERO = 1
WKE_ALIAS_CIRCULAR = 0
WKE_DEALIAS_PAD2 = 1
WKE_LAYOUT_AUTO = 0
WKE_LAYOUT_PER_GROUP = 1
WKE_LAYOUT_SHARED = 2
WKE_LAYOUT_SEPARABLE = 3
WKE_OMEGA_HALF_K2 = 0
WKE_OMEGA_K2 = 1

C_DOUBLE_P = ctypes.POINTER(ctypes.c_double)


class WkeQuadrature(ctypes.Structure):
    _fields_ = [
        ("n_r", ctypes.c_int), ("n_s", ctypes.c_int), ("n_sig", ctypes.c_int),
        ("sphere_rule", ctypes.c_int), ("sphere_rule_sig", ctypes.c_int),
        ("sphere_param", ctypes.c_int), ("sphere_param_sig", ctypes.c_int),
        ("user_s", C_DOUBLE_P), ("user_sig", C_DOUBLE_P),
        ("R", ctypes.c_double), ("precision", ctypes.c_int), ("nyquist", ctypes.c_int),
        ("dispersion", ctypes.c_int), ("pair_antipodal", ctypes.c_int),
        ("chunk_bytes", ctypes.c_size_t), ("alias", ctypes.c_int), ("layout", ctypes.c_int),
    ]


class WkeTuning(ctypes.Structure):
    _fields_ = [("pass2_points_per_thread", ctypes.c_int), ("pass1_units_per_block", ctypes.c_int),
                ("fuse_products", ctypes.c_int), ("forward_fp32", ctypes.c_int), ("rule_products", ctypes.c_int)]


class WkeRequest(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_int), ("L", ctypes.c_double),
                ("n_r", ctypes.c_int), ("n_s", ctypes.c_int), ("n_sig", ctypes.c_int),
                ("precision", ctypes.c_int), ("rk_stages", ctypes.c_int), ("steps", ctypes.c_int),
                ("dt", ctypes.c_double), ("f_host", ctypes.c_void_p), ("out_host", ctypes.c_void_p)]


class WkeRequestStats(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class WkePlanInfo(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("N", ctypes.c_int), ("M", ctypes.c_int), ("precision", ctypes.c_int),
        ("n_groups", ctypes.c_int), ("fields_per_group", ctypes.c_int),
        ("products_per_group", ctypes.c_int), ("groups_per_chunk", ctypes.c_int),
        ("n_chunks", ctypes.c_int), ("launches_per_collision", ctypes.c_int),
        ("flops_per_collision", ctypes.c_double), ("l2_bytes_per_collision", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t), ("N_compute", ctypes.c_int), ("shared_fields", ctypes.c_int),
        ("units_per_collision", ctypes.c_int), ("separable", ctypes.c_int),
        ("pair_planes_per_collision", ctypes.c_int), ("fused_products", ctypes.c_int),
        ("row_values_per_collision", ctypes.c_int), ("rule_products_available", ctypes.c_int),
    ]


EXPORTED = [
    "wke_quadrature_default", "wke_plan_create", "wke_plan_destroy", "wke_plan_footprint_bytes",
    "wke_plan_get_info", "wke_plan_describe", "wke_plan_node_table", "wke_collision", "wke_collision_ex",
    "wke_collision_host", "wke_collision_spectrum", "wke_plan_set_stream", "wke_step", "wke_moments",
    "wke_server_create", "wke_server_submit", "wke_server_cancel", "wke_server_wait", "wke_server_destroy",
    "wke_moments_noalloc", "wke_plan_get_tuning", "wke_plan_set_tuning", "wke_plan_autotune",
    "wke_plan_create_autotuned",
    "wke_plan_use_graphs", "wke_plan_profile", "wke_plan_profile_read", "wke_alu_peak", "wke_check_status",
    "wke_last_error_string", "wke_version",
]
CHECK_LIB_PATH = os.path.join(_HERE, "libwke_check.so")
PROF_CLASSES = ("forward", "pass1", "pass2", "finalize", "nyquist", "axis0")


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libwke.so is not built ({path}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    QP = ctypes.POINTER(WkeQuadrature)
    sig = {
        "wke_quadrature_default": (i, [QP]),
        "wke_plan_create": (i, [i, i, d, i, QP, ctypes.POINTER(vp)]),
        "wke_plan_destroy": (i, [vp]),
        "wke_plan_footprint_bytes": (i, [i, i, d, i, QP, ctypes.POINTER(sz)]),
        "wke_plan_get_info": (i, [vp, ctypes.POINTER(WkePlanInfo)]),
        "wke_plan_describe": (i, [i, i, d, i, QP, ctypes.POINTER(WkePlanInfo)]),
        "wke_plan_node_table": (i, [vp, C_DOUBLE_P]),
        "wke_collision": (i, [vp, vp, vp, vp]),
        "wke_collision_ex": (i, [vp, vp, vp, vp, vp]),
        "wke_collision_host": (i, [vp, vp, vp]),
        "wke_collision_spectrum": (i, [vp, vp, vp, vp, vp]),
        "wke_plan_set_stream": (i, [vp, vp]),
        "wke_step": (i, [vp, vp, d, i]),
        "wke_moments": (i, [vp, vp, vp, vp]),
        "wke_moments_noalloc": (i, [i, i, d, i, vp, vp, vp]),
        "wke_server_create": (i, [sz, i, ctypes.POINTER(vp)]),
        "wke_server_submit": (i, [vp, ctypes.POINTER(WkeRequest), ctypes.POINTER(ctypes.c_longlong)]),
        "wke_server_cancel": (i, [vp, ctypes.c_longlong]),
        "wke_server_wait": (i, [vp, ctypes.c_longlong, d, ctypes.POINTER(WkeRequestStats)]),
        "wke_server_destroy": (i, [vp]),
        "wke_plan_get_tuning": (i, [vp, ctypes.POINTER(WkeTuning)]),
        "wke_plan_set_tuning": (i, [vp, ctypes.POINTER(WkeTuning)]),
        "wke_plan_autotune": (i, [vp, vp, vp, i, ctypes.POINTER(WkeTuning), ctypes.POINTER(ctypes.c_double)]),
        "wke_plan_create_autotuned": (i, [i, i, d, i, QP, vp, vp, vp, i, ctypes.POINTER(vp), ctypes.POINTER(i),
                                          ctypes.POINTER(ctypes.c_double)]),
        "wke_plan_use_graphs": (i, [vp, i]),
        "wke_plan_profile": (i, [vp, i]),
        "wke_plan_profile_read": (i, [vp, C_DOUBLE_P]),
        "wke_alu_peak": (i, [i, i, C_DOUBLE_P, C_DOUBLE_P]),
        "wke_check_status": (i, [ctypes.POINTER(ctypes.c_uint)]),
        "wke_last_error_string": (ctypes.c_char_p, []),
        "wke_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class WkeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wke error {code}: {msg}")
        self.code = code


def _check(rc: int) -> None:
    if rc != WKE_OK:
        raise WkeError(rc, lib().wke_last_error_string().decode())


# ------------------------------------------------------------ C-named calls

def wke_quadrature_default() -> WkeQuadrature:
    q = WkeQuadrature()
    _check(lib().wke_quadrature_default(ctypes.byref(q)))
    return q


def wke_plan_create(d: int, N: int, L: float, M: int, quad: WkeQuadrature) -> ctypes.c_void_p:
    out = ctypes.c_void_p()
    _check(lib().wke_plan_create(d, N, L, M, ctypes.byref(quad), ctypes.byref(out)))
    return out


def wke_plan_destroy(plan) -> None:
    _check(lib().wke_plan_destroy(plan))


def wke_plan_footprint_bytes(d: int, N: int, L: float, M: int, quad: WkeQuadrature) -> int:
    out = ctypes.c_size_t()
    _check(lib().wke_plan_footprint_bytes(d, N, L, M, ctypes.byref(quad), ctypes.byref(out)))
    return out.value


def wke_plan_get_info(plan) -> WkePlanInfo:
    info = WkePlanInfo()
    _check(lib().wke_plan_get_info(plan, ctypes.byref(info)))
    return info


def wke_plan_describe(d: int, N: int, L: float, M: int, quad: WkeQuadrature) -> WkePlanInfo:
    info = WkePlanInfo()
    _check(lib().wke_plan_describe(d, N, L, M, ctypes.byref(quad), ctypes.byref(info)))
    return info


def wke_collision(plan, f_ptr: int, Q_ptr: int, stream: int = 0) -> None:
    _check(lib().wke_collision(plan, f_ptr, Q_ptr, stream))


def wke_collision_ex(plan, f_ptr: int, Q_ptr: int, Qim_ptr: int | None, stream: int = 0) -> None:
    _check(lib().wke_collision_ex(plan, f_ptr, Q_ptr, Qim_ptr, stream))


def wke_collision_spectrum(plan, f_ptr: int, Q_ptr: int, Qhat_ptr: int, stream: int = 0) -> None:
    _check(lib().wke_collision_spectrum(plan, f_ptr, Q_ptr, Qhat_ptr, stream))


def wke_collision_host(plan, f_host_ptr: int, Q_host_ptr: int) -> None:
    _check(lib().wke_collision_host(plan, f_host_ptr, Q_host_ptr))


def wke_plan_set_stream(plan, stream: int) -> None:
    _check(lib().wke_plan_set_stream(plan, stream))


def wke_step(plan, f_ptr: int, dt: float, rk_stages: int) -> None:
    _check(lib().wke_step(plan, f_ptr, dt, rk_stages))


def wke_moments(plan, g_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(lib().wke_moments(plan, g_ptr, out_ptr, stream))


def wke_moments_noalloc(d: int, N: int, L: float, precision: int, g_ptr: int, out_ptr: int,
                        stream: int = 0) -> None:
    """Plan-free moments for callers that cannot allocate device memory; the
    partial sums live in a fixed array inside the library (see wke.h)."""
    _check(lib().wke_moments_noalloc(d, N, L, precision, g_ptr, out_ptr, stream))


def wke_plan_get_tuning(plan) -> WkeTuning:
    t = WkeTuning()
    _check(lib().wke_plan_get_tuning(plan, ctypes.byref(t)))
    return t


def wke_plan_set_tuning(plan, pass2_points_per_thread: int, pass1_units_per_block: int = 0,
                        fuse_products: int | None = None, forward_fp32: int | None = None,
                        rule_products: int | None = None) -> None:
    """Set the launch layout; fuse_products / forward_fp32 / rule_products None keep the plan's
    current choice (rule_products: the plan's rule schedule whenever the products are fused)."""
    cur = wke_plan_get_tuning(plan)
    if fuse_products is None:
        fuse_products = cur.fuse_products
    if forward_fp32 is None:
        forward_fp32 = cur.forward_fp32
    if rule_products is None:
        if cur.fuse_products and fuse_products:
            rule_products = cur.rule_products
        else:
            rule_products = 1 if fuse_products and wke_plan_get_info(plan).rule_products_available else 0
    t = WkeTuning(pass2_points_per_thread, pass1_units_per_block, fuse_products, forward_fp32, rule_products)
    _check(lib().wke_plan_set_tuning(plan, ctypes.byref(t)))


def wke_plan_autotune(plan, f_ptr: int, Q_ptr: int, reps: int = 5):
    """Time the candidate layouts on this plan and keep the fastest;
    returns (tuning, ms per evaluation)."""
    t = WkeTuning()
    ms = ctypes.c_double()
    _check(lib().wke_plan_autotune(plan, f_ptr, Q_ptr, reps, ctypes.byref(t), ctypes.byref(ms)))
    return t, ms.value


def wke_plan_create_autotuned(d: int, N: int, L: float, M: int, quad: WkeQuadrature, f_ptr: int, Q_ptr: int,
                              stream: int | None = None, reps: int = 3):
    """Create the plan whose pencil and launch layouts time fastest on f;
    returns (plan handle, layout, ms per evaluation)."""
    out = ctypes.c_void_p()
    lay = ctypes.c_int()
    ms = ctypes.c_double()
    _check(lib().wke_plan_create_autotuned(d, N, L, M, ctypes.byref(quad), f_ptr, Q_ptr, stream, reps,
                                           ctypes.byref(out), ctypes.byref(lay), ctypes.byref(ms)))
    return out, lay.value, ms.value


def wke_plan_use_graphs(plan, enable: bool) -> None:
    _check(lib().wke_plan_use_graphs(plan, int(enable)))


def wke_plan_profile(plan, enable: bool) -> None:
    _check(lib().wke_plan_profile(plan, int(enable)))


def wke_plan_profile_read(plan) -> dict:
    """{class: (total_ms, launches)} recorded since profiling was enabled."""
    out = (ctypes.c_double * (2 * len(PROF_CLASSES)))()
    _check(lib().wke_plan_profile_read(plan, out))
    return {c: (out[2 * i], int(out[2 * i + 1])) for i, c in enumerate(PROF_CLASSES)}


def wke_alu_peak(precision: int, reps: int = 5):
    """Measured FMA throughput of the current device: (TFLOP/s, ms of the best launch)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().wke_alu_peak(precision, reps, ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def wke_check_status() -> int:
    """Bounds-check bits of the checked build since the last call (0 in the
    default build); raises WkeError when any is set."""
    flags = ctypes.c_uint(0)
    rc = lib().wke_check_status(ctypes.byref(flags))
    if rc != WKE_OK and flags.value == 0:
        _check(rc)
    return flags.value


def use_library(path: str) -> ctypes.CDLL:
    """Load another build of the library (e.g. CHECK_LIB_PATH) for the calls
    of this module; returns the previous handle for restore_library."""
    global _lib
    prev = _lib if _lib is not None else lib()
    _lib = load_library(path)
    return prev


def restore_library(handle: ctypes.CDLL) -> None:
    global _lib
    _lib = handle


def wke_server_create(device_budget_bytes: int, max_active: int):
    out = ctypes.c_void_p()
    _check(lib().wke_server_create(device_budget_bytes, max_active, ctypes.byref(out)))
    return out


def wke_server_submit(server, request: WkeRequest) -> int:
    rid = ctypes.c_longlong()
    _check(lib().wke_server_submit(server, ctypes.byref(request), ctypes.byref(rid)))
    return rid.value


def wke_server_cancel(server, rid: int) -> None:
    _check(lib().wke_server_cancel(server, rid))


def wke_server_wait(server, rid: int, timeout_s: float = -1.0) -> WkeRequestStats:
    st = WkeRequestStats()
    _check(lib().wke_server_wait(server, rid, timeout_s, ctypes.byref(st)))
    return st


def wke_server_destroy(server) -> None:
    _check(lib().wke_server_destroy(server))


class Server:
    """Continuous-batching server; requests carry numpy host arrays."""

    def __init__(self, device_budget_bytes: int, max_active: int = 8):
        self.handle = wke_server_create(device_budget_bytes, max_active)
        self._keep = {}

    def submit(self, f, n_r, n_s, n_sig, steps, dt, L=8.0, rk_stages=4, precision="fp32"):
        """Queue f (numpy, shape (N,)*d, float32 or float64 per precision);
        returns (request id, output array filled on completion)."""
        import numpy as np
        dtype = np.float32 if precision == "fp32" else np.float64
        f = np.ascontiguousarray(f, dtype=dtype)
        out = np.empty_like(f)
        req = WkeRequest(f.ndim, f.shape[0], L, n_r, n_s, n_sig,
                         WKE_FP32 if precision == "fp32" else WKE_FP64, rk_stages, steps, dt,
                         f.ctypes.data, out.ctypes.data)
        rid = wke_server_submit(self.handle, req)
        self._keep[rid] = (f, out)
        return rid, out

    def cancel(self, rid: int) -> None:
        wke_server_cancel(self.handle, rid)

    def wait(self, rid: int, timeout_s: float = -1.0) -> WkeRequestStats:
        st = wke_server_wait(self.handle, rid, timeout_s)
        self._keep.pop(rid, None)
        return st

    def close(self):
        if getattr(self, "handle", None):
            wke_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ torch helper

SPHERE_NAMES = {"midpoint": WKE_SPHERE_MIDPOINT_2D, "platonic": WKE_SPHERE_PLATONIC_3D,
                "cube": WKE_SPHERE_PLATONIC_3D, "octahedron": WKE_SPHERE_PLATONIC_3D,
                "icosahedron": WKE_SPHERE_PLATONIC_3D, "dodecahedron": WKE_SPHERE_PLATONIC_3D}


def _rule(name: str | None):
    """(rule, param) for a rule name; 'product:nt:nphi' gives the product rule."""
    if name is None:
        return WKE_SPHERE_DEFAULT, 0
    if name.startswith("product:"):
        return WKE_SPHERE_PRODUCT_3D, int(name.split(":")[1])
    return SPHERE_NAMES[name], 0


LAYOUT_NAMES = {"auto": WKE_LAYOUT_AUTO, "per_group": WKE_LAYOUT_PER_GROUP, "shared": WKE_LAYOUT_SHARED,
                "separable": WKE_LAYOUT_SEPARABLE}


def _quadrature(n_r, n_s, n_sig, sphere, sphere_sig, R, precision, nyquist, pair_antipodal, chunk_bytes,
                dispersion, user_s, user_sig, dealias, layout):
    """The wke_quadrature descriptor of Plan's keywords, and the arrays its
    user rules point into (to be kept alive with it)."""
    import numpy as np
    q = wke_quadrature_default()
    q.n_r, q.n_s, q.n_sig = n_r, n_s, n_sig
    q.sphere_rule, q.sphere_param = _rule(sphere)
    if sphere_sig is not None:
        q.sphere_rule_sig, q.sphere_param_sig = _rule(sphere_sig)
    keep = []
    if user_s is not None:
        arr = np.ascontiguousarray(user_s, dtype=np.float64)
        keep.append(arr)
        q.sphere_rule = WKE_SPHERE_USER
        q.user_s = arr.ctypes.data_as(C_DOUBLE_P)
    if user_sig is not None:
        arr = np.ascontiguousarray(user_sig, dtype=np.float64)
        keep.append(arr)
        q.sphere_rule_sig = WKE_SPHERE_USER
        q.user_sig = arr.ctypes.data_as(C_DOUBLE_P)
    q.R = R
    q.precision = {"fp64": WKE_FP64, "fp32": WKE_FP32, "split": WKE_SPLIT}[precision]
    q.nyquist = {"keep": WKE_NYQ_KEEP, "zero": WKE_NYQ_ZERO}[nyquist]
    q.dispersion = {"half_k2": WKE_OMEGA_HALF_K2, "k2": WKE_OMEGA_K2}[dispersion]
    q.pair_antipodal = int(pair_antipodal)
    q.chunk_bytes = chunk_bytes
    q.alias = WKE_DEALIAS_PAD2 if dealias else WKE_ALIAS_CIRCULAR
    q.layout = LAYOUT_NAMES[layout]
    return q, keep


class Plan:
    """A plan on the current CUDA device; tensors are torch CUDA tensors."""

    def __init__(self, d: int, N: int, L: float, n_r: int, n_s: int, n_sig: int,
                 sphere: str | None = None, sphere_sig: str | None = None, R: float = 0.0,
                 precision: str = "fp64", nyquist: str = "keep", pair_antipodal: bool = True,
                 chunk_bytes: int = 0, dispersion: str = "half_k2", user_s=None, user_sig=None,
                 dealias: bool = False, layout: str = "auto", _handle=None):
        q, self._keep = _quadrature(n_r, n_s, n_sig, sphere, sphere_sig, R, precision, nyquist, pair_antipodal,
                                    chunk_bytes, dispersion, user_s, user_sig, dealias, layout)
        self.d, self.N, self.L = d, N, L
        self.M = n_r * n_s * n_sig
        self.precision = precision
        self.quad = q                      # the descriptor (its user rules are kept alive above)
        self.layout = None                 # set by Plan.autotuned
        self.handle = wke_plan_create(d, N, L, self.M, q) if _handle is None else _handle

    @classmethod
    def autotuned(cls, f, d: int, N: int, L: float, n_r: int, n_s: int, n_sig: int, reps: int = 3, **kw):
        """The plan whose pencil layout (separable, shared or per-group) and
        launch layout time fastest on f (a CUDA tensor of the plan's grid
        and precision), through wke_plan_create_autotuned; the keywords are
        those of Plan.  Returns (plan, ms per evaluation)."""
        import torch
        prec = kw.get("precision", "fp64")
        dt = torch.float64 if prec == "fp64" else torch.float32
        if not (f.is_cuda and f.dtype == dt and f.is_contiguous() and tuple(f.shape) == (N,) * d):
            raise ValueError(f"expected a contiguous CUDA {dt} tensor of shape {(N,) * d}")
        q, keep = _quadrature(n_r, n_s, n_sig, kw.get("sphere"), kw.get("sphere_sig"), kw.get("R", 0.0), prec,
                              kw.get("nyquist", "keep"), kw.get("pair_antipodal", True), kw.get("chunk_bytes", 0),
                              kw.get("dispersion", "half_k2"), kw.get("user_s"), kw.get("user_sig"),
                              kw.get("dealias", False), kw.get("layout", "auto"))
        Q = torch.empty_like(f)
        h, lay, ms = wke_plan_create_autotuned(d, N, L, n_r * n_s * n_sig, q, f.data_ptr(), Q.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream, reps)
        plan = cls(d, N, L, n_r, n_s, n_sig, _handle=h, **kw)
        plan._keep += keep
        plan.layout = {v: k for k, v in LAYOUT_NAMES.items()}[lay]
        return plan, ms

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def info(self) -> WkePlanInfo:
        return wke_plan_get_info(self.handle)

    def node_table(self):
        import numpy as np
        out = np.zeros((self.M, 1 + 3 * self.d), dtype=np.float64)
        _check(lib().wke_plan_node_table(self.handle, out.ctypes.data_as(C_DOUBLE_P)))
        return out

    def _check_grid(self, t):
        import torch
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()
                and tuple(t.shape) == (self.N,) * self.d):
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor of shape {(self.N,) * self.d}")
        return t

    def collision(self, f, Q=None, Qim=None, stream=None):
        import torch
        self._check_grid(f)
        if Q is None:
            Q = torch.empty_like(f)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        wke_collision_ex(self.handle, f.data_ptr(), self._check_grid(Q).data_ptr(),
                         None if Qim is None else self._check_grid(Qim).data_ptr(), s)
        return Q

    def spectrum(self, f, Q=None, Qhat=None, stream=None):
        """Q and its Fourier coefficients Qhat (complex, DFT order; see
        wke_collision_spectrum).  Returns (Q, Qhat)."""
        import torch
        self._check_grid(f)
        if Q is None:
            Q = torch.empty_like(f)
        cdt = torch.complex128 if self.precision == "fp64" else torch.complex64
        if Qhat is None:
            Qhat = torch.empty((self.N,) * self.d, dtype=cdt, device=f.device)
        if not (Qhat.is_cuda and Qhat.dtype == cdt and Qhat.is_contiguous() and tuple(Qhat.shape) == (self.N,) * self.d):
            raise ValueError(f"expected a contiguous CUDA {cdt} tensor of shape {(self.N,) * self.d}")
        s = (stream or torch.cuda.current_stream()).cuda_stream
        wke_collision_spectrum(self.handle, f.data_ptr(), self._check_grid(Q).data_ptr(), Qhat.data_ptr(), s)
        return Q, Qhat

    def step(self, f, dt: float, rk_stages: int = 4, stream=None):
        import torch
        self._check_grid(f)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        wke_plan_set_stream(self.handle, s)
        wke_step(self.handle, f.data_ptr(), dt, rk_stages)
        return f

    def moments(self, g, stream=None):
        import torch
        self._check_grid(g)
        out = torch.empty(self.d + 2, dtype=torch.float64, device=g.device)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        wke_moments(self.handle, g.data_ptr(), out.data_ptr(), s)
        return out

    def autotune(self, f, reps: int = 5):
        """Pick the fastest launch layout for this plan on input f."""
        import torch
        self._check_grid(f)
        Q = torch.empty_like(f)
        wke_plan_set_stream(self.handle, torch.cuda.current_stream().cuda_stream)
        return wke_plan_autotune(self.handle, f.data_ptr(), Q.data_ptr(), reps)

    def collision_host(self, f_host, Q_host):
        """f_host, Q_host: CPU tensors (pinned for full bandwidth) of the plan dtype."""
        wke_collision_host(self.handle, f_host.data_ptr(), Q_host.data_ptr())
        return Q_host

    def close(self):
        if getattr(self, "handle", None):
            wke_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
