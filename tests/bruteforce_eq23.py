"""Brute-force quadrature of the collision operator in its original form.

Independent of the oracle: it starts from the resonant-manifold integral of
Eq. (2.3) (omega = |k|^2/2, beta = 0), not from the spherical form the paper
derives in Appendix A.  With k3 = k - k1 + k2 from the momentum delta, the
frequency mismatch is (|k1|^2 - |k2|^2 + |k3|^2 - |k|^2)/2 = (k1-k2).(k1-k).
Substituting u = k1 - k, v = k1 - k2 (unit Jacobian) and resolving
delta(u.v) on the hyperplane orthogonal to u gives

    K(k) = int_{R^d} du/|u| int_{v perp u} dv
           [f1 f2 f3 - f f2 f3 + f1 f f3 - f1 f2 f],
    k1 = k + u,  k2 = k + u - v,  k3 = k - v.

In 2D: u = rho (cos t, sin t), v = s (-sin t, cos t), du/|u| = drho dt.
In 3D: u = rho w (w on S^2), v = s (cos p e1 + sin p e2), du/|u| = rho drho dw,
dv = s ds dp.  Tensor Gauss-Legendre / trapezoid rules; f must decay fast.
"""
import math

import numpy as np


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * (x + 1.0) + a, 0.5 * (b - a) * w


def _bracket(f, k, k1, k2, k3):
    f0, f1, f2, f3 = f(k), f(k1), f(k2), f(k3)
    return f1 * f2 * f3 - f0 * f2 * f3 + f1 * f0 * f3 - f1 * f2 * f0


def collision_2d(f, k, n_rho=48, n_t=64, n_s=64, rho_max=9.0, s_max=9.0):
    k = np.asarray(k, dtype=np.float64)
    rho, w_rho = _gl(n_rho, 0.0, rho_max)
    t = (np.arange(n_t) + 0.5) * (2.0 * math.pi / n_t)
    s, w_s = _gl(n_s, -s_max, s_max)
    RH, T, S = np.meshgrid(rho, t, s, indexing="ij")
    u = np.stack([RH * np.cos(T), RH * np.sin(T)], axis=-1)
    v = np.stack([-S * np.sin(T), S * np.cos(T)], axis=-1)
    val = _bracket(f, k, k + u, k + u - v, k - v)
    w = w_rho[:, None, None] * (2.0 * math.pi / n_t) * w_s[None, None, :]
    return float(np.sum(w * val))


def collision_3d(f, k, n_rho=32, n_ct=24, n_ph=48, n_s=32, n_p=32, rho_max=9.0, s_max=9.0):
    k = np.asarray(k, dtype=np.float64)
    rho, w_rho = _gl(n_rho, 0.0, rho_max)
    ct, w_ct = np.polynomial.legendre.leggauss(n_ct)
    ph = (np.arange(n_ph) + 0.5) * (2.0 * math.pi / n_ph)
    s, w_s = _gl(n_s, 0.0, s_max)
    p = (np.arange(n_p) + 0.5) * (2.0 * math.pi / n_p)
    st = np.sqrt(1.0 - ct * ct)
    om = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)),
                   np.outer(ct, np.ones(n_ph))], axis=-1).reshape(-1, 3)
    w_om = np.outer(w_ct, np.full(n_ph, 2.0 * math.pi / n_ph)).reshape(-1)
    ref = np.where(np.abs(om[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(om, ref)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(om, e1)
    w = (w_rho * rho)[:, None, None] * (w_s * s)[None, :, None] * (2.0 * math.pi / n_p)
    total = 0.0
    cp = np.cos(p)[None, None, :, None]
    sp = np.sin(p)[None, None, :, None]
    for i in range(len(om)):
        u = rho[:, None, None, None] * om[i]
        v = s[None, :, None, None] * (cp * e1[i] + sp * e2[i])
        total += w_om[i] * np.sum(w * _bracket(f, k, k + u, k + u - v, k - v))
    return float(total)
