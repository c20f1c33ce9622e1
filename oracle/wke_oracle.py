"""CPU FP64 oracle for the 4-wave kinetic collision operator.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.  It shares no
code with the CUDA path (only the seeded generators of ``wke_inputs``).

It follows Qi, Shen and Wang, "A fast Fourier spectral method for wave
kinetic equation" (arXiv 2503.12805), for the Schroedinger dispersion
omega = |k|^2/2 with beta = 0 (Sec. 2, Eq. (2.3)) in its Boltzmann-type
spherical form (Eq. (2.7)-(2.8)):

    K(f)(k) = 2^{1-d} int_{B_R} int_{S^{d-1}} |q|^{d-2}
              [f(k') f(k-q) f(k2') - f(k) f(k-q) f(k2') + f(k') f(k) f(k2')
               - f(k') f(k-q) f(k)] dsigma dq,
    k' = k - (q - |q| sigma)/2,  k2' = k - (q + |q| sigma)/2      (Sec. 3.2).

Evaluators:
  * ``collision_alg1``    Algorithm 1 step by step (Fourier-space accumulation
                           of the four terms, final inverse transform).
  * ``collision_fast``    the same sum with the FFT / inverse-FFT round trips
                           of Algorithm 1 removed by linearity: every term is
                           accumulated on the grid (the form the GPU computes).
  * ``collision_direct``  the classical spectral sums Eqs. (3.3)-(3.6) with
                           the quadrature weights of Eq. (3.8) (or the exact
                           weights), O(N^{3d}); circular or linear index sums.
  * ``collision_realspace`` the quadrature of Eq. (2.7) with an analytic f.
  * ``collision_at_points`` ``collision_fast`` at chosen grid points only, by
                           direct evaluation of the truncated series (3.1).
  * ``collision_dealiased`` the linear-sum (de-aliased) counterpart of
                           ``collision_fast`` through 2N zero padding.

Readings of the paper where it is silent or ambiguous (all listed in the
design notes): grid k_i = -L + i 2L/N; coefficients by the rectangle rule
N^{-d} sum_i; the Nyquist modes j_c = -N/2 are kept (the mode range of Eq.
(3.1)), so shifted fields are complex and the output is Re Q with max|Im Q|
reported; products of N-point transforms are circular (aliased) as in
Algorithm 1; R = 4L/(3+sqrt 2) by default (R = 2S, L = (3+sqrt 2)S/2, Step 1);
the K3/K4 weights are w_r |q|^{2d-3} like K1/K2; the sigma-phase of
Algorithm 1's gamma-tilde uses sigma as in Eq. (3.8).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Sequence

import numpy as np
import scipy.special

# ----------------------------------------------------------------------------
# Step 1-2: grid, modes, coefficients (Sec. 3.2, Eq. (3.1))
# ----------------------------------------------------------------------------


def default_R(L: float) -> float:
    """R = 2S with S the largest support radius allowed by L >= (3+sqrt2)S/2
    (Sec. 3.2, Step 1)."""
    return 4.0 * L / (3.0 + math.sqrt(2.0))


def grid_1d(N: int, L: float) -> np.ndarray:
    """k_i = -L + i h, h = 2L/N, i = 0..N-1."""
    return -L + np.arange(N, dtype=np.float64) * (2.0 * L / N)


def grid_points(d: int, N: int, L: float) -> np.ndarray:
    """All grid points, shape (N,)*d + (d,)."""
    return np.stack(np.meshgrid(*([grid_1d(N, L)] * d), indexing="ij"), axis=-1)


def modes_1d(N: int) -> np.ndarray:
    """Signed mode number j in [-N/2, N/2-1] stored at DFT position j mod N."""
    return np.fft.fftfreq(N, d=1.0 / N).round().astype(np.int64)


def mode_vectors(d: int, N: int) -> np.ndarray:
    """Signed mode vectors at every DFT position, shape (N,)*d + (d,)."""
    return np.stack(np.meshgrid(*([modes_1d(N)] * d), indexing="ij"), axis=-1)


def _alternating_sign(d: int, N: int) -> np.ndarray:
    """(-1)^{j_1+...+j_d}: the factor exp(-i pi j.(-L)/L) from the grid's
    first point k_0 = -L."""
    s1 = np.where(modes_1d(N) % 2 == 0, 1.0, -1.0)
    out = s1
    for _ in range(d - 1):
        out = np.multiply.outer(out, s1)
    return out


def FFT(g: np.ndarray, L: float) -> np.ndarray:
    """Fourier coefficients of grid values, Eq. (3.1) with the integral
    (2L)^{-d} int_{D_L} replaced by the periodic rectangle rule:
    hat g_j = N^{-d} sum_i g_i exp(-i pi j.k_i / L), j in [-N/2, N/2-1]^d."""
    d, N = g.ndim, g.shape[0]
    return np.fft.fftn(g) / float(N ** d) * _alternating_sign(d, N)


def iFFT(ghat: np.ndarray, L: float) -> np.ndarray:
    """The truncated series of Eq. (3.1) on the grid:
    g(k_i) = sum_j hat g_j exp(i pi j.k_i / L)."""
    d, N = ghat.ndim, ghat.shape[0]
    return np.fft.ifftn(ghat * _alternating_sign(d, N)) * float(N ** d)


def phase(d: int, N: int, L: float, x: np.ndarray, sign: float = -1.0) -> np.ndarray:
    """exp(sign * i pi j.x / L) at every mode j (DFT positions)."""
    j = mode_vectors(d, N).astype(np.float64)
    return np.exp(sign * 1j * math.pi / L * (j @ np.asarray(x, dtype=np.float64)))


# ----------------------------------------------------------------------------
# Step 4: quadrature (Sec. 3.3, Eq. (3.8))
# ----------------------------------------------------------------------------


def radial_gauss_legendre(n_r: int, R: float):
    """Gauss-Legendre nodes |q|_{p1} and weights w_r on [0, R]."""
    x, w = np.polynomial.legendre.leggauss(n_r)
    return 0.5 * R * (x + 1.0), 0.5 * R * w


def circle_midpoint(n: int):
    """Mid-point rule on S^1: theta_p = (p - 1/2) 2 pi / n, weight 2 pi / n."""
    th = (np.arange(n, dtype=np.float64) + 0.5) * (2.0 * math.pi / n)
    return np.stack([np.cos(th), np.sin(th)], axis=-1), np.full(n, 2.0 * math.pi / n)


def _normalise(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _cyclic(triples):
    out = []
    for a, b, c in triples:
        out += [(a, b, c), (c, a, b), (b, c, a)]
    return out


def sphere_platonic(n: int):
    """Equal-weight spherical designs from the Platonic solids' vertices:
    octahedron (6, a 3-design), cube (8, 3-design), icosahedron (12,
    5-design), dodecahedron (20, 5-design).  Weight 4 pi / n each."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    if n == 6:
        pts = [(s, 0, 0) for s in (1, -1)] + [(0, s, 0) for s in (1, -1)] + \
              [(0, 0, s) for s in (1, -1)]
    elif n == 8:
        pts = [(a, b, c) for a in (1, -1) for b in (1, -1) for c in (1, -1)]
    elif n == 12:
        pts = _cyclic([(0, a, b * phi) for a in (1, -1) for b in (1, -1)])
    elif n == 20:
        pts = [(a, b, c) for a in (1, -1) for b in (1, -1) for c in (1, -1)]
        pts += _cyclic([(0, a / phi, b * phi) for a in (1, -1) for b in (1, -1)])
    else:
        raise ValueError(f"no Platonic design with {n} points")
    return _normalise(pts), np.full(n, 4.0 * math.pi / n)


def sphere_product(n_theta: int, n_phi: int):
    """Product rule on S^2: Gauss-Legendre in cos(theta) x mid-point in phi."""
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    ph = (np.arange(n_phi, dtype=np.float64) + 0.5) * (2.0 * math.pi / n_phi)
    st = np.sqrt(1.0 - ct * ct)
    pts = np.stack([np.outer(st, np.cos(ph)), np.outer(st, np.sin(ph)),
                    np.outer(ct, np.ones(n_phi))], axis=-1).reshape(-1, 3)
    w = np.outer(wt, np.full(n_phi, 2.0 * math.pi / n_phi)).reshape(-1)
    return pts, w


def sphere_rule(d: int, n: int, kind: str):
    """Directions (n, d) and weights (n,) on S^{d-1}."""
    if d == 2:
        if kind != "midpoint":
            raise ValueError("2D uses the mid-point rule")
        return circle_midpoint(n)
    if kind in ("platonic", "cube", "octahedron", "icosahedron", "dodecahedron"):
        want = {"cube": 8, "octahedron": 6, "icosahedron": 12, "dodecahedron": 20}.get(kind, n)
        if want != n:
            raise ValueError(f"{kind} has {want} points, not {n}")
        return sphere_platonic(n)
    if kind.startswith("product:"):
        nt, nph = (int(x) for x in kind.split(":")[1:])
        if nt * nph != n:
            raise ValueError("product rule size mismatch")
        return sphere_product(nt, nph)
    raise ValueError(f"unknown sphere rule {kind!r}")


@dataclasses.dataclass
class Quadrature:
    """Nodes and weights of Eq. (3.8): radial |q|_{p1}, w_r; directions
    qhat_{p2}, w_s; collision angles sigma_{p3}, w_sig."""
    d: int
    R: float
    r: np.ndarray
    w_r: np.ndarray
    qhat: np.ndarray
    w_s: np.ndarray
    sig: np.ndarray
    w_sig: np.ndarray

    @property
    def n_r(self):
        return len(self.r)

    @property
    def n_s(self):
        return len(self.w_s)

    @property
    def n_sig(self):
        return len(self.w_sig)

    @property
    def M(self):
        return self.n_r * self.n_s * self.n_sig

    def nodes(self):
        """Yield (p1, p2, p3, W, c, a, b) in lexicographic order, with
        W = w_r |q|^{2d-3} w_s w_sig (Eq. (3.8)), c = q = |q| qhat,
        a = (q - |q| sigma)/2, b = (q + |q| sigma)/2 so that
        k' = k - a and k2' = k - b (Sec. 3.2)."""
        d = self.d
        for p1 in range(self.n_r):
            r = self.r[p1]
            for p2 in range(self.n_s):
                q = r * self.qhat[p2]
                for p3 in range(self.n_sig):
                    s = r * self.sig[p3]
                    W = self.w_r[p1] * r ** (2 * d - 3) * self.w_s[p2] * self.w_sig[p3]
                    yield p1, p2, p3, W, q, 0.5 * (q - s), 0.5 * (q + s)


def make_quadrature(d: int, n_r: int, n_s: int, n_sig: int, R: float,
                    sphere: str = "midpoint", sphere_sig: str | None = None) -> Quadrature:
    r, w_r = radial_gauss_legendre(n_r, R)
    qhat, w_s = sphere_rule(d, n_s, sphere)
    sig, w_sig = sphere_rule(d, n_sig, sphere_sig or sphere)
    return Quadrature(d, R, r, w_r, qhat, w_s, sig, w_sig)


# ----------------------------------------------------------------------------
# Algorithm 1, literally (Sec. 3.4)
# ----------------------------------------------------------------------------


def collision_alg1(f: np.ndarray, L: float, quad: Quadrature, nyquist: str = "keep"):
    """Algorithm 1: for every node, the weighted spectra, inverse transforms,
    inner convolution FFT(g_l g_n), outer convolution FFT(f_m iFFT(.)), and
    accumulation of hat K_1..hat K_4 with weight w_r |q|^{2d-3} w_s w_sig;
    then hat K = 2^{1-d}(hat K_1 - hat K_2 + hat K_3 - hat K_4) and
    K = iFFT(hat K).  Returns (Re K, max |Im K|)."""
    d, N = f.ndim, f.shape[0]
    fhat = _apply_nyquist(FFT(f, L), nyquist)
    f0 = iFFT(fhat, L)                        # the unweighted field (K2, K3, K4)
    jv = mode_vectors(d, N).astype(np.float64)
    K1 = np.zeros_like(fhat)
    K2 = np.zeros_like(fhat)
    K3 = np.zeros_like(fhat)
    K4 = np.zeros_like(fhat)
    for p1 in range(quad.n_r):
        r = quad.r[p1]
        for p2 in range(quad.n_s):
            qh = quad.qhat[p2]
            alpha = np.exp(-1j * math.pi / L * r * (jv @ qh))
            beta = np.exp(-1j * math.pi / (2 * L) * r * (jv @ qh))
            gamma = beta
            F_m = alpha * fhat
            f_m = iFFT(F_m, L)
            for p3 in range(quad.n_sig):
                sg = quad.sig[p3]
                beta_t = np.exp(+1j * math.pi / (2 * L) * r * (jv @ sg))
                gamma_t = np.exp(-1j * math.pi / (2 * L) * r * (jv @ sg))
                g_l = iFFT(beta * beta_t * fhat, L)
                g_n = iFFT(gamma * gamma_t * fhat, L)
                w = quad.w_r[p1] * r ** (2 * d - 3) * quad.w_s[p2] * quad.w_sig[p3]
                F1 = FFT(g_l * g_n, L)            # inner convolution (l, n)
                F2 = FFT(f0 * g_n, L)
                F3 = F1
                F4 = FFT(g_l * f0, L)
                K1 += w * FFT(f_m * iFFT(F1, L), L)
                K2 += w * FFT(f_m * iFFT(F2, L), L)
                K3 += w * FFT(f0 * iFFT(F3, L), L)
                K4 += w * FFT(f_m * iFFT(F4, L), L)
    Khat = 2.0 ** (1 - d) * (K1 - K2 + K3 - K4)
    K = iFFT(Khat, L)
    return K.real.copy(), float(np.max(np.abs(K.imag)))


def _apply_nyquist(fhat: np.ndarray, nyquist: str) -> np.ndarray:
    if nyquist == "keep":
        return fhat
    if nyquist != "zero":
        raise ValueError(nyquist)
    d, N = fhat.ndim, fhat.shape[0]
    out = fhat.copy()
    for ax in range(d):
        idx = [slice(None)] * d
        idx[ax] = N // 2
        out[tuple(idx)] = 0.0
    return out


# ----------------------------------------------------------------------------
# The same sum accumulated on the grid
# ----------------------------------------------------------------------------


def shifted_field(fhat: np.ndarray, L: float, x: np.ndarray) -> np.ndarray:
    """f_N(k_i - x) on the grid: iFFT of fhat_j exp(-i pi j.x / L)."""
    d, N = fhat.ndim, fhat.shape[0]
    return iFFT(fhat * phase(d, N, L, x), L)


def collision_fast(f: np.ndarray, L: float, quad: Quadrature, nyquist: str = "keep",
                   node_range: tuple[int, int] | None = None, return_complex: bool = False):
    """Algorithm 1 with its transform pairs cancelled by linearity.

    Per node, on the grid: F = f(k_i), C = f_N(k_i - q) [= f(k2)],
    A = f_N(k_i - a) [= f(k')], B = f_N(k_i - b) [= f(k2')], and the four
    terms of Eq. (2.7) are K1 = A C B, K2 = F C B, K3 = A F B, K4 = A C F.
    Q = 2^{1-d} sum_p W_p (K1 - K2 + K3 - K4).  The sum of FFTs of the
    products equals the FFT of their sum, and each FFT(iFFT(.)) is the
    identity on [-N/2, N/2-1]^d, so this equals ``collision_alg1`` up to
    rounding.  ``node_range`` restricts the sum to flat node indices
    [lo, hi) (lexicographic order) for timing samples.
    Returns (Re Q, max |Im Q|), or the complex Q if ``return_complex``."""
    d, N = f.ndim, f.shape[0]
    fhat = _apply_nyquist(FFT(f, L), nyquist)
    F = f.astype(np.float64)
    acc = np.zeros(f.shape, dtype=np.complex128)
    lo, hi = node_range if node_range is not None else (0, quad.M)
    last_q = None
    C = None
    for flat, (p1, p2, p3, W, q, a, b) in enumerate(quad.nodes()):
        if flat < lo or flat >= hi:
            continue
        if last_q is None or (p1, p2) != last_q:
            C = shifted_field(fhat, L, q)
            last_q = (p1, p2)
        A = shifted_field(fhat, L, a)
        B = shifted_field(fhat, L, b)
        K1 = A * C * B
        K2 = F * C * B
        K3 = A * F * B
        K4 = A * C * F
        acc += W * (K1 - K2 + K3 - K4)
    Q = 2.0 ** (1 - d) * acc
    if return_complex:
        return Q
    return Q.real.copy(), float(np.max(np.abs(Q.imag)))


# ----------------------------------------------------------------------------
# The de-aliased sum: linear index sums through zero-padded transforms
# ----------------------------------------------------------------------------


def pad_coefficients(fhat: np.ndarray, factor: int = 2) -> np.ndarray:
    """The coefficients of the same truncated series (3.1) on a grid `factor`
    times finer over the same D_L: every mode j in [-N/2, N/2-1]^d keeps its
    value, the new modes are zero (DFT positions of each grid)."""
    d, N = fhat.ndim, fhat.shape[0]
    idx = np.mod(modes_1d(N), factor * N)
    out = np.zeros((factor * N,) * d, dtype=np.complex128)
    out[np.ix_(*([idx] * d))] = fhat
    return out


def truncate_coefficients(ghat: np.ndarray, N: int) -> np.ndarray:
    """The modes j in [-N/2, N/2-1]^d of a finer grid's coefficients, in the
    DFT positions of the N grid."""
    d = ghat.ndim
    idx = np.mod(modes_1d(N), ghat.shape[0])
    return ghat[np.ix_(*([idx] * d))].copy()


def collision_dealiased(f: np.ndarray, L: float, quad: Quadrature, nyquist: str = "keep",
                        return_complex: bool = False):
    """The sum of ``collision_fast`` with the linear index sums l + m + n = j
    of Eqs. (3.3)-(3.6) instead of the circular ones: the classical padding
    de-aliasing the paper points to for its fast algorithm (Sec. 3.2 remark).

    The coefficients are padded to a 2N grid over the same D_L; there the
    fields f_N(k - x) and f_N(k) are evaluated, the products are formed and
    weighted as in ``collision_fast``, and the fine-grid coefficients of the
    sum are kept on [-N/2, N/2-1]^d.  Products of three series with modes in
    [-N/2, N/2-1] have modes in [-3N/2, 3N/2-3], and such a mode can reach a
    kept mode j modulo 2N only through itself, so the kept coefficients are
    the linear sums exactly.  Returns (Re Q, max |Im Q|) on the N grid, or the
    complex Q if ``return_complex``."""
    d, N = f.ndim, f.shape[0]
    fhat = _apply_nyquist(FFT(f, L), nyquist)
    ghat = pad_coefficients(fhat, 2)
    F = iFFT(ghat, L)
    acc = np.zeros(ghat.shape, dtype=np.complex128)
    last_q = None
    C = None
    for p1, p2, p3, W, q, a, b in quad.nodes():
        if last_q is None or (p1, p2) != last_q:
            C = shifted_field(ghat, L, q)
            last_q = (p1, p2)
        A = shifted_field(ghat, L, a)
        B = shifted_field(ghat, L, b)
        acc += W * (A * C * B - F * C * B + A * F * B - A * C * F)
    Khat = truncate_coefficients(FFT(2.0 ** (1 - d) * acc, L), N)
    Q = iFFT(Khat, L)
    if return_complex:
        return Q
    return Q.real.copy(), float(np.max(np.abs(Q.imag)))


# ----------------------------------------------------------------------------
# Q at chosen grid points (direct evaluation of the truncated series)
# ----------------------------------------------------------------------------


def collision_at_points(f: np.ndarray, L: float, quad: Quadrature, points: Sequence,
                        nyquist: str = "keep", chunk: int = 256):
    """``collision_fast`` at grid indices ``points`` (list of d-tuples) only.

    Each shifted value f_N(k_i - x) = sum_j fhat_j exp(i pi j.(k_i - x)/L) is
    summed directly over all N^d modes (Eq. (3.1)), one axis at a time, for
    all nodes at once; no FFT is involved.  Returns complex Q at the points.
    """
    d, N = f.ndim, f.shape[0]
    fhat = _apply_nyquist(FFT(f, L), nyquist)
    k1 = grid_1d(N, L)
    j1 = modes_1d(N).astype(np.float64)
    nodes = list(quad.nodes())
    W = np.array([n[3] for n in nodes])
    shifts = {"c": np.array([n[4] for n in nodes]),
              "a": np.array([n[5] for n in nodes]),
              "b": np.array([n[6] for n in nodes])}
    out = []
    for pt in points:
        pt = tuple(int(v) for v in pt)
        kpt = np.array([k1[v] for v in pt])
        vals = {}
        for key, X in shifts.items():
            res = np.empty(len(nodes), dtype=np.complex128)
            for s in range(0, len(nodes), chunk):
                Xc = X[s:s + chunk]                        # (P, d)
                # e[ax][p, j] = exp(i pi j (k_ax - x_ax)/L)
                e = [np.exp(1j * math.pi / L * np.outer(kpt[ax] - Xc[:, ax], j1))
                     for ax in range(d)]
                t = fhat.reshape(-1, N) @ e[d - 1].T         # (N^{d-1}, P)
                t = t.T.reshape((len(Xc),) + (N,) * (d - 1))
                for ax in range(d - 2, -1, -1):
                    t = np.einsum("p...j,pj->p...", t, e[ax])
                res[s:s + chunk] = t
            vals[key] = res
        F = f[pt]
        A, B, C = vals["a"], vals["b"], vals["c"]
        P = A * C * B - F * C * B + A * F * B - A * C * F
        out.append(2.0 ** (1 - d) * np.sum(W * P))
    return np.array(out)


# ----------------------------------------------------------------------------
# Classical spectral sums, Eqs. (3.3)-(3.6)
# ----------------------------------------------------------------------------


def _triples(d: int, N: int, wrap: bool):
    """All (l, m, n, j) mode-index triples with l + m + n = j: modulo N when
    ``wrap`` (what N-point transforms compute), exactly otherwise.  Indices
    are flat DFT positions; the signed vectors come with them."""
    jv = mode_vectors(d, N).reshape(-1, d)
    P = jv.shape[0]
    li, mi = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    li, mi = li.ravel(), mi.ravel()
    out = []
    for jflat in range(P):
        nvec = jv[jflat][None, :] - jv[li] - jv[mi]
        if wrap:
            nvec = (nvec + N // 2) % N - N // 2
            keep = np.ones(len(li), dtype=bool)
        else:
            keep = np.all((nvec >= -N // 2) & (nvec <= N // 2 - 1), axis=1)
        npos = np.ravel_multi_index(tuple((nvec[keep] % N).T), (N,) * d)
        out.append((li[keep], mi[keep], npos, jflat))
    return jv, out


def _vector_code(v: np.ndarray, half: int) -> np.ndarray:
    """Flat index of integer vectors with components in [-half, half]."""
    base = 2 * half + 1
    code = np.zeros(v.shape[0], dtype=np.int64)
    for ax in range(v.shape[1]):
        code = code * base + (v[:, ax] + half)
    return code


def _all_vectors(d: int, half: int) -> np.ndarray:
    """Every integer vector with components in [-half, half], in code order."""
    r = np.arange(-half, half + 1)
    return np.stack(np.meshgrid(*([r] * d), indexing="ij"), axis=-1).reshape(-1, d)


class _SeparatedWeights:
    """G_1 - G_2 + G_3 - G_4 of Eqs. (3.3)-(3.6) in the separated quadrature
    form of Sec. 3.3 (Eq. (3.8) and its K2-K4 analogues).

    Every term is sum_{p1} w_r |q|^{2d-3} Sq_{p1}(u) Ss_{p1}(v) with
    Sq(u) = sum_{p2} w_s exp(-i pi |q| u.qhat/(2L)) and
    Ss(v) = sum_{p3} w_sig exp(+i pi |q| v.sigma/(2L)) for integer vectors
      G1: u = 2m+l+n, v = l-n   (alpha(m) beta(l) gamma(n), beta~(l) gamma~(n))
      G2: u = 2m+n,   v = -n    (alpha(m) gamma(n),         gamma~(n))
      G3: u = l+n,    v = l-n   (beta(l) gamma(n),          beta~(l) gamma~(n))
      G4: u = 2m+l,   v = l     (alpha(m) beta(l),          beta~(l))
    Sq and Ss are tabulated once over every integer vector that can occur."""

    def __init__(self, L: float, quad: Quadrature, N: int):
        d = quad.d
        self.hu, self.hv = 2 * N, N
        uu = _all_vectors(d, self.hu).astype(np.float64)
        vv = _all_vectors(d, self.hv).astype(np.float64)
        c = math.pi / (2.0 * L)
        self.wr = quad.w_r * quad.r ** (2 * d - 3)
        self.Sq = np.stack([np.exp(-1j * c * r * (uu @ quad.qhat.T)) @ quad.w_s for r in quad.r])
        self.Ss = np.stack([np.exp(+1j * c * r * (vv @ quad.sig.T)) @ quad.w_sig for r in quad.r])

    def __call__(self, lv, mv, nv):
        us = [2 * mv + lv + nv, 2 * mv + nv, lv + nv, 2 * mv + lv]
        vs = [lv - nv, -nv, lv - nv, lv]
        sign = [1.0, -1.0, 1.0, -1.0]
        G = np.zeros(lv.shape[0], dtype=np.complex128)
        for t in range(4):
            iu = _vector_code(us[t], self.hu)
            iv = _vector_code(vs[t], self.hv)
            G += sign[t] * (self.wr @ (self.Sq[:, iu] * self.Ss[:, iv]))
        return G


def _sphere_mean_phase(d: int, x: np.ndarray) -> np.ndarray:
    """int_{S^{d-1}} exp(i x.sigma) dsigma as a function of |x|:
    2 pi J0(|x|) for d = 2 and 4 pi sin|x|/|x| for d = 3."""
    if d == 2:
        return 2.0 * math.pi * scipy.special.j0(x)
    return 4.0 * math.pi * np.sinc(x / math.pi)


def psi_exact(d: int, R: float, a: np.ndarray, b: np.ndarray, n_gl: int = 384) -> np.ndarray:
    """int_0^R r^{2d-3} Phi_d(r a) Phi_d(r b) dr, Phi_d the sphere mean above;
    the angular integrals are exact and the smooth radial one uses a
    Gauss-Legendre rule of ``n_gl`` nodes."""
    x, w = np.polynomial.legendre.leggauss(n_gl)
    r = 0.5 * R * (x + 1.0)
    w = 0.5 * R * w
    a = np.asarray(a, dtype=np.float64)[..., None]
    b = np.asarray(b, dtype=np.float64)[..., None]
    integrand = r ** (2 * d - 3) * _sphere_mean_phase(d, r * a) * _sphere_mean_phase(d, r * b)
    return np.sum(w * integrand, axis=-1)


def _weights_exact(L, d, R, lv, mv, nv):
    """G_1 - G_2 + G_3 - G_4 without quadrature: each weight reduces to
    int_0^R r^{2d-3} Phi(r|u|) Phi(r|v|) dr with u the q-frequency and v the
    sigma-frequency of the term (same u, v as ``_SeparatedWeights``, scaled
    by pi/(2L))."""
    us = [2 * mv + lv + nv, 2 * mv + nv, lv + nv, 2 * mv + lv]
    vs = [lv - nv, -nv, lv - nv, lv]
    sign = [1.0, -1.0, 1.0, -1.0]
    c = math.pi / (2.0 * L)
    G = np.zeros(lv.shape[0], dtype=np.float64)
    for t in range(4):
        key = np.stack([np.sum(us[t] ** 2, axis=1), np.sum(vs[t] ** 2, axis=1)], axis=1)
        kk, inv = np.unique(key, axis=0, return_inverse=True)
        vals = psi_exact(d, R, c * np.sqrt(kk[:, 0]), c * np.sqrt(kk[:, 1]))
        G += sign[t] * vals[inv.reshape(-1)]
    return G.astype(np.complex128)


def collision_direct(f: np.ndarray, L: float, quad: Quadrature, wrap: bool = True,
                     weights: str = "quadrature", nyquist: str = "keep",
                     return_hat: bool = False):
    """hat K_j = 2^{1-d} sum_{l+m+n=j} (G_1 - G_2 + G_3 - G_4) f_l f_m f_n,
    Eqs. (3.2)-(3.6), O(N^{3d}).  ``wrap`` sums over l+m+n = j mod N (the
    circular sums N-point transforms produce, so equal to the fast form);
    otherwise over l+m+n = j exactly as printed.  ``weights`` is
    "quadrature" (the separated forms of Sec. 3.3 with Eq. (3.8)'s nodes) or
    "exact" (closed-form angular integrals; ``quad`` supplies d and R).
    Returns (Re K, max |Im K|) on the grid, or hat K if ``return_hat``."""
    d, N = f.ndim, f.shape[0]
    fhat = _apply_nyquist(FFT(f, L), nyquist).reshape(-1)
    jv, trip = _triples(d, N, wrap)
    Khat = np.zeros(N ** d, dtype=np.complex128)
    sep = _SeparatedWeights(L, quad, N) if weights == "quadrature" else None
    for l, m, n, jflat in trip:
        if weights == "quadrature":
            G = sep(jv[l], jv[m], jv[n])
        else:
            G = _weights_exact(L, d, quad.R, jv[l], jv[m], jv[n])
        Khat[jflat] = 2.0 ** (1 - d) * np.sum(G * fhat[l] * fhat[m] * fhat[n])
    Khat = Khat.reshape((N,) * d)
    if return_hat:
        return Khat
    K = iFFT(Khat, L)
    return K.real.copy(), float(np.max(np.abs(K.imag)))


# ----------------------------------------------------------------------------
# Eq. (2.7) with an analytic f
# ----------------------------------------------------------------------------


def collision_realspace(fun: Callable, k: np.ndarray, quad: Quadrature,
                        chunk: int = 4096) -> np.ndarray:
    """The quadrature of Eq. (2.7) at points k (shape (..., d)) with f
    evaluated exactly at k' = k - a, k2 = k - q, k2' = k - b (no
    interpolation, no periodisation).  ``fun`` maps (..., d) to (...)."""
    d = quad.d
    k = np.asarray(k, dtype=np.float64)
    shape = k.shape[:-1]
    kf = k.reshape(-1, d)
    nodes = list(quad.nodes())
    W = np.array([n[3] for n in nodes])
    c = np.array([n[4] for n in nodes])
    a = np.array([n[5] for n in nodes])
    b = np.array([n[6] for n in nodes])
    F = fun(kf)[:, None]
    acc = np.zeros(kf.shape[0], dtype=np.float64)
    for s in range(0, len(nodes), chunk):
        sl = slice(s, s + chunk)
        A = fun(kf[:, None, :] - a[None, sl, :])
        B = fun(kf[:, None, :] - b[None, sl, :])
        C = fun(kf[:, None, :] - c[None, sl, :])
        acc += (A * C * B - F * C * B + A * F * B - A * C * F) @ W[sl]
    return (2.0 ** (1 - d) * acc).reshape(shape)


# ----------------------------------------------------------------------------
# Macroscopic quantities (Sec. 2)
# ----------------------------------------------------------------------------


def moments(g: np.ndarray, L: float) -> np.ndarray:
    """[rho, momentum_1..d, E] = h^d sum_i g_i [1, k_i, |k_i|^2] (the grid
    rectangle rule for rho = int f, E = int f |k|^2)."""
    d, N = g.ndim, g.shape[0]
    h = 2.0 * L / N
    k = grid_points(d, N, L)
    w = h ** d
    out = [w * np.sum(g)]
    out += [w * np.sum(g * k[..., a]) for a in range(d)]
    out += [w * np.sum(g * np.sum(k * k, axis=-1))]
    return np.array(out)


# ----------------------------------------------------------------------------
# Time stepping of the Galerkin system (Sec. 4, RK4)
# ----------------------------------------------------------------------------


def rk_step(f: np.ndarray, L: float, quad: Quadrature, dt: float, stages: int,
            nyquist: str = "keep", dealias: bool = False) -> np.ndarray:
    """One explicit Runge-Kutta step of df/dt = Re Q(f) on the grid values:
    1 = forward Euler, 2 = Heun, 4 = classical RK4 (the paper's integrator).
    ``dealias`` steps the linear-sum operator of ``collision_dealiased``."""
    evaluate = collision_dealiased if dealias else collision_fast
    Q = lambda g: evaluate(g, L, quad, nyquist)[0]
    if stages == 1:
        return f + dt * Q(f)
    if stages == 2:
        k1 = Q(f)
        k2 = Q(f + dt * k1)
        return f + 0.5 * dt * (k1 + k2)
    if stages == 4:
        k1 = Q(f)
        k2 = Q(f + 0.5 * dt * k1)
        k3 = Q(f + 0.5 * dt * k2)
        k4 = Q(f + dt * k3)
        return f + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    raise ValueError("stages must be 1, 2 or 4")
