"""Seeded synthetic inputs for the collision-operator workloads.

This module is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path's tests and benchmark.  It holds no arithmetic of the method
itself: it samples initial data f on the periodic grid, draws the seeded
random numbers those data use, and names the workload sizes.

Grid (Sec. 3.2, Step 1 and Eq. (3.1)): the periodic box D_L = [-L, L]^d is
sampled at k_i = -L + i * 2L/N, i = 0..N-1 on every axis, arrays in
row-major order with the last axis fastest.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: draw i of
stream ``seed`` is mix(seed + (i + 1) * 0x9E3779B97F4A7C15), and the top 53
bits give a double in [0, 1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 20250316


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from SplitMix64 stream ``seed`` (counter-based)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed % (1 << 64)) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def grid_axes(d: int, N: int, L: float):
    """The d coordinate arrays k_1..k_d on the N^d grid (broadcast-ready)."""
    x = -L + np.arange(N, dtype=np.float64) * (2.0 * L / N)
    return np.meshgrid(*([x] * d), indexing="ij")


def _k2(d, N, L):
    ks = grid_axes(d, N, L)
    return ks, sum(k * k for k in ks)


# ---------------------------------------------------------------- generators

def gaussian(d: int, N: int, L: float, width: float = 1.0) -> np.ndarray:
    """Isotropic Gaussian exp(-|k|^2 / (2 width^2))."""
    _, k2 = _k2(d, N, L)
    return np.exp(-k2 / (2.0 * width * width))


def rayleigh_jeans(d: int, N: int, L: float, mu: float, nu, xi: float) -> np.ndarray:
    """Rayleigh-Jeans state 1 / (mu + nu.k + xi |k|^2), Eq. (2.6)."""
    ks, k2 = _k2(d, N, L)
    nu = list(nu) + [0.0] * (d - len(nu))
    den = mu + xi * k2
    for a in range(d):
        den = den + nu[a] * ks[a]
    return 1.0 / den


def rayleigh_jeans_fn(d: int, mu: float, nu, xi: float):
    """The same state as a function of points k (shape (..., d))."""
    nu = np.asarray(list(nu) + [0.0] * (d - len(nu)), dtype=np.float64)

    def fn(k):
        k = np.asarray(k, dtype=np.float64)
        return 1.0 / (mu + k @ nu + xi * np.sum(k * k, axis=-1))
    return fn


def two_gaussians(N: int, L: float, seed: int, width: float = 0.7,
                  centre: float = 2.0) -> np.ndarray:
    """2D sum of two Gaussians at (+-centre, 0), amplitudes 1 + 0.1 (u - 1/2)."""
    (k1, k2), _ = _k2(2, N, L)
    u = splitmix64_uniform(seed, 2)
    f = np.zeros_like(k1)
    for s, us in zip((+1.0, -1.0), u):
        amp = 1.0 + 0.1 * (us - 0.5)
        f += amp * np.exp(-((k1 - s * centre) ** 2 + k2 ** 2) / (2.0 * width * width))
    return f


def gaussian_noise(d: int, N: int, L: float, seed: int, eps: float = 0.01) -> np.ndarray:
    """exp(-|k|^2/2) * (1 + eps (2u - 1)), one uniform draw per grid point."""
    base = gaussian(d, N, L)
    u = splitmix64_uniform(seed, N ** d).reshape((N,) * d)
    return base * (1.0 + eps * (2.0 * u - 1.0))


def ring(d: int, N: int, L: float, radius: float = 3.0) -> np.ndarray:
    """Ring-shaped exp(-(|k| - radius)^2)."""
    _, k2 = _k2(d, N, L)
    return np.exp(-(np.sqrt(k2) - radius) ** 2)


def discontinuous(d: int, N: int, L: float, rho1=1.2, rho2=0.8, T1=2.0 / 3.0,
                  T2=1.5) -> np.ndarray:
    """Two-temperature data split at k_1 = 0, Eq. (4.2) (2D normalisation
    1/(2 pi T), and (2 pi T)^(-d/2) in general)."""
    ks, k2 = _k2(d, N, L)
    g1 = rho1 * (2 * math.pi * T1) ** (-d / 2) * np.exp(-k2 / (2 * T1))
    g2 = rho2 * (2 * math.pi * T2) ** (-d / 2) * np.exp(-k2 / (2 * T2))
    return np.where(ks[0] > 0, g1, g2)


@dataclasses.dataclass(frozen=True)
class TrigPoly:
    """Real trigonometric polynomial 1 + eps * sum_t a_t cos(pi j_t.k / L + phi_t).

    Every mode has |j_t| <= jmax per component, so for N > 2 jmax the grid
    samples determine it exactly.
    """
    L: float
    modes: np.ndarray     # (T, d) integer mode vectors
    amps: np.ndarray      # (T,)
    phases: np.ndarray    # (T,)
    eps: float

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        arg = (math.pi / self.L) * (k @ self.modes.T.astype(np.float64)) + self.phases
        return 1.0 + self.eps * (np.cos(arg) @ self.amps)

    def on_grid(self, N: int) -> np.ndarray:
        d = self.modes.shape[1]
        ks = np.stack(grid_axes(d, N, self.L), axis=-1)
        return self(ks)


def trig_poly(d: int, L: float, jmax: int, n_terms: int, seed: int,
              eps: float = 0.2) -> TrigPoly:
    """Seeded band-limited real trig polynomial with |j_c| <= jmax."""
    u = splitmix64_uniform(seed, n_terms * (d + 2))
    u = u.reshape(n_terms, d + 2)
    modes = np.floor(u[:, :d] * (2 * jmax + 1)).astype(np.int64) - jmax
    amps = u[:, d] / n_terms
    phases = 2.0 * math.pi * u[:, d + 1]
    return TrigPoly(L=L, modes=modes, amps=amps, phases=phases, eps=eps)


# ---------------------------------------------------------------- workloads

@dataclasses.dataclass(frozen=True)
class Workload:
    """A named problem size: dimension, grid, box, quadrature counts."""
    name: str
    d: int
    N: int
    L: float
    n_r: int
    n_s: int
    n_sig: int
    sphere: str   # "midpoint" (2D), "cube", "octahedron", ... (3D)
    seed: int

    @property
    def M(self) -> int:
        return self.n_r * self.n_s * self.n_sig

    def initial(self) -> np.ndarray:
        return INITIAL[self.name](self)


# The five workload shapes: 2D N=16 M=32; 2D N=128 M=512; 3D N=32 M=1024;
# 3D N=64 M=2048 (the headline size); and the mixed serving stream.
WORKLOADS = {
    "2d_n16_m32": Workload("2d_n16_m32", 2, 16, 8.0, 8, 4, 1, "midpoint", BASE_SEED + 0),
    "2d_n128_m512": Workload("2d_n128_m512", 2, 128, 8.0, 32, 4, 4, "midpoint", BASE_SEED + 1),
    "3d_n32_m1024": Workload("3d_n32_m1024", 3, 32, 8.0, 16, 8, 8, "cube", BASE_SEED + 2),
    "3d_n64_m2048": Workload("3d_n64_m2048", 3, 64, 8.0, 32, 8, 8, "cube", BASE_SEED + 3),
}

INITIAL = {
    "2d_n16_m32": lambda w: gaussian(2, w.N, w.L),
    "2d_n128_m512": lambda w: two_gaussians(w.N, w.L, w.seed),
    "3d_n32_m1024": lambda w: gaussian_noise(3, w.N, w.L, w.seed),
    "3d_n64_m2048": lambda w: ring(3, w.N, w.L),
}


def serving_request_sizes():
    """(d, N, n_r, n_s, n_sig) choices of the mixed serving stream: 2D N in
    {64, 128, 256} with M = 4N (N/4 x 4 x 4) and 3D N in {32, 48, 64} with
    M = 32N (N/2 x 8 x 8)."""
    out = [(2, n, n // 4, 4, 4) for n in (64, 128, 256)]
    out += [(3, n, n // 2, 8, 8) for n in (32, 48, 64)]
    return out
