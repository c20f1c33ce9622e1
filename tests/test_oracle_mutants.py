"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
the pins catch each one.  A mutation the pins could not see would mean the
oracle is not pinned where that mutation lives.
"""
import itertools
import os
import sys
import types

import pytest

from tests import pins

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "wke_oracle.py")

# (name, text in the oracle, planted replacement, pin, d)
MUTANTS = [
    ("drop the 2^(1-d) prefactor of Eq. (2.7)",
     "return (2.0 ** (1 - d) * acc).reshape(shape)", "return (acc).reshape(shape)",
     pins.operator_vs_bruteforce, 2),
    ("radial weight |q|^(d-2) instead of |q|^(2d-3)",
     "W = self.w_r[p1] * r ** (2 * d - 3)", "W = self.w_r[p1] * r ** (d - 2)",
     pins.weight_total, 3),
    ("radial weight |q|^(d-2) seen by the operator",
     "W = self.w_r[p1] * r ** (2 * d - 3)", "W = self.w_r[p1] * r ** (d - 2)",
     pins.operator_vs_bruteforce, 2),
    ("drop the direction weight w_s",
     "* self.w_s[p2] * self.w_sig[p3]", "* self.w_sig[p3]",
     pins.weight_total, 2),
    ("flip the sign of the K2 term",
     "acc += (A * C * B - F * C * B + A * F * B - A * C * F) @ W[sl]",
     "acc += (A * C * B + F * C * B + A * F * B - A * C * F) @ W[sl]",
     pins.rj_zero, 2),
    ("flip the sign of the K3 term (seen by the operator)",
     "acc += (A * C * B - F * C * B + A * F * B - A * C * F) @ W[sl]",
     "acc += (A * C * B - F * C * B - A * F * B - A * C * F) @ W[sl]",
     pins.operator_vs_bruteforce, 3),
    ("k2' shifted by (q - s)/2 like k'",
     "yield p1, p2, p3, W, q, 0.5 * (q - s), 0.5 * (q + s)",
     "yield p1, p2, p3, W, q, 0.5 * (q - s), 0.5 * (q - s)",
     pins.rj_zero, 3),
    ("k2 = k - q/2 instead of k - q",
     "yield p1, p2, p3, W, q, 0.5 * (q - s), 0.5 * (q + s)",
     "yield p1, p2, p3, W, 0.5 * q, 0.5 * (q - s), 0.5 * (q + s)",
     pins.rj_zero, 2),
    ("phase of the shift with the wrong sign",
     "def phase(d: int, N: int, L: float, x: np.ndarray, sign: float = -1.0)",
     "def phase(d: int, N: int, L: float, x: np.ndarray, sign: float = +1.0)",
     pins.fast_vs_realspace, 2),
    ("fast form: K4 uses B for A",
     "        K4 = A * C * F\n", "        K4 = B * C * F\n",
     pins.fast_vs_direct, 3),
    ("fast form: C shifted by a instead of q",
     "            C = shifted_field(fhat, L, q)", "            C = shifted_field(fhat, L, a)",
     pins.fast_vs_realspace, 3),
    ("direct sums: G2 with u = 2m + l",
     "        us = [2 * mv + lv + nv, 2 * mv + nv, lv + nv, 2 * mv + lv]",
     "        us = [2 * mv + lv + nv, 2 * mv + lv, lv + nv, 2 * mv + lv]",
     pins.fast_vs_direct, 2),
    ("Algorithm 1: outer convolution of K3 weighted by alpha",
     "K3 += w * FFT(f0 * iFFT(F3, L), L)", "K3 += w * FFT(f_m * iFFT(F3, L), L)",
     pins.alg1_vs_fast, 2),
    ("Algorithm 1: beta-tilde with the sign of gamma-tilde",
     "beta_t = np.exp(+1j * math.pi / (2 * L) * r * (jv @ sg))",
     "beta_t = np.exp(-1j * math.pi / (2 * L) * r * (jv @ sg))",
     pins.alg1_vs_fast, 3),
    ("coefficients without the (-1)^j of the grid origin",
     "    return np.fft.fftn(g) / float(N ** d) * _alternating_sign(d, N)",
     "    return np.fft.fftn(g) / float(N ** d)",
     pins.naive_dft, 2),
    ("de-aliased: no padding (circular sums)",
     "    ghat = pad_coefficients(fhat, 2)", "    ghat = pad_coefficients(fhat, 1)",
     pins.dealiased_vs_linear, 2),
    ("de-aliased: padded modes stored at the first N positions",
     "    idx = np.mod(modes_1d(N), factor * N)", "    idx = np.arange(N)",
     pins.dealiased_vs_linear, 3),
    ("de-aliased: truncation keeps the first N positions",
     "    idx = np.mod(modes_1d(N), ghat.shape[0])", "    idx = np.arange(N)",
     pins.dealiased_vs_linear, 2),
    ("transposed phase table in the shifted field",
     "    return iFFT(fhat * phase(d, N, L, x), L)",
     "    return iFFT(fhat * np.swapaxes(phase(d, N, L, x), 0, 1), L)",
     pins.fast_vs_realspace, 2),
    ("point evaluator: phase of the shift with the wrong sign",
     "np.exp(1j * math.pi / L * np.outer(kpt[ax] - Xc[:, ax], j1))",
     "np.exp(1j * math.pi / L * np.outer(kpt[ax] + Xc[:, ax], j1))",
     pins.at_points_vs_fast, 3),
    ("point evaluator: first axis's phases on the last axis",
     "t = fhat.reshape(-1, N) @ e[d - 1].T", "t = fhat.reshape(-1, N) @ e[0].T",
     pins.at_points_vs_fast, 2),
    ("point evaluator: contraction over the axes in the wrong order",
     "for ax in range(d - 2, -1, -1):", "for ax in range(d - 1):",
     pins.at_points_vs_fast, 3),
    ("moments: cell volume h^(d-1)",
     "    w = h ** d\n", "    w = h ** (d - 1)\n",
     pins.moments_gaussian, 3),
    ("moments: grid without its -L offset in the momentum",
     "out += [w * np.sum(g * k[..., a]) for a in range(d)]",
     "out += [w * np.sum(g * (k[..., a] + L)) for a in range(d)]",
     pins.moments_gaussian, 2),
    ("moments: energy weight (sum k)^2 instead of |k|^2",
     "out += [w * np.sum(g * np.sum(k * k, axis=-1))]",
     "out += [w * np.sum(g * np.sum(k, axis=-1) ** 2)]",
     pins.moments_gaussian, 2),
]

# Mistakes in the time integrator: the pin is the observed order of accuracy,
# which a correct oracle meets to about 0.2 and a wrong stage weight or stage
# argument misses by at least one order.
RK_MUTANTS = [
    ("RK4: weights 1/3 instead of 1/6, 1/3, 1/3, 1/6",
     "return f + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)",
     "return f + dt / 3.0 * (k1 + k2 + k3 + k4)", 2),
    ("RK4: third stage from k1 instead of k2",
     "k3 = Q(f + 0.5 * dt * k2)", "k3 = Q(f + 0.5 * dt * k1)", 3),
    ("RK4: fourth stage at half the step",
     "k4 = Q(f + dt * k3)", "k4 = Q(f + 0.5 * dt * k3)", 2),
    ("Heun: second stage at half the step",
     "k2 = Q(f + dt * k1)", "k2 = Q(f + 0.5 * dt * k1)", 2),
]


_COUNTER = itertools.count()


def _mutant(old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, f"mutation target not found exactly once: {old!r}"
    name = f"wke_oracle_mutant_{next(_COUNTER)}"
    mod = types.ModuleType(name)
    sys.modules[name] = mod          # dataclasses resolve the defining module
    exec(compile(src.replace(old, new), ORACLE_SRC + "[mutant]", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name,old,new,pin,d", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(name, old, new, pin, d):
    err = pin(_mutant(old, new), d)
    assert err > 1e-6, f"pin {pin.__name__} did not see: {name} (discrepancy {err:.3g})"


@pytest.mark.parametrize("name,old,new,d", RK_MUTANTS, ids=[m[0] for m in RK_MUTANTS])
def test_rk_order_pin_catches_planted_mistake(name, old, new, d):
    defect = pins.rk_order_defect(_mutant(old, new), d)
    assert defect > 0.6, f"order pin did not see: {name} (order defect {defect:.3g})"


def test_unmutated_copy_passes():
    mod = _mutant("def FFT(", "def FFT(")
    assert pins.fast_vs_realspace(mod, 2) < 1e-12
