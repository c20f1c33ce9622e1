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


def test_unmutated_copy_passes():
    mod = _mutant("def FFT(", "def FFT(")
    assert pins.fast_vs_realspace(mod, 2) < 1e-12
