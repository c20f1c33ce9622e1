"""Helpers for the GPU tests: a CUDA check and oracle comparisons."""
import math

import numpy as np
import pytest


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2503_12805_gb300 import wke
    wke.lib()          # raises when the library is missing: no fallback path exists
    return torch


def rel_max_err(got, ref, scale=None):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    s = np.max(np.abs(ref)) if scale is None else scale
    return float(np.max(np.abs(got - ref)) / s)


def gpu_collision(torch, plan, f_np, want_imag=False):
    f = torch.tensor(np.ascontiguousarray(f_np), dtype=plan.dtype, device="cuda")
    Qim = torch.empty_like(f) if want_imag else None
    Q = plan.collision(f, Qim=Qim)
    torch.cuda.synchronize()
    if want_imag:
        return Q.double().cpu().numpy(), Qim.double().cpu().numpy()
    return Q.double().cpu().numpy()


EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -53


def cancellation(f, L, quad, dealias=False, nyquist="keep"):
    """kappa = max T / max |Q| with T(k) = 2^{1-d} sum_p |W_p| (|A B C| +
    |F C B| + |A F B| + |A C F|): how much larger the four cubic terms are than
    the Q they cancel to.  With `dealias` the terms are taken on the 2N grid
    the de-aliased evaluation uses."""
    from oracle import wke_oracle as O
    d, N = f.ndim, f.shape[0]
    fhat = O._apply_nyquist(O.FFT(f, L), nyquist)
    if dealias:
        fhat = O.pad_coefficients(fhat, 2)
    fN = O.iFFT(fhat, L)
    F = np.abs(fN)
    T = np.zeros(fN.shape)
    acc = np.zeros(fN.shape, dtype=np.complex128)
    C = None
    last = None
    for p1, p2, p3, W, q, a, b in quad.nodes():
        if (p1, p2) != last:
            C = O.shifted_field(fhat, L, q)
            last = (p1, p2)
        A = O.shifted_field(fhat, L, a)
        B = O.shifted_field(fhat, L, b)
        T += abs(W) * (np.abs(A * B * C) + F * np.abs(C * B) + F * np.abs(A * B) + F * np.abs(A * C))
        acc += W * (A * B * (C + fN) - C * fN * (A + B))
    return float(np.max(T) / np.max(np.abs(acc)))


def tolerance(prec, f, L, quad, dealias=False, nyquist="keep"):
    """Tolerance (relative max-norm against max |Q|) derived from the
    arithmetic: the shifted fields carry errors of order eps log2(N^d)
    relative to their own size (a log2(N^d)-stage transform), and Q inherits
    them amplified by the cancellation kappa, so the bound is
    eps log2(N^d) kappa; never below the targets 1e-12 (FP64) and 1e-5 (FP32).
    The transform grid is 2N per axis for a de-aliased plan."""
    d, N = f.ndim, f.shape[0] * (2 if dealias else 1)
    eps, floor = (EPS64, 1e-12) if prec == "fp64" else (EPS32, 1e-5)
    return max(floor, eps * math.log2(N ** d) * cancellation(f, L, quad, dealias, nyquist))


def fp32_tolerance(f, L, quad, floor=1e-5, dealias=False, nyquist="keep"):
    """The FP32 case of ``tolerance``."""
    return max(floor, tolerance("fp32", f, L, quad, dealias, nyquist))
