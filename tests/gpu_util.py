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


def fp32_tolerance(f, L, quad, floor=1e-5):
    """FP32 tolerance (relative max-norm) for one input, from the arithmetic.

    Q is a sum of four cubic terms that cancel: the rounding error of an FP32
    evaluation scales with the size of the terms, not of Q.  With the terms'
    magnitude T(k) = 2^{1-d} sum_p |W_p| (|A B C| + |F C B| + |A F B| + |A C F|)
    and kappa = max T / max |Q|, the shifted fields carry errors of order
    eps32 log2(N^d) relative to their own size (a log2(N^d)-stage transform in
    FP32), so the bound is eps32 log2(N^d) kappa, and never below the target
    `floor` (1e-5)."""
    from oracle import wke_oracle as O
    d, N = f.ndim, f.shape[0]
    fhat = O.FFT(f, L)
    F = np.abs(f.astype(np.float64))
    T = np.zeros(f.shape)
    acc = np.zeros(f.shape, dtype=np.complex128)
    C = None
    last = None
    for p1, p2, p3, W, q, a, b in quad.nodes():
        if (p1, p2) != last:
            C = O.shifted_field(fhat, L, q)
            last = (p1, p2)
        A = O.shifted_field(fhat, L, a)
        B = O.shifted_field(fhat, L, b)
        T += abs(W) * (np.abs(A * B * C) + F * np.abs(C * B) + F * np.abs(A * B) + F * np.abs(A * C))
        acc += W * (A * B * (C + f) - C * f * (A + B))
    kappa = float(np.max(T) / np.max(np.abs(acc)))
    return max(floor, EPS32 * math.log2(N ** d) * kappa)
