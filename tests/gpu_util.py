"""Helpers for the GPU tests: a CUDA check and oracle comparisons."""
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
