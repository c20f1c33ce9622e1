"""Serving loop: continuous batching of time-stepping requests.

Each request's result must be the same when it runs alone and when it runs
in a mix with other requests overlapping on the GPU; requests that cannot fit
the device budget are rejected without affecting the others; a cancelled
request does not disturb the rest of the stream.
"""
import numpy as np
import pytest

import wke_inputs as I
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu

# (d, N, n_r, n_s, n_sig, steps, generator)
MIX = [
    (2, 64, 16, 4, 4, 3, lambda: I.two_gaussians(64, 8.0, 1)),
    (3, 32, 8, 8, 8, 2, lambda: I.gaussian_noise(3, 32, 8.0, 2)),
    (2, 128, 8, 4, 4, 4, lambda: I.two_gaussians(128, 8.0, 3)),
    (3, 16, 8, 8, 8, 5, lambda: I.ring(3, 16, 8.0)),
    (2, 64, 16, 4, 4, 2, lambda: I.gaussian_noise(2, 64, 8.0, 4, 0.05)),
    (3, 32, 8, 8, 8, 1, lambda: I.ring(3, 32, 8.0)),
    (3, 48, 4, 8, 8, 2, lambda: I.ring(3, 48, 8.0)),
]


def _alone(torch, wke, d, N, n_r, n_s, n_sig, steps, f, dt=1e-3):
    with wke.Plan(d, N, 8.0, n_r, n_s, n_sig, precision="fp32") as plan:
        ft = torch.tensor(f, dtype=torch.float32, device="cuda")
        for _ in range(steps):
            plan.step(ft, dt, 4)
        torch.cuda.synchronize()
        return ft.cpu().numpy()


def test_results_same_alone_and_in_the_mix():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    inputs = [gen().astype(np.float32) for *_, gen in MIX]
    with wke.Server(device_budget_bytes=8 << 30, max_active=4) as srv:
        subs = [srv.submit(f, n_r, n_s, n_sig, steps, 1e-3) for (d, N, n_r, n_s, n_sig, steps, _), f in zip(MIX, inputs)]
        stats = [srv.wait(rid, timeout_s=120) for rid, _ in subs]
    assert all(st.status == wke.WKE_OK for st in stats)
    for (d, N, n_r, n_s, n_sig, steps, _), f, (rid, out) in zip(MIX, inputs, subs):
        ref = _alone(torch, wke, d, N, n_r, n_s, n_sig, steps, f)
        assert np.array_equal(out, ref), (d, N)
        assert not np.array_equal(out, f)               # the steps did change f


def test_oversize_request_rejected_others_unaffected():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    small = I.two_gaussians(64, 8.0, 9).astype(np.float32)
    big = I.ring(3, 64, 8.0).astype(np.float32)
    with wke.Server(device_budget_bytes=32 << 20, max_active=2) as srv:
        rid_big, _ = srv.submit(big, 32, 8, 8, 1, 1e-3)
        rid_small, out = srv.submit(small, 16, 4, 4, 2, 1e-3)
        st_big = srv.wait(rid_big, timeout_s=60)
        st_small = srv.wait(rid_small, timeout_s=60)
    assert st_big.status == wke.WKE_ERR_OOM
    assert st_small.status == wke.WKE_OK
    assert np.array_equal(out, _alone(torch, wke, 2, 64, 16, 4, 4, 2, small))


def test_cancelled_request_does_not_disturb_the_stream():
    torch = require_cuda()
    from paper_2503_12805_gb300 import wke
    fs = [I.two_gaussians(64, 8.0, s).astype(np.float32) for s in (11, 12, 13)]
    with wke.Server(device_budget_bytes=4 << 30, max_active=1) as srv:
        r0, o0 = srv.submit(fs[0], 16, 4, 4, 20, 1e-3)
        r1, _ = srv.submit(fs[1], 16, 4, 4, 20, 1e-3)
        r2, o2 = srv.submit(fs[2], 16, 4, 4, 3, 1e-3)
        srv.cancel(r1)
        st = [srv.wait(r, timeout_s=120) for r in (r0, r1, r2)]
    assert [s.status for s in st] == [wke.WKE_OK, wke.WKE_CANCELLED, wke.WKE_OK]
    assert np.array_equal(o0, _alone(torch, wke, 2, 64, 16, 4, 4, 20, fs[0]))
    assert np.array_equal(o2, _alone(torch, wke, 2, 64, 16, 4, 4, 3, fs[2]))
    assert st[2].t_admit >= st[0].t_submit


def test_admitted_requests_overlap_on_the_device():
    """A request admitted while another runs starts at once: the two
    requests' [admission, completion] intervals overlap."""
    require_cuda()
    from paper_2503_12805_gb300 import wke
    long_f = I.ring(3, 64, 8.0).astype(np.float32)
    short_f = I.gaussian_noise(3, 32, 8.0, 31).astype(np.float32)
    with wke.Server(device_budget_bytes=4 << 30, max_active=4) as srv:
        r1, _ = srv.submit(long_f, 32, 8, 8, 60, 1e-5)        # about 60 x 4 evaluations of 1 ms
        r2, _ = srv.submit(short_f, 16, 8, 8, 2, 1e-3)
        s1 = srv.wait(r1, timeout_s=120)
        s2 = srv.wait(r2, timeout_s=120)
    assert s1.status == wke.WKE_OK and s2.status == wke.WKE_OK
    assert s1.t_submit <= s1.t_admit <= s1.t_done and s2.t_submit <= s2.t_admit <= s2.t_done
    assert s2.t_admit < s1.t_done and s1.t_admit < s2.t_done      # the intervals overlap


def test_small_request_passes_one_waiting_for_memory():
    """With a budget that holds the running request and a small one but not a
    large one as well, a small request submitted after the large one is
    admitted first (the large one waits for memory); the large one still runs
    once the first request is done."""
    require_cuda()
    from paper_2503_12805_gb300 import wke
    a = I.gaussian_noise(3, 32, 8.0, 32).astype(np.float32)     # about 17 MiB
    big = I.ring(3, 64, 8.0).astype(np.float32)                  # about 53 MiB
    small = I.two_gaussians(64, 8.0, 33).astype(np.float32)      # about 4 MiB
    with wke.Server(device_budget_bytes=60 << 20, max_active=4) as srv:
        ra, _ = srv.submit(a, 16, 8, 8, 60, 1e-4)
        rb, _ = srv.submit(big, 32, 8, 8, 1, 1e-5)
        rc, _ = srv.submit(small, 16, 4, 4, 1, 1e-3)
        sa, sb, sc = (srv.wait(r, timeout_s=120) for r in (ra, rb, rc))
    assert (sa.status, sb.status, sc.status) == (wke.WKE_OK,) * 3
    assert sc.t_admit < sb.t_admit                  # passed the request waiting for memory
    assert sb.t_admit >= sa.t_done - 1e-3           # which started once memory was free


def test_served_fp64_request_matches_oracle_rk4():
    """One served FP64 request (2D N=32, 4 x 4 x 4 mid-point rule, two RK4
    steps) against the oracle's Runge-Kutta step applied twice."""
    require_cuda()
    from oracle import wke_oracle as O
    from paper_2503_12805_gb300 import wke
    f0 = I.two_gaussians(32, 8.0, 34)
    with wke.Server(device_budget_bytes=1 << 30, max_active=2) as srv:
        rid, out = srv.submit(f0, 4, 4, 4, 2, 1e-3, precision="fp64")
        st = srv.wait(rid, timeout_s=120)
    assert st.status == wke.WKE_OK
    quad = O.make_quadrature(2, 4, 4, 4, O.default_R(8.0), "midpoint")
    ref = f0.copy()
    for _ in range(2):
        ref = O.rk_step(ref, 8.0, quad, 1e-3, 4)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))
