"""Process-parallel driver of the oracle's fast form (test infrastructure only).

``collision_fast`` sums over the quadrature nodes in lexicographic order.  This
module splits that node list into contiguous ranges of whole groups (p1, p2),
evaluates each range with ``collision_fast(..., node_range=...)`` in a
``spawn`` process pool, and adds the partial sums in node order.  The result
equals one ``collision_fast`` call up to the order of floating-point additions.
Only ``tests/`` and ``bench.py``'s CPU legs use it; the pool is started with
``spawn`` so it is safe to create after CUDA has been initialised.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np


def _partial(args):
    f, L, quad_args, nyquist, lo, hi = args
    from oracle import wke_oracle as O
    quad = O.make_quadrature(*quad_args)
    t = time.perf_counter()
    q = O.collision_fast(f, L, quad, nyquist=nyquist, node_range=(lo, hi), return_complex=True)
    return q, time.perf_counter() - t


def node_ranges(M: int, group: int, parts: int):
    """At most `parts` contiguous ranges [lo, hi) covering 0..M, each made of
    whole groups of `group` nodes."""
    groups = M // group
    parts = max(1, min(parts, groups))
    bounds = [round(k * groups / parts) * group for k in range(parts + 1)]
    return [(bounds[k], bounds[k + 1]) for k in range(parts) if bounds[k + 1] > bounds[k]]


class OraclePool:
    """A spawn process pool evaluating the oracle's fast form over node ranges."""

    def __init__(self, workers: int | None = None):
        self.workers = workers or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.workers)

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def collision_fast(self, f, L, quad_args, nyquist="keep", parts=None):
        """Complex Q of ``collision_fast`` for the quadrature
        ``make_quadrature(*quad_args)`` = (d, n_r, n_s, n_sig, R, sphere,
        sphere_sig).  Returns (Q, wall seconds, summed worker seconds)."""
        d, n_r, n_s, n_sig = quad_args[:4]
        ranges = node_ranges(n_r * n_s * n_sig, n_sig, parts or 2 * self.workers)
        t = time.perf_counter()
        outs = self.pool.map(_partial, [(np.ascontiguousarray(f), L, tuple(quad_args), nyquist, lo, hi)
                                        for lo, hi in ranges])
        wall = time.perf_counter() - t
        Q = np.zeros(f.shape, dtype=np.complex128)
        for q, _ in outs:
            Q += q
        return Q, wall, sum(s for _, s in outs)
