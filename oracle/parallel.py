"""The oracle's K and K^T applied over all host cores (detector subsets in worker
processes).

TEST INFRASTRUCTURE ONLY: used by the test-suite (full-size parity cases) and by the
benchmark's CPU-baseline / reference leg.  The CUDA library never imports it.

Nothing here changes the oracle's arithmetic.  ``forward`` and ``adjoint`` of
``pat_oracle`` already loop over detectors one at a time (Sec. 4.2, eq. (K_def):
every data row belongs to one detector).  So K u is the concatenation of the oracle's
K u over detector subsets, and K^T y is the sum over the subsets of the oracle's K^T
of their rows.  The subsets are contiguous, and the partial images are added in subset
order, so the result does not depend on scheduling.

Workers are started with the ``spawn`` method, which is safe after CUDA has been
initialised in the parent process.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from dataclasses import replace

import numpy as np

from . import pat_oracle as O


def _forward(args):
    g, u = args
    return O.forward(g, u)


def _adjoint(args):
    g, y = args
    return O.adjoint(g, y)


def _forward_rows(args):
    g, u, rows = args
    return O.forward_rows(g, u, rows)


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class OraclePool:
    """K and K^T of ``g`` split over ``workers`` processes (default: all host cores)."""

    def __init__(self, g: O.Geometry, workers: int | None = None):
        self.g = g
        self.workers = max(1, min(workers or host_cores(), g.n_det))
        bounds = np.linspace(0, g.n_det, self.workers + 1).round().astype(int)
        self.spans = [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        self.subs = [replace(g, det_xy=g.det_xy[a:b].copy()) for a, b in self.spans]
        self.pool = mp.get_context("spawn").Pool(len(self.spans)) if len(self.spans) > 1 else None

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _map(self, fn, tasks):
        if self.pool is None:
            return [fn(t) for t in tasks]
        return self.pool.map(fn, tasks)

    def forward(self, u) -> np.ndarray:
        u = np.asarray(u, dtype=np.float64).reshape(self.g.n, self.g.n)
        parts = self._map(_forward, [(s, u) for s in self.subs])
        return np.concatenate(parts, axis=0)

    def adjoint(self, y) -> np.ndarray:
        y = np.asarray(y, dtype=np.float64).reshape(self.g.n_det, self.g.n_t)
        parts = self._map(_adjoint, [(s, y[a:b]) for s, (a, b) in zip(self.subs, self.spans)])
        out = np.zeros((self.g.n, self.g.n))
        for p in parts:                       # fixed order
            out += p
        return out

    def forward_rows(self, u, rows) -> np.ndarray:
        """Selected entries d*T + k of K u (the oracle's ``forward_rows``), rows split
        evenly over the workers."""
        u = np.asarray(u, dtype=np.float64).reshape(self.g.n, self.g.n)
        rows = np.asarray(rows)
        chunks = [c for c in np.array_split(rows, len(self.spans)) if len(c)]
        parts = self._map(_forward_rows, [(self.g, u, c) for c in chunks])
        return np.concatenate(parts) if parts else np.zeros(0)

    def problem(self, f, **kw) -> O.Problem:
        """An oracle ``Problem`` whose K, K^T and |K| sums run on the pool."""
        n = self.g.n
        krow = self.forward(np.ones((n, n))).ravel()
        kcol = self.adjoint(np.ones((self.g.n_det, self.g.n_t)))
        return O.Problem(n=n, K=lambda u: self.forward(u).ravel(), KT=lambda y: self.adjoint(y),
                         f=np.asarray(f, dtype=np.float64).ravel(), k_abs_rows=krow, k_abs_cols=kcol, **kw)
