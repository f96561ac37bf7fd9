"""A handle of the C library with torch device buffers (marshalling only)."""
from __future__ import annotations

import numpy as np

from . import capi


class Solver:
    """AMG-DD setup on a matrix; solves with torch CUDA tensors.

    rowptr/col/val: host CSR of A_0; part/nsub: subdomain of every unknown;
    padding: eta_l (int or per-level list, last value repeats).
    """

    def __init__(self, rowptr, col, val, part, nsub, padding=1, n_fac=2, theta=0.25,
                 max_coarse=16, max_levels=25, host_only=False, threads=0, schedule=0, precision=0,
                 hybrid_level=0, interp=0, p_max=4, coarsen=0, strict_assumption=0, stream=None):
        o = capi.amgdd_options_default()
        o.n_fac = n_fac
        o.theta = theta
        o.max_coarse = max_coarse
        o.max_levels = max_levels
        o.host_only = int(host_only)
        o.threads = threads
        o.schedule = schedule
        o.precision = precision
        o.hybrid_level = hybrid_level
        o.interp = {"direct": 0, "exti": 1}.get(interp, interp)
        o.p_max = p_max
        o.coarsen = {"rs": 0, "hmis": 1}.get(coarsen, coarsen)
        o.strict_assumption = int(strict_assumption)
        self.n = len(rowptr) - 1
        self.h = capi.amgdd_setup(rowptr, col, val, part, nsub, padding, o, stream)
        self.stats = capi.amgdd_get_stats(self.h)
        self.nlev = self.stats.num_levels
        self.level_n = [self.stats.n[l] for l in range(self.nlev)]
        self.offsets = np.concatenate([[0], np.cumsum(self.level_n)]).astype(np.int64)
        self.nsub = nsub

    def close(self):
        if getattr(self, "h", None):
            capi.amgdd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, x, tol=1e-8, max_iter=200, stream=None):
        return capi.amgdd_solve(self.h, b, x, tol, max_iter, stream)

    def vcycle_solve(self, b, x, tol=1e-8, max_iter=200, stream=None):
        return capi.amg_vcycle_solve(self.h, b, x, tol, max_iter, stream)

    def solve_multi(self, B, X, tol=1e-8, max_iter=200, stream=None):
        """All columns of B / X (device tensors of shape (n, 2) or (n, 4))."""
        return capi.amgdd_solve_multi(self.h, B, X, tol, max_iter, stream)

    def hybrid_solve(self, b, x, tol=1e-8, max_iter=200, stream=None):
        """Hybrid AMG-DD (set up with hybrid_level >= 1)."""
        return capi.amg_hybrid_solve(self.h, b, x, tol, max_iter, stream)
