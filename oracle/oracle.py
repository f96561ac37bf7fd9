"""ctypes wrapper around the plain C oracle (amgdd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline of the benchmark, never by the product library. The C file cites the
paper section each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amgdd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64, no contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def oracle_lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build_oracle())
        vp = C.c_void_p
        sig = {
            "orc_hier_build": (vp, [C.c_int, i64p, i32p, f64p, C.c_double, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, i32p]),
            "orc_hier_free": (None, [vp]),
            "orc_hier_status": (C.c_int, [vp]),
            "orc_hier_nlev": (C.c_int, [vp]),
            "orc_hier_n": (C.c_int, [vp, C.c_int]),
            "orc_hier_nnz": (C.c_int64, [vp, C.c_int, C.c_int]),
            "orc_hier_rows": (C.c_int, [vp, C.c_int, C.c_int]),
            "orc_hier_cols": (C.c_int, [vp, C.c_int, C.c_int]),
            "orc_hier_get": (None, [vp, C.c_int, C.c_int, i64p, i32p, f64p]),
            "orc_hier_get_cf": (None, [vp, C.c_int, i32p]),
            "orc_hier_get_l1inv": (None, [vp, C.c_int, f64p]),
            "orc_hier_get_ainv": (None, [vp, f64p]),
            "orc_comp_build": (vp, [vp, i32p, C.c_int, i32p]),
            "orc_comp_free": (None, [vp]),
            "orc_comp_violations": (C.c_int64, [vp]),
            "orc_comp_violation_flag": (C.c_int, [vp, C.c_int, C.c_int]),
            "orc_comp_count": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
            "orc_comp_get_map": (None, [vp, C.c_int, C.c_int, i32p, u8p]),
            "orc_comp_overhead": (C.c_double, [vp, vp]),
            "orc_residual": (None, [vp, f64p, f64p, f64p]),
            "orc_restrict_all": (None, [vp, f64p]),
            "orc_levels_total": (C.c_int64, [vp]),
            "orc_vcycle_apply": (None, [vp, f64p, f64p]),
            "orc_vcycle_solve": (C.c_int, [vp, f64p, f64p, C.c_double, C.c_int, f64p]),
            "orc_algfac": (None, [vp, vp, C.c_int, f64p, C.c_int, f64p, f64p]),
            "orc_masked_fac": (None, [vp, vp, C.c_int, f64p, C.c_int, f64p, f64p]),
            "orc_amgdd_iteration": (None, [vp, vp, f64p, f64p, C.c_int, i32p, C.c_int, f64p]),
            "orc_amgdd_solve": (C.c_int, [vp, vp, f64p, f64p, C.c_double, C.c_int, C.c_int, C.c_int, f64p]),
            "orc_algfac32": (None, [vp, vp, C.c_int, f64p, C.c_int, f64p, f64p]),
            "orc_hier_sub": (vp, [vp, C.c_int]),
            "orc_hier_sub_free": (None, [vp]),
            "orc_part_on_level": (None, [vp, i32p, C.c_int, i32p]),
            "orc_hybrid_apply": (None, [vp, vp, vp, C.c_int, C.c_int, f64p, f64p]),
            "orc_hybrid_solve": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, f64p, f64p, C.c_double, C.c_int,
                                          f64p]),
            "orc_amgdd_iteration32": (None, [vp, vp, f64p, f64p, C.c_int, f64p]),
            "orc_set_threads": (C.c_int, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def set_threads(n):
    """Threads of the oracle's OpenMP loops (0 keeps the current count);
    returns the count in effect."""
    return int(oracle_lib().orc_set_threads(int(n)))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Hierarchy + composite grids of one problem, with the solve routines.

    rowptr/col/val: CSR of A_0 (any integer types); part/nsub: subdomain of
    every unknown; padding: int or per-level list (eta_l).
    """

    def __init__(self, rowptr, col, val, part=None, nsub=1, padding=1,
                 theta=0.25, max_coarse=16, max_levels=25, interp="direct", pmax=4, coarsen="rs"):
        lib = oracle_lib()
        self.lib = lib
        self.h = None
        self.c = None
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        v = _c64(val)
        self.n = len(rp) - 1
        if interp not in ("direct", "exti"):
            raise ValueError("interp is 'direct' or 'exti' (extended+i)")
        if coarsen not in ("rs", "hmis"):
            raise ValueError("coarsen is 'rs' (Ruge-Stueben first pass) or 'hmis'")
        # HMIS coarsens within the subdomains first; without a partition it
        # sees one subdomain
        sub = np.zeros(self.n, np.int32) if part is None else np.ascontiguousarray(part, dtype=np.int32)
        self.h = lib.orc_hier_build(self.n, rp, ci, v, float(theta), int(max_coarse), int(max_levels),
                                    1 if interp == "exti" else 0, int(pmax), 1 if coarsen == "hmis" else 0, sub)
        st = lib.orc_hier_status(self.h)
        if st != 0:
            lib.orc_hier_free(self.h)
            self.h = None
            raise RuntimeError("oracle: coarsest matrix is %s"
                               % ("singular" if st == 1 else "too large for a dense inverse"))
        self.nlev = lib.orc_hier_nlev(self.h)
        self.level_n = [lib.orc_hier_n(self.h, l) for l in range(self.nlev)]
        self.offsets = np.concatenate([[0], np.cumsum(self.level_n)]).astype(np.int64)
        self.c = None
        if part is not None:
            part = np.ascontiguousarray(part, dtype=np.int32)
            if np.isscalar(padding):
                pad = np.full(self.nlev, int(padding), dtype=np.int32)
            else:
                pad = np.ascontiguousarray(padding, dtype=np.int32)
                if len(pad) < self.nlev:
                    pad = np.concatenate([pad, np.full(self.nlev - len(pad), pad[-1], np.int32)])
            self.nsub = int(nsub)
            self.padding = pad
            self.part = part
            self.c = lib.orc_comp_build(self.h, part, self.nsub, pad)
        self._hyb = {}

    def __del__(self):
        try:
            for hs, cs in getattr(self, "_hyb", {}).values():
                self.lib.orc_comp_free(cs)
                self.lib.orc_hier_sub_free(hs)
            if self.c:
                self.lib.orc_comp_free(self.c)
            if self.h:
                self.lib.orc_hier_free(self.h)
        except Exception:
            pass

    # ---- hierarchy ------------------------------------------------------
    def matrix(self, l, which="A"):
        """(rowptr int64, col int32, val f64, shape) of A_l, P_l or R_l."""
        w = {"A": 0, "P": 1, "R": 2}[which]
        nnz = self.lib.orc_hier_nnz(self.h, l, w)
        rows = self.lib.orc_hier_rows(self.h, l, w)
        cols = self.lib.orc_hier_cols(self.h, l, w)
        rp = np.zeros(rows + 1, np.int64)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1), np.float64)
        self.lib.orc_hier_get(self.h, l, w, rp, ci, v)
        return rp, ci[:nnz], v[:nnz], (rows, cols)

    def scipy(self, l, which="A"):
        import scipy.sparse as sp
        rp, ci, v, shape = self.matrix(l, which)
        return sp.csr_matrix((v, ci, rp), shape=shape)

    def cf(self, l):
        o = np.zeros(self.level_n[l], np.int32)
        self.lib.orc_hier_get_cf(self.h, l, o)
        return o

    def l1inv(self, l):
        o = np.zeros(self.level_n[l], np.float64)
        self.lib.orc_hier_get_l1inv(self.h, l, o)
        return o

    def ainv(self):
        nL = self.level_n[-1]
        o = np.zeros(nL * nL, np.float64)
        self.lib.orc_hier_get_ainv(self.h, o)
        return o.reshape(nL, nL)

    # ---- composite grids ------------------------------------------------
    def comp_sizes(self, p, l):
        return (self.lib.orc_comp_count(self.c, p, l, 0),
                self.lib.orc_comp_count(self.c, p, l, 1),
                self.lib.orc_comp_count(self.c, p, l, 2))

    def comp_map(self, p, l):
        """(global index, kind) in local order: owned, other real, ghost."""
        nr, ng, _ = self.comp_sizes(p, l)
        g = np.zeros(max(nr + ng, 1), np.int32)
        k = np.zeros(max(nr + ng, 1), np.uint8)
        self.lib.orc_comp_get_map(self.c, p, l, g, k)
        return g[:nr + ng], k[:nr + ng]

    def violations(self):
        return int(self.lib.orc_comp_violations(self.c))

    def violation_pairs(self):
        """(subdomain, level) pairs that break the connectivity assumption of
        Sections 4.2 and 4.5 between level l and l + 1, in order."""
        return [(p, l) for p in range(self.nsub) for l in range(self.nlev - 1)
                if self.lib.orc_comp_violation_flag(self.c, p, l)]

    def overhead(self):
        return float(self.lib.orc_comp_overhead(self.h, self.c))

    # ---- solve phase ----------------------------------------------------
    def residual(self, b, x):
        r = np.zeros(self.n)
        self.lib.orc_residual(self.h, _c64(b), _c64(x), r)
        return r

    def restrict_all(self, r0):
        rl = np.zeros(int(self.offsets[-1]))
        rl[:self.n] = r0
        self.lib.orc_restrict_all(self.h, rl)
        return [rl[self.offsets[l]:self.offsets[l + 1]].copy() for l in range(self.nlev)]

    def vcycle_apply(self, f, u=None):
        u = np.zeros(self.n) if u is None else _c64(u).copy()
        self.lib.orc_vcycle_apply(self.h, _c64(f), u)
        return u

    def vcycle_solve(self, b, x0=None, tol=1e-8, maxit=200):
        x = np.zeros(self.n) if x0 is None else _c64(x0).copy()
        hist = np.zeros(maxit + 1)
        k = self.lib.orc_vcycle_solve(self.h, _c64(b), x, float(tol), int(maxit), hist)
        return x, hist[:k + 1]

    def _split(self, a):
        return [a[self.offsets[l]:self.offsets[l + 1]].copy() for l in range(self.nlev)]

    def algfac(self, p, rl, nfac):
        """AlgFAC on composite grid p; returns per-level (u_l, f_l), global indexing."""
        flat = _c64(np.concatenate(rl))
        u = np.zeros(int(self.offsets[-1]))
        f = np.zeros(int(self.offsets[-1]))
        self.lib.orc_algfac(self.h, self.c, int(p), flat, int(nfac), u, f)
        return self._split(u), self._split(f)

    def masked_fac(self, p, r0, nfac):
        u = np.zeros(int(self.offsets[-1]))
        f = np.zeros(int(self.offsets[-1]))
        self.lib.orc_masked_fac(self.h, self.c, int(p), _c64(r0), int(nfac), u, f)
        return self._split(u), self._split(f)

    def amgdd_iteration(self, b, x, nfac, subset=None):
        x = _c64(x).copy()
        rl = np.zeros(int(self.offsets[-1]))
        if subset is None:
            sel = np.zeros(1, np.int32)
            ns = -1
        else:
            sel = np.ascontiguousarray(subset, dtype=np.int32)
            ns = len(sel)
        self.lib.orc_amgdd_iteration(self.h, self.c, _c64(b), x, int(nfac), sel, ns, rl)
        return x

    def amgdd_solve(self, b, nfac, x0=None, tol=1e-8, maxit=200, mixed=False):
        """Algorithm 2 to tol; mixed=True runs the AlgFAC cycles in FP32."""
        x = np.zeros(self.n) if x0 is None else _c64(x0).copy()
        hist = np.zeros(maxit + 1)
        k = self.lib.orc_amgdd_solve(self.h, self.c, _c64(b), x, float(tol), int(maxit),
                                     int(nfac), int(bool(mixed)), hist)
        return x, hist[:k + 1]

    def algfac32(self, p, rl, nfac):
        """FP32 AlgFAC on composite grid p (values widened to double)."""
        flat = _c64(np.concatenate(rl))
        u = np.zeros(int(self.offsets[-1]))
        f = np.zeros(int(self.offsets[-1]))
        self.lib.orc_algfac32(self.h, self.c, int(p), flat, int(nfac), u, f)
        return self._split(u), self._split(f)

    def amgdd_iteration32(self, b, x, nfac):
        x = _c64(x).copy()
        rl = np.zeros(int(self.offsets[-1]))
        self.lib.orc_amgdd_iteration32(self.h, self.c, _c64(b), x, int(nfac), rl)
        return x


    # ---- hybrid AMG-DD (Algorithm 3) ---------------------------------------
    def _hybrid(self, lev0):
        if lev0 not in self._hyb:
            hs = self.lib.orc_hier_sub(self.h, int(lev0))
            pl = np.zeros(self.level_n[lev0], np.int32)
            self.lib.orc_part_on_level(self.h, self.part, int(lev0), pl)
            cs = self.lib.orc_comp_build(hs, pl, self.nsub,
                                         np.ascontiguousarray(self.padding[lev0:], np.int32))
            self._hyb[lev0] = (hs, cs)
        return self._hyb[lev0]

    def hybrid_apply(self, lev0, f, u, nfac):
        hs, cs = self._hybrid(lev0)
        u = _c64(u).copy()
        self.lib.orc_hybrid_apply(self.h, hs, cs, int(lev0), int(nfac), _c64(f), u)
        return u

    def hybrid_solve(self, lev0, b, nfac, x0=None, tol=1e-8, maxit=200):
        hs, cs = self._hybrid(lev0)
        x = np.zeros(self.n) if x0 is None else _c64(x0).copy()
        hist = np.zeros(maxit + 1)
        k = self.lib.orc_hybrid_solve(self.h, hs, cs, int(lev0), int(nfac), _c64(b), x, float(tol),
                                      int(maxit), hist)
        return x, hist[:k + 1]


def kappa_gradient(kappa, x, lam):
    """d(-lam^T A(kappa) x)/d kappa for the 3D 7-point diffusion operator with
    harmonic-mean faces 2 k_i k_j/(k_i + k_j) and Dirichlet faces using k_i.

    lam^T A x = sum over interior faces c_f (lam_i - lam_j)(x_i - x_j)
              + sum over boundary faces of i of k_i lam_i x_i,
    dc_f/dk_i = 2 k_j^2 / (k_i + k_j)^2. kappa: (nz, ny, nx); x, lam: flat,
    lexicographic (i fastest). Plain per-axis loops over the faces."""
    k = np.asarray(kappa, np.float64)
    X = np.asarray(x, np.float64).reshape(k.shape)
    Lm = np.asarray(lam, np.float64).reshape(k.shape)
    g = np.zeros_like(k)
    nb = np.zeros_like(k)
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, -1)
        hi[ax] = slice(1, None)
        lo, hi = tuple(lo), tuple(hi)
        ka, kb = k[lo], k[hi]
        prod = (Lm[lo] - Lm[hi]) * (X[lo] - X[hi])
        g[lo] += 2 * kb * kb / ((ka + kb) ** 2) * prod
        g[hi] += 2 * ka * ka / ((ka + kb) ** 2) * prod
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = 0
        last[ax] = -1
        nb[tuple(first)] += 1
        nb[tuple(last)] += 1
    g += nb * Lm * X
    return -g.reshape(-1)
