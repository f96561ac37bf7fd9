"""ctypes binding of libamgdd.so (the C ABI declared in include/amgdd.h).

Argument marshalling only: every step of the solve phase runs in the
library's CUDA kernels. Device vectors are passed as torch tensors (their
data_ptr()), streams as torch.cuda.Stream or raw cudaStream_t integers. If
the shared library has not been built the import fails loudly; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamgdd.so")

MAX_LEVELS = 40

STATUS = {
    0: "AMGDD_OK", 1: "AMGDD_ERR_INVALID_ARG", 2: "AMGDD_ERR_NOT_SYMMETRIC",
    3: "AMGDD_ERR_HIERARCHY_ASSUMPTION", 4: "AMGDD_ERR_OOM", 5: "AMGDD_ERR_CUDA",
    6: "AMGDD_ERR_NO_CONVERGENCE", 7: "AMGDD_ERR_DEVICE_TIMEOUT", 8: "AMGDD_ERR_SINGULAR",
    9: "AMGDD_ERR_NOT_ON_DEVICE",
}


class amgdd_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class amgdd_options(C.Structure):
    _fields_ = [("theta", C.c_double), ("max_coarse", C.c_int32), ("max_levels", C.c_int32),
                ("n_fac", C.c_int32), ("strict_assumption", C.c_int32), ("host_only", C.c_int32),
                ("threads", C.c_int32), ("schedule", C.c_int32), ("precision", C.c_int32),
                ("hybrid_level", C.c_int32), ("interp", C.c_int32), ("p_max", C.c_int32),
                ("coarsen", C.c_int32), ("reserved", C.c_int32 * 2)]


class amgdd_setup_stats(C.Structure):
    _fields_ = [("num_levels", C.c_int32), ("nsub", C.c_int32), ("n", C.c_int32 * MAX_LEVELS),
                ("nnz", C.c_int64 * MAX_LEVELS), ("nnz_P", C.c_int64 * MAX_LEVELS),
                ("comp_real", C.c_int64 * MAX_LEVELS), ("comp_ghost", C.c_int64 * MAX_LEVELS),
                ("comp_nnz_real", C.c_int64 * MAX_LEVELS), ("comp_nnz_A", C.c_int64 * MAX_LEVELS),
                ("comp_nnz_P", C.c_int64 * MAX_LEVELS), ("comp_nnz_R", C.c_int64 * MAX_LEVELS),
                ("operator_complexity", C.c_double), ("grid_complexity", C.c_double),
                ("composite_overhead", C.c_double), ("assumption_violations", C.c_int64),
                ("device_bytes", C.c_int64), ("fac_fma", C.c_int64), ("fac_entry_bytes", C.c_int64),
                ("setup_seconds", C.c_double)]


class amgdd_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("final_relres", C.c_double),
                ("history", C.POINTER(C.c_double)), ("seconds", C.c_double),
                ("kernel_launches", C.c_int64)]


EXPORTS = [
    "amgdd_options_default", "amgdd_box_partition", "amgdd_setup", "amgdd_destroy",
    "amgdd_last_error", "amgdd_get_stats", "amgdd_get_maps", "amgdd_get_operator", "amgdd_get_cf",
    "amgdd_get_coarse_inverse", "amgdd_residual", "amgdd_restrict", "amgdd_fac",
    "amgdd_get_fac_state", "amgdd_iterate", "amgdd_solve", "amg_vcycle", "amg_vcycle_solve",
    "amgdd_residual_csr_noalloc", "amgdd_iterate_multi", "amgdd_fac_multi", "amgdd_solve_multi",
    "amg_hybrid_cycle", "amg_hybrid_solve", "amgdd_kappa_grad_3d",
    "amgdd_set_fac_kernel", "amgdd_autotune", "amgdd_plan_teams",
]

FAC_CANDIDATES = 32
TUNE_ALLOW_REORDERED = 1

_lib = None


def load(path: str = LIB_PATH):
    """Load libamgdd.so (raises OSError when it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libamgdd.so is not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "amgdd_options_default": [C.POINTER(amgdd_options)],
        "amgdd_box_partition": [i32, i32, i32, i32, i32, i32, vp, C.POINTER(i32)],
        "amgdd_setup": [C.POINTER(amgdd_csr), vp, i32, vp, i32, C.POINTER(amgdd_options), vp,
                        C.POINTER(vp)],
        "amgdd_get_stats": [vp, C.POINTER(amgdd_setup_stats)],
        "amgdd_get_maps": [vp, i32, i32, vp, vp, C.POINTER(i32)],
        "amgdd_get_operator": [vp, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64), vp,
                               vp, vp],
        "amgdd_get_cf": [vp, i32, vp, vp],
        "amgdd_get_coarse_inverse": [vp, vp],
        "amgdd_residual": [vp, vp, vp, vp, C.POINTER(f64), vp],
        "amgdd_restrict": [vp, vp, vp],
        "amgdd_fac": [vp, vp, vp, vp],
        "amgdd_get_fac_state": [vp, i32, i32, vp, vp],
        "amgdd_iterate": [vp, vp, vp, vp],
        "amgdd_solve": [vp, vp, vp, f64, i32, vp, C.POINTER(amgdd_solve_info)],
        "amg_vcycle": [vp, vp, vp, vp],
        "amg_vcycle_solve": [vp, vp, vp, f64, i32, vp, C.POINTER(amgdd_solve_info)],
        "amgdd_residual_csr_noalloc": [i32, vp, vp, vp, vp, vp, vp, vp, vp],
        "amgdd_iterate_multi": [vp, vp, vp, i32, vp],
        "amgdd_fac_multi": [vp, vp, vp, i32, vp],
        "amgdd_set_fac_kernel": [vp, i32, i32],
        "amgdd_autotune": [vp, i32, i32, i32, vp, C.POINTER(i32), vp],
        "amg_hybrid_cycle": [vp, vp, vp, vp],
        "amgdd_kappa_grad_3d": [i32, i32, i32, vp, vp, vp, vp, vp],
        "amg_hybrid_solve": [vp, vp, vp, f64, i32, vp, C.POINTER(amgdd_solve_info)],
        "amgdd_solve_multi": [vp, vp, vp, i32, f64, i32, vp, C.POINTER(amgdd_solve_info)],
        "amgdd_plan_teams": [vp, i32, i32, vp, vp, vp, vp, vp, C.POINTER(i32)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.amgdd_destroy.argtypes = [vp]
    lib.amgdd_destroy.restype = None
    lib.amgdd_last_error.argtypes = [vp]
    lib.amgdd_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class AmgddError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _check(st, h=None):
    if st != 0:
        msg = load().amgdd_last_error(h)
        raise AmgddError(st, msg.decode() if msg else "")


def _ptr(a):
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(s):
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    return getattr(s, "cuda_stream", s)


# ---- functions with the C names ---------------------------------------------

def amgdd_options_default():
    o = amgdd_options()
    _check(load().amgdd_options_default(C.byref(o)))
    return o


def amgdd_box_partition(shape, box):
    shape = list(shape) + [1] * (3 - len(shape))
    box = list(box) + [1] * (3 - len(box))
    part = np.zeros(int(np.prod(shape)), np.int32)
    ns = C.c_int32()
    _check(load().amgdd_box_partition(*[int(s) for s in shape], *[int(b) for b in box],
                                      part.ctypes.data, C.byref(ns)))
    return part, ns.value


def amgdd_setup(rowptr, col, val, part, nsub, padding, opts=None, stream=None):
    """Returns a handle (int). Host numpy CSR arrays; see include/amgdd.h."""
    lib = load()
    rp = np.ascontiguousarray(rowptr, np.int32)
    ci = np.ascontiguousarray(col, np.int32)
    v = np.ascontiguousarray(val, np.float64)
    pt = np.ascontiguousarray(part, np.int32)
    pad = np.ascontiguousarray(np.atleast_1d(padding), np.int32)
    A = amgdd_csr(len(rp) - 1, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
    o = opts if opts is not None else amgdd_options_default()
    h = C.c_void_p()
    st = lib.amgdd_setup(C.byref(A), pt.ctypes.data, int(nsub), pad.ctypes.data, len(pad),
                         C.byref(o), _stream(stream) if not o.host_only else None, C.byref(h))
    _check(st)
    return h.value


def amgdd_destroy(h):
    load().amgdd_destroy(h)


def amgdd_get_stats(h):
    s = amgdd_setup_stats()
    _check(load().amgdd_get_stats(h, C.byref(s)), h)
    return s


def amgdd_get_maps(h, sub, level):
    lib = load()
    n = C.c_int32()
    _check(lib.amgdd_get_maps(h, sub, level, None, None, C.byref(n)), h)
    g = np.zeros(max(n.value, 1), np.int32)
    k = np.zeros(max(n.value, 1), np.uint8)
    _check(lib.amgdd_get_maps(h, sub, level, g.ctypes.data, k.ctypes.data, C.byref(n)), h)
    return g[:n.value], k[:n.value]


def amgdd_get_operator(h, level, which):
    lib = load()
    w = {"A": 0, "P": 1, "R": 2}[which] if isinstance(which, str) else int(which)
    rows, cols, nnz = C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib.amgdd_get_operator(h, level, w, C.byref(rows), C.byref(cols), C.byref(nnz),
                                  None, None, None), h)
    rp = np.zeros(rows.value + 1, np.int64)
    ci = np.zeros(max(nnz.value, 1), np.int32)
    v = np.zeros(max(nnz.value, 1), np.float64)
    _check(lib.amgdd_get_operator(h, level, w, None, None, None, rp.ctypes.data, ci.ctypes.data,
                                  v.ctypes.data), h)
    return rp, ci[:nnz.value], v[:nnz.value], (rows.value, cols.value)


def amgdd_get_cf(h, level, n, with_cf=True):
    cf = np.zeros(n, np.int32) if with_cf else None
    l1 = np.zeros(n, np.float64)
    _check(load().amgdd_get_cf(h, level, None if cf is None else cf.ctypes.data, l1.ctypes.data), h)
    return cf, l1


def amgdd_plan_teams(work, nblocks):
    """The team plan of FAC candidate 31 for per-grid work (host only): a list
    per block of its teams as (first warp, warps, grids)."""
    work = np.ascontiguousarray(work, np.int64)
    nsub = len(work)
    cap = 15 * int(nblocks)
    block_off = np.zeros(nblocks + 1, np.int32)
    w0 = np.zeros(cap, np.int32)
    nw = np.zeros(cap, np.int32)
    grid_off = np.zeros(cap + 1, np.int32)
    grid = np.zeros(max(nsub, 1), np.int32)
    nteams = C.c_int32()
    _check(load().amgdd_plan_teams(work.ctypes.data, nsub, int(nblocks), block_off.ctypes.data, w0.ctypes.data,
                                   nw.ctypes.data, grid_off.ctypes.data, grid.ctypes.data, C.byref(nteams)))
    plan = []
    for b in range(nblocks):
        plan.append([(int(w0[k]), int(nw[k]), [int(g) for g in grid[grid_off[k]:grid_off[k + 1]]])
                     for k in range(block_off[b], block_off[b + 1])])
    return plan


def amgdd_get_coarse_inverse(h, nL):
    a = np.zeros(nL * nL, np.float64)
    _check(load().amgdd_get_coarse_inverse(h, a.ctypes.data), h)
    return a.reshape(nL, nL)


def amgdd_residual(h, b, x, r, stream=None):
    nrm2 = C.c_double()
    _check(load().amgdd_residual(h, _ptr(b), _ptr(x), _ptr(r), C.byref(nrm2), _stream(stream)), h)
    return nrm2.value


def amgdd_restrict(h, r_all, stream=None):
    _check(load().amgdd_restrict(h, _ptr(r_all), _stream(stream)), h)


def amgdd_fac(h, r_all, x, stream=None):
    _check(load().amgdd_fac(h, _ptr(r_all), _ptr(x), _stream(stream)), h)


def amgdd_get_fac_state(h, sub, level, count):
    u = np.zeros(count, np.float64)
    f = np.zeros(count, np.float64)
    _check(load().amgdd_get_fac_state(h, sub, level, u.ctypes.data, f.ctypes.data), h)
    return u, f


def amgdd_iterate(h, b, x, stream=None):
    _check(load().amgdd_iterate(h, _ptr(b), _ptr(x), _stream(stream)), h)


def _solve(fn, h, b, x, tol, max_iter, stream, raise_on_noconv):
    hist = np.zeros(max_iter + 1, np.float64)
    info = amgdd_solve_info()
    info.history = hist.ctypes.data_as(C.POINTER(C.c_double))
    st = fn(h, _ptr(b), _ptr(x), float(tol), int(max_iter), _stream(stream), C.byref(info))
    if st != 0 and not (st == 6 and not raise_on_noconv):
        _check(st, h)
    return dict(iterations=info.iterations, converged=bool(info.converged),
                final_relres=info.final_relres, history=hist[:info.iterations + 1].copy(),
                seconds=info.seconds, kernel_launches=info.kernel_launches)


def amgdd_solve(h, b, x, tol=1e-8, max_iter=200, stream=None, raise_on_noconv=True):
    return _solve(load().amgdd_solve, h, b, x, tol, max_iter, stream, raise_on_noconv)


def amg_vcycle(h, b, x, stream=None):
    _check(load().amg_vcycle(h, _ptr(b), _ptr(x), _stream(stream)), h)


def amg_vcycle_solve(h, b, x, tol=1e-8, max_iter=200, stream=None, raise_on_noconv=True):
    return _solve(load().amg_vcycle_solve, h, b, x, tol, max_iter, stream, raise_on_noconv)


def amgdd_residual_csr_noalloc(n, rowptr, col, val, b, x, r, nrm2, stream=None):
    """r = b - A x and nrm2[0] = ||r||^2 for a device CSR, with no allocation
    (all arguments are device tensors the caller owns)."""
    _check(load().amgdd_residual_csr_noalloc(int(n), _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b),
                                              _ptr(x), _ptr(r), _ptr(nrm2), _stream(stream)))


def amgdd_iterate_multi(h, B, X, stream=None):
    """One AMG-DD iteration for every column of B / X (device, shape (n, nrhs))."""
    _check(load().amgdd_iterate_multi(h, _ptr(B), _ptr(X), int(B.shape[1]), _stream(stream)), h)


def amgdd_fac_multi(h, R_all, X, stream=None):
    """FAC step for every column: R_all (device, shape (sum_l n_l, nrhs)) holds
    the restricted residuals of all levels; X (device, (n, nrhs)) is updated."""
    _check(load().amgdd_fac_multi(h, _ptr(R_all), _ptr(X), int(X.shape[1]), _stream(stream)), h)


def amgdd_set_fac_kernel(h, nrhs, candidate):
    """FAC kernel candidate for nrhs columns (see amgdd_autotune)."""
    _check(load().amgdd_set_fac_kernel(h, int(nrhs), int(candidate)), h)


def amgdd_autotune(h, nrhs=1, reps=3, stream=None, allow_reordered=False):
    """Times every FAC kernel candidate for nrhs columns and keeps the fastest
    (with allow_reordered, also the group-per-row candidates whose row sums
    round differently). Returns (best candidate, ms per candidate, -1 where
    not timed)."""
    ms = np.zeros(FAC_CANDIDATES, np.float64)
    best = C.c_int32(-1)
    flags = TUNE_ALLOW_REORDERED if allow_reordered else 0
    _check(load().amgdd_autotune(h, int(nrhs), int(reps), flags, ms.ctypes.data, C.byref(best), _stream(stream)), h)
    return int(best.value), ms


def amgdd_solve_multi(h, B, X, tol=1e-8, max_iter=200, stream=None, raise_on_noconv=True):
    """AMG-DD for all columns of B / X (device, shape (n, nrhs), nrhs = 2 or 4)."""
    nrhs = int(B.shape[1])
    hist = np.zeros(nrhs * (max_iter + 1), np.float64)
    info = amgdd_solve_info()
    info.history = hist.ctypes.data_as(C.POINTER(C.c_double))
    st = load().amgdd_solve_multi(h, _ptr(B), _ptr(X), nrhs, float(tol), int(max_iter), _stream(stream),
                                  C.byref(info))
    if st != 0 and not (st == 6 and not raise_on_noconv):
        _check(st, h)
    k = info.iterations
    return dict(iterations=k, converged=bool(info.converged), final_relres=info.final_relres,
                history=hist.reshape(nrhs, max_iter + 1)[:, :k + 1].copy(), seconds=info.seconds,
                kernel_launches=info.kernel_launches)


def amg_hybrid_cycle(h, b, x, stream=None):
    _check(load().amg_hybrid_cycle(h, _ptr(b), _ptr(x), _stream(stream)), h)


def amg_hybrid_solve(h, b, x, tol=1e-8, max_iter=200, stream=None, raise_on_noconv=True):
    return _solve(load().amg_hybrid_solve, h, b, x, tol, max_iter, stream, raise_on_noconv)


def amgdd_kappa_grad_3d(shape, kappa, x, lam, grad, stream=None):
    """grad = d(-lam^T A(kappa) x)/d kappa for the 3D diffusion operator
    (shape = (nx, ny, nz); all arrays device tensors of nx*ny*nz doubles)."""
    nx, ny, nz = (int(v) for v in shape)
    _check(load().amgdd_kappa_grad_3d(nx, ny, nz, _ptr(kappa), _ptr(x), _ptr(lam), _ptr(grad),
                                      _stream(stream)))
