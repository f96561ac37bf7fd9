"""Parity at the two larger configurations, in the launch configuration the
benchmark times: FP32 composite grids inside FP64 refinement, the FAC kernel
chosen by the autotuner (among the candidates that keep the ascending fma
chain).

* 256^3 diffusion, kappa checkerboard {1, 1e3}, 4096 subdomains of 16^3;
* the 64-system batch (24.9M unknowns, 6083 subdomains), four columns.

The oracle cannot run thousands of composite grids in seconds, so each check
samples: composite maps of sampled subdomains on every level, the whole
residual and restriction chain, and one AMG-DD iteration whose update on the
owned points of sampled subdomains (corner, edge, face and interior boxes;
for the batch, boxes of systems of every edge length) equals the oracle's
FP32 AlgFAC on exactly those subdomains, bit for bit. The batch also checks
that columns solved together equal one-column iterations bit for bit, and a
full solve reaches 1e-8 with the final residual recomputed on the host.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import amgdd_inputs as I
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import Solver, capi  # noqa: E402


def _owned_update(o, w, rl, p):
    """x after one iteration from x = 0 on the owned points of grid p: the
    level-0 FP32 AlgFAC correction (0 + u is exact)."""
    u, _ = o.algfac32(p, rl, w["n_fac"])
    own = np.nonzero(w["part"] == p)[0]
    return own, u[0][own]


def _check_maps(o, s, sample):
    assert s.level_n == o.level_n
    for p in sample:
        for l in range(s.nlev):
            g1, k1 = o.comp_map(p, l)
            g2, k2 = capi.amgdd_get_maps(s.h, p, l)
            assert np.array_equal(g1, g2) and np.array_equal(k1, k2), (p, l)


def test_kappa256_mixed_sampled():
    w = I.workload("kappa3d_256", seed=0)
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"])
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
               precision=1)
    best, _ = capi.amgdd_autotune(s.h, 1, reps=1)
    nb = 16
    sample = [0, 5, 5 + nb * 7, 5 + nb * (7 + nb * 9), 4095, 1000, 2730]
    _check_maps(o, s, sample)
    b = w["b"]
    bd = torch.from_numpy(b).cuda()
    r_all = torch.zeros(int(s.offsets[-1]), dtype=torch.float64, device="cuda")
    capi.amgdd_residual(s.h, bd, torch.zeros_like(bd), r_all[:s.n])
    capi.amgdd_restrict(s.h, r_all)
    rl = o.restrict_all(o.residual(b, np.zeros(s.n)))
    assert np.array_equal(r_all.cpu().numpy(), np.concatenate(rl))
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_iterate(s.h, bd, x)
    xg = x.cpu().numpy()
    for p in sample:
        own, ref = _owned_update(o, w, rl, p)
        assert np.array_equal(xg[own], ref), (best, p)
    assert np.count_nonzero(xg) > 0.99 * s.n
    # the teams kernel with lists of grids (4096 grids for 304 blocks of
    # 1024 threads: two teams of 16 warps each) gives the same x everywhere
    capi.amgdd_set_fac_kernel(s.h, 1, 31)
    x31 = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_iterate(s.h, bd, x31)
    assert np.array_equal(x31.cpu().numpy(), xg)
    s.close()


def test_batched64_four_columns_sampled():
    w = I.workload("batched_64", seed=0)
    nsys = len(w["edges"])
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], max_coarse=16 * nsys)
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
               precision=1, max_coarse=16 * nsys)
    best4, _ = capi.amgdd_autotune(s.h, 4, reps=1)
    best1, _ = capi.amgdd_autotune(s.h, 1, reps=1)
    # first and last box of a system of every edge length, and the batch's last box
    sub0 = np.concatenate([[0], np.cumsum([(e // 16) ** 3 for e in w["edges"]])])
    sample, seen = [], set()
    for k, e in enumerate(w["edges"]):
        if e not in seen:
            seen.add(e)
            sample += [int(sub0[k]), int(sub0[k + 1] - 1)]
    sample.append(int(w["nsub"] - 1))
    _check_maps(o, s, sample)
    Bh = w["B"]
    B = torch.from_numpy(np.ascontiguousarray(Bh)).cuda()
    X = torch.zeros_like(B)
    capi.amgdd_iterate_multi(s.h, B, X)
    Xg = X.cpu().numpy()
    for j in range(4):
        rl = o.restrict_all(o.residual(Bh[:, j], np.zeros(s.n)))
        for p in sample:
            own, ref = _owned_update(o, w, rl, p)
            assert np.array_equal(Xg[own, j], ref), (best4, j, p)
        x1 = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        capi.amgdd_iterate(s.h, B[:, j].contiguous(), x1)
        assert np.array_equal(x1.cpu().numpy(), Xg[:, j]), (best1, j)
    del o
    X.zero_()
    info = s.solve_multi(B, X, tol=1e-8, max_iter=100)
    assert info["converged"]
    A = sp.csr_matrix((w["val"], w["col"], w["rowptr"]), shape=(s.n, s.n))
    Xh = X.cpu().numpy()
    for j in range(4):
        rel = np.linalg.norm(Bh[:, j] - A @ Xh[:, j]) / np.linalg.norm(Bh[:, j])
        assert rel <= 1e-8 and np.isclose(rel, info["history"][j][-1], rtol=1e-6), j
    s.close()


@pytest.mark.parametrize("interp", ["direct", "exti"])
def test_aniso512_full_iteration_bit_exact(interp):
    """The 512^2 rotated-anisotropy workload at full size (256 composite
    grids): the oracle runs every grid here, so one AMG-DD iteration and one
    V-cycle are compared on every unknown, with direct and extended+i
    interpolation, in the autotuned launch configuration."""
    w = I.workload("aniso2d_512", seed=0)
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], interp=interp)
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=w["n_fac"],
               interp=interp)
    capi.amgdd_autotune(s.h, 1, reps=1)
    b = w["b"]
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_iterate(s.h, bd, x)
    assert np.array_equal(x.cpu().numpy(), o.amgdd_iteration(b, np.zeros(s.n), w["n_fac"]))
    x0 = np.random.default_rng(5).uniform(-1.0, 1.0, s.n)
    xv = torch.from_numpy(x0.copy()).cuda()
    capi.amg_vcycle(s.h, bd, xv)
    assert np.array_equal(xv.cpu().numpy(), o.vcycle_apply(b, x0))
    s.close()
