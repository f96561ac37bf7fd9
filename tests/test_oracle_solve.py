"""Pins of the oracle's solve phase.

* AlgFAC (Algorithm 4) must reproduce the global cycle that relaxes only at
  the real points D_l (the equivalence principle stated at the start of
  Section 4), at every Dbar_l point for u_l and every D_l point for f_l.
* With one subdomain the composite grid is the whole hierarchy, so the masked
  cycle is the plain V-cycle (Algorithm 1) and one AMG-DD iteration from x = 0
  is n_fac V-cycles.
* Converged solutions match a dense direct solve; the V(1,1)-cycle with
  C-then-F pre- and F-then-C post-smoothing and R = P^T is a symmetric
  operator.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import amgdd_inputs as I
from oracle import Oracle


def _problem2d(nx, ny, box, eta, seed=0):
    rp, ci, v = I.poisson2d(nx, ny)
    part, nsub = I.box_partition((nx, ny), box)
    o = Oracle(rp, ci, v, part, nsub, eta)
    return o, sp.csr_matrix((v, ci, rp)), I.uniform_rhs(nx * ny, seed)


def _problem3d(n, box, eta, seed=0):
    rp, ci, v = I.poisson3d(n, n, n)
    part, nsub = I.box_partition((n, n, n), (box,) * 3)
    o = Oracle(rp, ci, v, part, nsub, eta)
    return o, sp.csr_matrix((v, ci, rp)), I.uniform_rhs(n ** 3, seed)


def test_residual_and_restriction_match_scipy():
    o, A, b = _problem2d(30, 30, (10, 10), 1)
    x = np.random.default_rng(3).standard_normal(900)
    r = o.residual(b, x)
    assert np.allclose(r, b - A @ x, rtol=0, atol=1e-13)
    rl = o.restrict_all(r)
    for l in range(o.nlev - 1):
        assert np.allclose(rl[l + 1], o.scipy(l, "R") @ rl[l], rtol=0, atol=1e-12)


def _aniso(nx, ny, box, eta, seed=0):
    rp, ci, v = I.rotated_anisotropic2d(nx, ny)
    part, nsub = I.box_partition((nx, ny), box)
    o = Oracle(rp, ci, v, part, nsub, eta)
    return o, sp.csr_matrix((v, ci, rp)), I.uniform_rhs(nx * ny, seed)


@pytest.mark.parametrize("kind,eta,nfac", [("2d", 1, 2), ("2d", 2, 3), ("3d", 1, 2), ("3d", 2, 1),
                                           ("aniso", 2, 2)])
def test_algfac_equals_masked_global_cycle(kind, eta, nfac):
    if kind == "2d":
        o, A, b = _problem2d(40, 36, (10, 9), eta)
    elif kind == "aniso":   # 9-point rotated anisotropy: positive off-diagonals, long-range coarse stencils
        o, A, b = _aniso(40, 36, (10, 9), eta)
    else:
        o, A, b = _problem3d(16, 8, eta)
    assert o.violations() == 0
    r0 = b.copy()
    rl = o.restrict_all(r0)
    for p in range(o.nsub):
        uf, ff = o.algfac(p, rl, nfac)
        um, fm = o.masked_fac(p, r0, nfac)
        for l in range(o.nlev):
            g, k = o.comp_map(p, l)
            real = g[k < 2]
            su = max(abs(um[l][g]).max(), 1e-300)
            sf = max(abs(fm[l][real]).max(), 1e-300)
            assert abs(uf[l][g] - um[l][g]).max() <= 1e-12 * su, (p, l)
            assert abs(ff[l][real] - fm[l][real]).max() <= 1e-12 * sf, (p, l)
            # nothing is written outside the composite grid
            mask = np.ones(o.level_n[l], bool)
            mask[g] = False
            assert not uf[l][mask].any() and not ff[l][mask].any()


def test_full_mask_is_the_vcycle():
    rp, ci, v = I.poisson2d(24, 20)
    o = Oracle(rp, ci, v, np.zeros(480, np.int32), 1, 1)
    b = I.uniform_rhs(480, 1)
    um, fm = o.masked_fac(0, b, 1)
    assert np.array_equal(um[0], o.vcycle_apply(b))
    # AMG-DD iteration from x = 0 with one composite grid == n_fac V-cycles;
    # AlgFAC recomputes the coarse right-hand sides (Section 4.4) instead of
    # restricting residuals, so the two agree to rounding, not bit for bit
    for nfac in (1, 2, 3):
        x1 = o.amgdd_iteration(b, np.zeros(480), nfac)
        xv = np.zeros(480)
        for _ in range(nfac):
            xv = o.vcycle_apply(b, xv)
        assert abs(x1 - xv).max() <= 1e-14 * abs(xv).max()
    # several subdomains whose padding covers the whole grid (eta >= the grid
    # diameter on every level): every composite grid is the whole hierarchy,
    # so the iteration equals the one-subdomain iteration bit for bit
    part, nsub = I.box_partition((24, 20), (12, 10))
    ow = Oracle(rp, ci, v, part, nsub, 50)
    assert all(ow.comp_sizes(p, l)[0] == ow.level_n[l] for p in range(nsub) for l in range(ow.nlev))
    for nfac in (1, 2):
        assert np.array_equal(ow.amgdd_iteration(b, np.zeros(480), nfac), o.amgdd_iteration(b, np.zeros(480), nfac))
    # whole histories agree up to that rounding, which grows relative to the
    # shrinking residual (about 1e-15 * ||A|| ||x|| / ||r_k||)
    _, hd = o.amgdd_solve(b, 1, tol=1e-10)
    _, hv = o.vcycle_solve(b, tol=1e-10)
    assert len(hd) == len(hv)
    assert np.allclose(hd, hv, rtol=1e-5, atol=0)


def test_vcycle_is_symmetric_and_contracts():
    o, A, b = _problem2d(33, 31, (11, 11), 1)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(A.shape[0])
    s = rng.standard_normal(A.shape[0])
    Vr = o.vcycle_apply(r)
    Vs = o.vcycle_apply(s)
    assert abs(Vr @ s - r @ Vs) <= 1e-12 * abs(Vr @ s)
    _, h = o.vcycle_solve(b, tol=1e-10)
    assert np.all(np.diff(h) < 0)
    assert h[-1] <= 1e-10


def test_converged_solutions_match_dense_solve():
    o, A, b = _problem2d(12, 12, (6, 6), 1, seed=2)
    xd = np.linalg.solve(A.toarray(), b)
    xv, hv = o.vcycle_solve(b, tol=1e-13, maxit=300)
    xa, ha = o.amgdd_solve(b, 2, tol=1e-13, maxit=300)
    for x in (xv, xa):
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.all(np.diff(ha) < 0)
    o3, A3, b3 = _problem3d(10, 5, 2, seed=1)
    xd = np.linalg.solve(A3.toarray(), b3)
    xa, ha = o3.amgdd_solve(b3, 2, tol=1e-12)
    assert np.linalg.norm(xa - xd) <= 1e-9 * np.linalg.norm(xd)
    oa, Aa, ba = _aniso(24, 20, (8, 10), 2, seed=4)
    xd = np.linalg.solve(Aa.toarray(), ba)
    for x, h in (oa.amgdd_solve(ba, 2, tol=1e-12, maxit=400), oa.vcycle_solve(ba, tol=1e-12, maxit=800)):
        assert h[-1] <= 1e-12 and np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_amgdd_history_definition():
    o, A, b = _problem2d(32, 32, (8, 8), 1)
    x, h = o.amgdd_solve(b, 2, tol=1e-8)
    assert h[0] == 1.0
    assert h[-1] <= 1e-8 and h[-2] > 1e-8
    assert np.isclose(h[-1], np.linalg.norm(b - A @ x) / np.linalg.norm(b), rtol=1e-6)
    # b = 0 normalises by the initial residual (the paper's random x0, zero rhs)
    x0 = np.random.default_rng(0).uniform(-1, 1, 1024)
    x, h = o.amgdd_solve(np.zeros(1024), 2, x0=x0, tol=1e-6)
    assert h[0] == 1.0 and h[-1] <= 1e-6


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_fp32_algfac_tracks_fp64_algfac(kind):
    """The FP32 cycle is the FP64 one up to single-precision rounding."""
    if kind == "2d":
        o, A, b = _problem2d(40, 36, (10, 9), 1)
    else:
        o, A, b = _problem3d(16, 8, 2)
    rl = o.restrict_all(b)
    for p in range(o.nsub):
        u64, f64 = o.algfac(p, rl, 2)
        u32, f32 = o.algfac32(p, rl, 2)
        for l in range(o.nlev):
            g, k = o.comp_map(p, l)
            su = abs(u64[l][g]).max()
            assert abs(u32[l][g] - u64[l][g]).max() <= 2e-5 * su, (p, l)
            # the FP32 result really is a different (rounded) computation
        assert not np.array_equal(u32[0], u64[0])


def test_mixed_precision_refinement_converges_to_fp64_solution():
    o, A, b = _problem2d(24, 24, (8, 8), 1, seed=3)
    xd = np.linalg.solve(A.toarray(), b)
    xm, hm = o.amgdd_solve(b, 2, tol=1e-11, mixed=True)
    x64, h64 = o.amgdd_solve(b, 2, tol=1e-11)
    assert np.linalg.norm(xm - xd) <= 1e-9 * np.linalg.norm(xd)
    assert abs(len(hm) - len(h64)) <= 2
    # early iterations: the FP32 correction is as good as the FP64 one
    assert np.allclose(hm[:4], h64[:4], rtol=1e-4)


def test_hybrid_limits_and_convergence():
    """Algorithm 3: switching to AMG-DD on level 0 is the AMG-DD iteration;
    switching on the coarsest level (stored whole in every composite grid)
    is the plain V-cycle; in between the cycle still solves the system."""
    o, A, b = _problem2d(40, 36, (10, 9), 1, seed=4)
    x0 = np.random.default_rng(1).standard_normal(o.n)
    assert np.array_equal(o.hybrid_apply(0, b, x0, 2), o.amgdd_iteration(b, x0, 2))
    L = o.nlev - 1
    assert np.array_equal(o.hybrid_apply(L, b, x0, 2), o.vcycle_apply(b, x0))
    xd = np.linalg.solve(A.toarray(), b)
    for lev0 in (1, 2):
        x, h = o.hybrid_solve(lev0, b, 2, tol=1e-12)
        assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
        assert np.all(np.diff(h) < 0)


@pytest.mark.parametrize("modes", [[(1, 1)], [(3, 2), (17, 11)]])
def test_dirichlet_eigenvector_right_hand_side_gives_v_over_lambda(modes):
    """b = sum of Dirichlet Laplacian eigenvectors v_ab (closed form, not a
    factorisation): both solvers must return sum v_ab / lambda_ab. The
    relative error is at most the relative residual times the condition
    number (209 on this grid): 2.1e-11 for a 1e-13 residual; the test allows
    2e-10."""
    nx, ny = 24, 20
    o, A, _ = _problem2d(nx, ny, (8, 10), 1)
    i = np.arange(1, nx + 1)[:, None]
    j = np.arange(1, ny + 1)[None, :]
    b = np.zeros(nx * ny)
    xe = np.zeros(nx * ny)
    for a, c in modes:
        # lexicographic numbering, i fastest: entry (i, j) is at i - 1 + nx (j - 1)
        v = (np.sin(a * np.pi * i / (nx + 1)) * np.sin(c * np.pi * j / (ny + 1))).T.ravel()
        lam = 4 - 2 * np.cos(a * np.pi / (nx + 1)) - 2 * np.cos(c * np.pi / (ny + 1))
        b += v
        xe += v / lam
    assert np.allclose(A @ xe, b, rtol=0, atol=1e-12)
    for x, h in (o.amgdd_solve(b, 2, tol=1e-13, maxit=400), o.vcycle_solve(b, tol=1e-13, maxit=800)):
        assert h[-1] <= 1e-13
        assert np.linalg.norm(x - xe) <= 2e-10 * np.linalg.norm(xe)
