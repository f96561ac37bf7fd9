"""Pins of the oracle's extended+i interpolation (the distance-two
interpolation of the hypre defaults named in Section 6), against properties
its definition fixes rather than a second copy of its formula:

* in 1D no F point has a strong F neighbour, so it must reproduce the
  hand-derived direct hierarchy of the 7-point chain exactly;
* a row of A with zero row sum interpolates constants exactly (row sum 1),
  on every level, with and without truncation;
* every untruncated F row solves the local equation that defines it: with
  e_i = sum_j w_ij e_j for arbitrary values e_j on the interpolatory set, the
  i-th equation sum_j a_ij e_j = 0 holds once each strong F neighbour's value
  is replaced by the average of its values on the interpolatory set and i
  weighted by its own opposite-sign entries (the "+i"), and weak connections
  take the value e_i; the interpolatory set is rebuilt here from the strength
  definition (strong C neighbours, plus the strong C neighbours of strong F
  neighbours);
* truncation keeps the largest |w| (at most pmax per row) and the row sum.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import amgdd_inputs as I
from oracle import Oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _strong(A, theta=0.25):
    """S[i] = strong influencers of i: -a_ij >= theta max_k(-a_ik), max > 0."""
    S = []
    for i in range(A.shape[0]):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        off = cols != i
        m = (-vals[off]).max() if off.any() else 0.0
        S.append(set(cols[off][-vals[off] >= theta * m]) if m > 0 else set())
    return S


def test_chain7_reproduces_the_direct_hierarchy():
    with open(os.path.join(GOLD, "chain7_hierarchy.json")) as f:
        g = json.load(f)
    n = g["matrix"]["n"]
    A = sp.diags([np.full(n - 1, g["matrix"]["off"]), np.full(n, g["matrix"]["diag"]),
                  np.full(n - 1, g["matrix"]["off"])], [-1, 0, 1]).tocsr()
    A.sort_indices()
    for pmax in (0, 2, 4):      # rows have at most 2 entries: no truncation
        o = Oracle(A.indptr, A.indices, A.data, max_coarse=g["max_coarse"], interp="exti", pmax=pmax)
        assert o.level_n == g["level_n"]
        for l in range(len(g["cf"])):
            assert np.array_equal(o.scipy(l, "P").toarray(), np.array(g["P"][l], float)), (pmax, l)


CASES = [("poisson2d", lambda: I.poisson2d(20, 18)), ("poisson3d", lambda: I.poisson3d(10, 9, 8)),
         ("aniso", lambda: I.rotated_anisotropic2d(20, 18)),
         ("kappa3d", lambda: I.diffusion3d(I.checkerboard_kappa(10, 2, 1)))]


@pytest.mark.parametrize("pmax", [0, 4])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_constants_interpolated_on_zero_row_sum_rows(name, make, pmax):
    o = Oracle(*make(), interp="exti", pmax=pmax)
    checked = 0
    for l in range(o.nlev - 1):
        A = o.scipy(l)
        P = o.scipy(l, "P")
        rs = np.asarray(A.sum(axis=1)).ravel()
        scale = abs(A).sum(axis=1).A.ravel()
        zero = np.abs(rs) <= 1e-14 * scale
        prs = np.asarray(P.sum(axis=1)).ravel()
        nz = np.diff(P.indptr) > 0
        sel = zero & nz
        assert np.allclose(prs[sel], 1.0, rtol=0, atol=1e-12), l
        if pmax:
            assert np.diff(P.indptr).max() <= pmax
        checked += sel.sum()
    assert checked > 0


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_untruncated_rows_solve_their_local_equation(name, make):
    o = Oracle(*make(), interp="exti", pmax=0)
    rng = np.random.default_rng(0)
    for l in range(min(2, o.nlev - 1)):
        A = o.scipy(l)
        P = o.scipy(l, "P")
        cf = o.cf(l).astype(bool)
        cidx = np.cumsum(cf) - 1            # fine -> coarse index of C points
        S = _strong(A)
        dense = A.toarray()
        for i in np.nonzero(~cf)[0]:
            Ci = {j for j in S[i] if cf[j]}
            Fi = {k for k in S[i] if not cf[k]}
            Chat = set(Ci)
            for k in Fi:
                Chat |= {j for j in S[k] if cf[j]}
            row = P.indices[P.indptr[i]:P.indptr[i + 1]]
            assert sorted(cidx[j] for j in Chat) == list(row), (l, i)
            if not Chat:
                continue
            Ch = sorted(Chat)
            e = dict(zip(Ch, rng.standard_normal(len(Ch))))
            w = dict(zip(Ch, P.data[P.indptr[i]:P.indptr[i + 1]]))
            ei = sum(w[j] * e[j] for j in Ch)
            e_ext = dict(e)
            e_ext[i] = ei
            lhs = dense[i, i] * ei
            scale = abs(dense[i, i] * ei)
            for n in np.nonzero(dense[i])[0]:
                if n == i:
                    continue
                a = dense[i, n]
                if n in Chat:
                    val = e[n]
                elif n in Fi:
                    pts = Ch + [i]
                    ab = np.array([dense[n, m] if dense[n, m] * dense[n, n] < 0 else 0.0 for m in pts])
                    den = ab.sum()
                    val = ab @ np.array([e_ext[m] for m in pts]) / den if den != 0 else ei
                else:
                    val = ei
                lhs += a * val
                scale += abs(a * val)
            assert abs(lhs) <= 1e-12 * scale, (l, i, lhs)


@pytest.mark.parametrize("name,make", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_truncation_keeps_largest_and_row_sum(name, make):
    full = Oracle(*make(), interp="exti", pmax=0)
    tr = Oracle(*make(), interp="exti", pmax=3)
    P0 = full.scipy(0, "P")
    P1 = tr.scipy(0, "P")
    for i in range(P0.shape[0]):
        c0 = P0.indices[P0.indptr[i]:P0.indptr[i + 1]]
        w0 = P0.data[P0.indptr[i]:P0.indptr[i + 1]]
        c1 = P1.indices[P1.indptr[i]:P1.indptr[i + 1]]
        w1 = P1.data[P1.indptr[i]:P1.indptr[i + 1]]
        if len(c0) <= 3:
            assert np.array_equal(c0, c1) and np.array_equal(w0, w1)
            continue
        order = sorted(range(len(c0)), key=lambda t: (-abs(w0[t]), c0[t]))[:3]
        assert list(c1) == sorted(c0[t] for t in order)
        assert np.isclose(w1.sum(), w0.sum(), rtol=1e-13)
        keep = np.isin(c0, c1)
        assert np.allclose(w1, w0[keep] * (w0.sum() / w0[keep].sum()), rtol=1e-14)


def test_exti_solves_match_dense_and_fac_equals_masked_cycle():
    for rp, ci, v, shape, box in [(*I.rotated_anisotropic2d(24, 20), (24, 20), (8, 10)),
                                  (*I.poisson3d(12, 12, 12), (12, 12, 12), (6, 6, 6))]:
        part, nsub = I.box_partition(shape, box)
        o = Oracle(rp, ci, v, part, nsub, 2, interp="exti", pmax=4)
        assert o.violations() == 0
        A = sp.csr_matrix((v, ci, rp))
        b = I.uniform_rhs(A.shape[0], 3)
        xd = np.linalg.solve(A.toarray(), b)
        for x, h in (o.amgdd_solve(b, 2, tol=1e-12, maxit=400), o.vcycle_solve(b, tol=1e-12, maxit=800)):
            assert h[-1] <= 1e-12 and np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
        rl = o.restrict_all(b)
        for p in range(o.nsub):
            uf, ff = o.algfac(p, rl, 2)
            um, fm = o.masked_fac(p, b, 2)
            for l in range(o.nlev):
                g, k = o.comp_map(p, l)
                su = max(abs(um[l][g]).max(), 1e-300)
                assert abs(uf[l][g] - um[l][g]).max() <= 1e-12 * su, (p, l)
