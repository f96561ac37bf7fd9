"""Pins of the oracle's HMIS coarsening (the coarsening of the hypre defaults
that Section 6 names, after De Sterck, Yang and Heys 2006, with the
subdomains as the processors and SplitMix64 draws for PMIS's random numbers).

* SplitMix64 reproduces the published output sequence of its reference
  generator (seed 0).
* One subdomain: every point is interior, so HMIS is the Ruge-Stueben first
  pass and the whole hierarchy equals the default one bit for bit.
* One point per subdomain: no point is interior, so HMIS is PMIS; the
  splitting of every level equals PMIS written out here from its definition,
  and has the PMIS properties (C independent where the strength graph is
  symmetric, every F point either influences nobody or depends strongly on a
  C point).
* Box subdomains: the same properties; HMIS + extended+i (the paper's
  hierarchy) gives a symmetric Galerkin hierarchy, AlgFAC equals the masked
  global cycle (the equivalence principle of Section 4), and the solves match
  a dense direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import amgdd_inputs as I
from oracle import Oracle

M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(x):
    z = (x + GOLDEN) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_reference_sequence():
    # the generator's state after k steps from seed 0 is k * GOLDEN; its first
    # outputs, as published with the reference implementation
    assert [splitmix64(k * GOLDEN & M64) for k in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _strength(A, theta=0.25):
    """S_i: j != i with -a_ij >= theta * max_k(-a_ik), none when max <= 0."""
    A = A.tocsr()
    S = [[] for _ in range(A.shape[0])]
    for i in range(A.shape[0]):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        off = [(j, a) for j, a in zip(cols, vals) if j != i]
        m = max([-a for _, a in off], default=0.0)
        if m > 0:
            S[i] = sorted(j for j, a in off if -a >= theta * m)
    return S


def _pmis(S, level=0):
    """PMIS from its definition: C if ahead of every undecided strong
    neighbour in the order (|S_i^T|, SplitMix64 draw, smaller index)."""
    n = len(S)
    St = [[] for _ in range(n)]
    for i in range(n):
        for j in S[i]:
            St[j].append(i)
    key = [(len(St[i]), splitmix64((level << 40) + i), -i) for i in range(n)]
    state = ["U"] * n
    for i in range(n):
        if not St[i]:
            state[i] = "F"
    while True:
        for i in range(n):
            if state[i] == "U" and any(state[j] == "C" for j in S[i]):
                state[i] = "F"
        und = [i for i in range(n) if state[i] == "U"]
        if not und:
            break
        new_c = [i for i in und
                 if all(state[j] != "U" or key[i] > key[j] for j in set(S[i]) | set(St[i]) if j != i)]
        for i in new_c:
            state[i] = "C"
    return np.array([1 if s == "C" else 0 for s in state], dtype=np.int32)


def _check_pmis_properties(A, cf):
    """Every F point influences nobody or depends strongly on a C point; where
    the strength graph is symmetric, no two C points are strongly connected
    (with one-sided strength a C point may depend on a later one)."""
    S = _strength(A)
    St = [[] for _ in range(len(S))]
    for i in range(len(S)):
        for j in S[i]:
            St[j].append(i)
    symmetric = all(sorted(S[i]) == sorted(St[i]) for i in range(len(S)))
    for i in range(len(S)):
        if cf[i] == 0:
            assert not St[i] or any(cf[j] for j in S[i]), i
        elif symmetric:
            assert not any(cf[j] for j in S[i]), i
    return symmetric


PROBLEMS = [
    ("2d", lambda: (*I.poisson2d(30, 26), (30, 26), (10, 13))),
    ("3d", lambda: (*I.poisson3d(12, 12, 12), (12, 12, 12), (6, 6, 4))),
    ("kappa", lambda: (*I.diffusion3d(I.checkerboard_kappa(12, 3, 5)), (12, 12, 12), (6, 4, 6))),
    ("aniso", lambda: (*I.rotated_anisotropic2d(28, 24), (28, 24), (7, 8))),
]


@pytest.mark.parametrize("name,make", PROBLEMS, ids=[p[0] for p in PROBLEMS])
def test_one_subdomain_is_the_first_pass_hierarchy(name, make):
    rp, ci, v, shape, box = make()
    n = len(rp) - 1
    for interp in ("direct", "exti"):
        a = Oracle(rp, ci, v, np.zeros(n, np.int32), 1, 1, interp=interp)
        b = Oracle(rp, ci, v, np.zeros(n, np.int32), 1, 1, interp=interp, coarsen="hmis")
        assert a.level_n == b.level_n
        for l in range(a.nlev):
            for which in ("A", "P", "R") if l < a.nlev - 1 else ("A",):
                x, y = a.matrix(l, which), b.matrix(l, which)
                assert all(np.array_equal(p, q) for p, q in zip(x[:3], y[:3])), (interp, l, which)


@pytest.mark.parametrize("name,make", PROBLEMS, ids=[p[0] for p in PROBLEMS])
def test_one_point_per_subdomain_is_pmis(name, make):
    rp, ci, v, shape, box = make()
    n = len(rp) - 1
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    o = Oracle(rp, ci, v, np.arange(n, dtype=np.int32), n, 1, coarsen="hmis")
    # a C point keeps the subdomain of its fine point, so every point of every
    # level is still alone in its subdomain: PMIS on every level, with the
    # level's own draws
    assert o.nlev >= 3
    for l in range(o.nlev - 1):
        Al = A if l == 0 else o.scipy(l, "A")
        cf = o.cf(l)
        assert np.array_equal(cf, _pmis(_strength(Al), level=l)), l
        _check_pmis_properties(Al, cf)


@pytest.mark.parametrize("name,make", PROBLEMS, ids=[p[0] for p in PROBLEMS])
def test_box_subdomains_splitting_properties(name, make):
    rp, ci, v, shape, box = make()
    n = len(rp) - 1
    part, nsub = I.box_partition(shape, box)
    o = Oracle(rp, ci, v, part, nsub, 1, coarsen="hmis", interp="exti")
    for l in range(o.nlev - 1):
        _check_pmis_properties(o.scipy(l, "A"), o.cf(l))
    rs = Oracle(rp, ci, v, part, nsub, 1)
    # the subdomains change the splitting (boundary points go through PMIS)
    assert not np.array_equal(o.cf(0), rs.cf(0))


def test_hmis_exti_hierarchy_solves_and_algfac_equivalence():
    """The paper's hierarchy (HMIS + extended+i): symmetric Galerkin levels,
    AlgFAC equal to the global cycle relaxed only on D_l, solves equal to a
    dense solve."""
    nx, ny = 24, 20
    rp, ci, v = I.poisson2d(nx, ny)
    part, nsub = I.box_partition((nx, ny), (8, 10))
    b = I.uniform_rhs(nx * ny, 2)
    A = sp.csr_matrix((v, ci, rp))
    for interp in ("direct", "exti"):
        o = Oracle(rp, ci, v, part, nsub, 1, coarsen="hmis", interp=interp)
        for l in range(o.nlev):
            Al = o.scipy(l, "A")
            assert abs(Al - Al.T).max() <= 1e-14 * abs(Al).max()
        assert o.violations() == 0
        r0 = b.copy()
        rl = o.restrict_all(r0)
        for p in range(nsub):
            uf, ff = o.algfac(p, rl, 2)
            um, fm = o.masked_fac(p, r0, 2)
            for l in range(o.nlev):
                g, k = o.comp_map(p, l)
                real = g[k < 2]
                su = max(abs(um[l][g]).max(), 1e-300)
                sf = max(abs(fm[l][real]).max(), 1e-300)
                assert abs(uf[l][g] - um[l][g]).max() <= 1e-12 * su, (interp, p, l)
                assert abs(ff[l][real] - fm[l][real]).max() <= 1e-12 * sf, (interp, p, l)
        xd = np.linalg.solve(A.toarray(), b)
        x, h = o.amgdd_solve(b, 2, tol=1e-12, maxit=400)
        assert h[-1] <= 1e-12 and np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
