"""Pins of the oracle's composite grids (Section 3, eq. (1)) against closed
forms and a brute-force breadth-first search done with scipy's csgraph."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import amgdd_inputs as I
from oracle import Oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_level0_closed_form_sizes_2d():
    g = json.load(open(os.path.join(GOLD, "composite_level0_sizes.json")))
    case = [c for c in g["cases"] if c["dims"] == 2][0]
    rp, ci, v = I.poisson2d(64, 64)
    part, nsub = I.box_partition((64, 64), (case["box"],) * 2)
    o = Oracle(rp, ci, v, part, nsub, case["eta"])
    interior = [5, 6, 9, 10]
    for p in interior:
        nr, ng, no = o.comp_sizes(p, 0)
        assert (nr, nr + ng, no) == (case["D0"], case["Dbar0"], case["owned"])


def test_level0_closed_form_sizes_3d():
    g = json.load(open(os.path.join(GOLD, "composite_level0_sizes.json")))
    case = [c for c in g["cases"] if c["dims"] == 3][0]
    n = 48
    rp, ci, v = I.poisson3d(n, n, n)
    part, nsub = I.box_partition((n, n, n), (case["box"],) * 3)
    o = Oracle(rp, ci, v, part, nsub, case["eta"])
    p = 1 + 3 * (1 + 3 * 1)  # the centre box
    nr, ng, no = o.comp_sizes(p, 0)
    assert (nr, nr + ng, no) == (case["D0"], case["Dbar0"], case["owned"])


def _brute(o, part, nsub, eta):
    """Composite grids from all-pairs graph distances (scipy csgraph)."""
    out = {}
    L = o.nlev - 1
    dists = []
    for l in range(o.nlev):
        A = o.scipy(l)
        G = sp.csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape)
        G.setdiag(0)
        G.eliminate_zeros()
        dists.append(shortest_path(G, unweighted=True))
    cmaps = []
    for l in range(L):
        cf = o.cf(l).astype(bool)
        cm = np.full(len(cf), -1)
        cm[cf] = np.arange(cf.sum())
        cmaps.append((cf, cm))
    for p in range(nsub):
        owned = np.nonzero(part == p)[0]
        seeds = owned
        for l in range(o.nlev):
            if l < L:
                D = np.nonzero(dists[l][seeds].min(axis=0) <= eta)[0]
                bar = np.nonzero(dists[l][D].min(axis=0) <= 1)[0]
            else:
                D = np.arange(o.level_n[l])
                bar = D
            ghost = np.setdiff1d(bar, D)
            rest = np.setdiff1d(D, owned)
            out[(p, l)] = (np.concatenate([owned, rest, ghost]),
                           np.concatenate([np.zeros(len(owned)), np.ones(len(rest)),
                                           2 * np.ones(len(ghost))]).astype(np.uint8))
            if l < L:
                cf, cm = cmaps[l]
                seeds = cm[D[cf[D]]]
                owned = cm[owned[cf[owned]]]
    return out


@pytest.mark.parametrize("coarsen,interp", [("rs", "direct"), ("hmis", "exti")])
def test_composite_maps_match_bruteforce_2d(coarsen, interp):
    rp, ci, v = I.poisson2d(20, 18)
    part, nsub = I.box_partition((20, 18), (7, 6))
    for eta in (1, 2):
        o = Oracle(rp, ci, v, part, nsub, eta, coarsen=coarsen, interp=interp)
        ref = _brute(o, part, nsub, eta)
        for (p, l), (g, k) in ref.items():
            gg, kk = o.comp_map(p, l)
            assert np.array_equal(gg, g) and np.array_equal(kk, k), (p, l, eta)


@pytest.mark.parametrize("coarsen,interp", [("rs", "direct"), ("hmis", "exti")])
def test_composite_maps_match_bruteforce_3d(coarsen, interp):
    rp, ci, v = I.poisson3d(10, 9, 8)
    part, nsub = I.box_partition((10, 9, 8), (5, 5, 4))
    o = Oracle(rp, ci, v, part, nsub, 2, coarsen=coarsen, interp=interp)
    ref = _brute(o, part, nsub, 2)
    for (p, l), (g, k) in ref.items():
        gg, kk = o.comp_map(p, l)
        assert np.array_equal(gg, g) and np.array_equal(kk, k), (p, l)


def test_assumption_holds_on_workloads_and_overhead_definition():
    w = I.workload("poisson2d_64")
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"])
    assert o.violations() == 0
    # overhead: nnz of real rows over all grids / nnz of all A_l
    num = 0
    den = 0
    for l in range(o.nlev):
        A = o.scipy(l)
        den += A.nnz
        rl = np.diff(A.indptr)
        for p in range(w["nsub"]):
            g, k = o.comp_map(p, l)
            num += rl[g[k < 2]].sum()
    assert np.isclose(o.overhead(), num / den, rtol=1e-15)
    # one subdomain: the composite grid is the whole hierarchy
    o1 = Oracle(w["rowptr"], w["col"], w["val"], np.zeros(4096, np.int32), 1, 1)
    for l in range(o1.nlev):
        nr, ng, no = o1.comp_sizes(0, l)
        assert nr == o1.level_n[l] and ng == 0
