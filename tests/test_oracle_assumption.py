"""Pins of the connectivity-assumption check (Sections 4.2 and 4.5) against a
hand-derived case where it fails.

The assumption: a coarse point that Dbar_l reaches through P_l (equivalently
through the columns of R_l = P_l^T) but that lies outside Dbar_{l+1} must not
reach a real point of any coarser level through the interpolatory sets. The
golden `assumption_chain17.json` builds the situation Section 4.2 describes (a
fine point y with no interpolation connection between two injected C points,
so that A_{l+1} has no entry across y) on a 17-point chain, and derives by
hand the hierarchy and, for padding 0, 1 and 2, exactly which (subdomain,
level) pairs break the assumption. The oracle must reproduce that list; the
library must count the same pairs and, with strict_assumption, refuse the
setup with AMGDD_ERR_HIERARCHY_ASSUMPTION.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle
from paper_1906_10575_gb300 import Solver, capi

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "assumption_chain17.json")))


def _problem():
    rp, ci, v = I.weak_link_chain(8, 8)
    part = np.asarray(GOLD["part"], np.int32)
    return rp, ci, v, part, GOLD["nsub"]


def test_weak_link_chain_is_the_golden_matrix():
    rp, ci, v, _, _ = _problem()
    A = np.zeros((17, 17))
    for i in range(17):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    y = GOLD["matrix"]["y"]
    assert A[y, y] == 1.0 and A[y, y - 1] == A[y, y + 1] == 0.25
    assert np.array_equal(A, A.T)
    # irreducibly diagonally dominant (connected, dominant everywhere, strictly
    # on some rows) with a positive diagonal: symmetric positive definite
    off = np.abs(A - np.diag(np.diag(A))).sum(1)
    assert np.all(np.diag(A) >= off) and np.any(np.diag(A) > off)
    assert np.linalg.eigvalsh(A).min() > 0


def test_hierarchy_matches_hand_derivation():
    rp, ci, v, part, nsub = _problem()
    o = Oracle(rp, ci, v, part, nsub, 1, max_coarse=GOLD["max_coarse"])
    assert o.level_n == GOLD["level_n"]
    for l, cf in enumerate(GOLD["cf"]):
        assert o.cf(l).tolist() == cf, l
    for l, pat in enumerate(GOLD["P_pattern"]):
        prp, pci, _, _ = o.matrix(l, "P")
        got = [pci[prp[i]:prp[i + 1]].tolist() for i in range(len(prp) - 1)]
        assert got == pat, l
    A1 = o.scipy(1).toarray()
    diag = [float(Fraction(d)) if isinstance(d, str) else d for d in GOLD["A1_diag"]]
    assert np.allclose(np.diag(A1), diag, rtol=1e-15, atol=0)
    for a, b in GOLD["A1_blocks"]:
        for i in range(a, b):
            assert A1[i, i + 1] == A1[i + 1, i] == GOLD["A1_offdiag"]
    # block diagonal: nothing couples the two halves across y
    assert not np.any(A1[:4, 4:]) and not np.any(A1[4:, :4])


@pytest.mark.parametrize("eta", [0, 1, 2])
def test_oracle_violation_pairs_match_hand_derivation(eta):
    rp, ci, v, part, nsub = _problem()
    o = Oracle(rp, ci, v, part, nsub, eta, max_coarse=GOLD["max_coarse"])
    want = [tuple(x) for x in GOLD["violations"][str(eta)]]
    assert o.violation_pairs() == want
    assert o.violations() == len(want)


@pytest.mark.parametrize("eta", [0, 1, 2])
def test_library_counts_the_same_violations_and_maps(eta):
    rp, ci, v, part, nsub = _problem()
    s = Solver(rp, ci, v, part, nsub, eta, max_coarse=GOLD["max_coarse"], host_only=1)
    assert s.stats.assumption_violations == len(GOLD["violations"][str(eta)])
    o = Oracle(rp, ci, v, part, nsub, eta, max_coarse=GOLD["max_coarse"])
    for p in range(nsub):
        for l in range(o.nlev):
            g1, k1 = o.comp_map(p, l)
            g2, k2 = capi.amgdd_get_maps(s.h, p, l)
            assert np.array_equal(g1, g2) and np.array_equal(k1, k2), (p, l)
    s.close()


def test_strict_assumption_refuses_a_violating_setup():
    rp, ci, v, part, nsub = _problem()
    with pytest.raises(capi.AmgddError) as e:
        Solver(rp, ci, v, part, nsub, 1, max_coarse=GOLD["max_coarse"], host_only=1, strict_assumption=1)
    assert e.value.status == 3
    assert "connectivity assumption" in str(e.value)
    # the same option accepts a hierarchy that satisfies the assumption
    w = I.workload("poisson2d_64")
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], host_only=1,
               strict_assumption=1)
    assert s.stats.assumption_violations == 0
    s.close()

