"""Host-side checks of the C-ABI library (no GPU needed).

* libamgdd.so loads and exports every function include/amgdd.h declares;
* the library's own setup (host_only) reproduces the oracle's hierarchy and
  composite-grid index maps bit for bit (both follow the same definitions,
  written independently);
* argument validation returns the documented status codes.
"""
import os
import re

import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle
from paper_1906_10575_gb300 import Solver, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "amgdd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(amgdd_\w+|amg_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    lib = capi.load()
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(capi.EXPORTS) == names


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    that a C compiler gives the header's structs, and the constants agree
    (status codes, AMGDD_MAX_LEVELS, AMGDD_FAC_CANDIDATES, tuning flag)."""
    import ctypes
    import subprocess
    structs = {"amgdd_csr": capi.amgdd_csr, "amgdd_options": capi.amgdd_options,
               "amgdd_setup_stats": capi.amgdd_setup_stats, "amgdd_solve_info": capi.amgdd_solve_info}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "amgdd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    consts = {"AMGDD_MAX_LEVELS": capi.MAX_LEVELS, "AMGDD_FAC_CANDIDATES": capi.FAC_CANDIDATES,
              "AMGDD_TUNE_ALLOW_REORDERED": capi.TUNE_ALLOW_REORDERED}
    consts.update({v: k for k, v in capi.STATUS.items()})
    for c in consts:
        lines.append('printf("const %s %%d\\n", (int)%s);' % (c, c))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
    for c, v in consts.items():
        assert got[("const", c)] == v, c


def _header_signatures():
    """name -> list of parameter kinds ('p' pointer, 'i32', 'i64', 'f64') of
    every function include/amgdd.h declares."""
    txt = open(os.path.join(ROOT, "include", "amgdd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(amgdd_\w+|amg_\w+)\s*\(([^)]*)\)\s*;", txt):
        kinds = []
        for prm in [q.strip() for q in m.group(2).split(",") if q.strip() and q.strip() != "void"]:
            if "*" in prm or prm.startswith("amgdd_handle"):
                kinds.append("p")
            elif prm.startswith("int32_t"):
                kinds.append("i32")
            elif prm.startswith("int64_t"):
                kinds.append("i64")
            elif prm.startswith("double"):
                kinds.append("f64")
            else:
                raise AssertionError("unclassified parameter %r of %s" % (prm, m.group(1)))
        out[m.group(1)] = kinds
    return out


def test_binding_argument_types_match_the_header():
    """Every declared function is bound with as many arguments as the header
    gives it, each of the same kind (pointer, 32- or 64-bit integer, double)."""
    import ctypes
    lib = capi.load()
    kind = {ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_double: "f64"}
    sigs = _header_signatures()
    assert sorted(sigs) == sorted(capi.EXPORTS)
    for name, want in sigs.items():
        got = [kind.get(t, "p") for t in getattr(lib, name).argtypes]
        assert got == want, (name, got, want)


def _pair(rp, ci, v, part, nsub, pad, **kw):
    o = Oracle(rp, ci, v, part, nsub, pad, **kw)
    s = Solver(rp, ci, v, part, nsub, pad, host_only=True, **kw)
    return o, s


CASES = [
    ("2d64_eta1", lambda: (*I.poisson2d(64, 64), *I.box_partition((64, 64), (16, 16)), 1)),
    ("2d45_eta2", lambda: (*I.poisson2d(45, 37), *I.box_partition((45, 37), (9, 10)), 2)),
    ("3d24_eta2", lambda: (*I.poisson3d(24, 24, 24), *I.box_partition((24, 24, 24), (8, 8, 8)), 2)),
    ("3d_kappa", lambda: (*I.diffusion3d(I.checkerboard_kappa(20, 4, 3)),
                          *I.box_partition((20, 20, 20), (10, 10, 5)), [2, 1])),
    ("2d_aniso", lambda: (*I.rotated_anisotropic2d(40, 36), *I.box_partition((40, 36), (10, 9)), 2)),
]


@pytest.mark.parametrize("coarsen,interp,pmax", [("rs", "direct", 4), ("rs", "exti", 4), ("rs", "exti", 0),
                                                  ("hmis", "direct", 4), ("hmis", "exti", 4)])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_hierarchy_and_maps_bit_exact(name, make, coarsen, interp, pmax):
    """Ruge-Stueben first pass or HMIS over the subdomains; direct and
    extended+i interpolation (truncated to 4 or untruncated)."""
    rp, ci, v, part, nsub, pad = make()
    o = Oracle(rp, ci, v, part, nsub, pad, interp=interp, pmax=pmax, coarsen=coarsen)
    s = Solver(rp, ci, v, part, nsub, pad, host_only=True, interp=interp, p_max=pmax, coarsen=coarsen)
    assert s.level_n == o.level_n
    for l in range(o.nlev):
        for which in ("A", "P", "R"):
            if which != "A" and l == o.nlev - 1:
                continue
            a = o.matrix(l, which)
            b = capi.amgdd_get_operator(s.h, l, which)
            assert a[3] == b[3]
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
            assert np.array_equal(a[2], b[2]), (l, which)  # bitwise values
        cf, l1 = capi.amgdd_get_cf(s.h, l, o.level_n[l], with_cf=l < o.nlev - 1)
        if l < o.nlev - 1:
            assert np.array_equal(cf, o.cf(l))
        assert np.array_equal(l1, o.l1inv(l))
    assert np.array_equal(capi.amgdd_get_coarse_inverse(s.h, o.level_n[-1]), o.ainv())
    for p in range(nsub):
        for l in range(o.nlev):
            g1, k1 = o.comp_map(p, l)
            g2, k2 = capi.amgdd_get_maps(s.h, p, l)
            assert np.array_equal(g1, g2) and np.array_equal(k1, k2), (p, l)
    assert s.stats.assumption_violations == o.violations()
    assert np.isclose(s.stats.composite_overhead, o.overhead(), rtol=1e-14)


def test_box_partition_matches_inputs():
    for shape, box in [((64, 64), (16, 16)), ((20, 18, 7), (7, 6, 4))]:
        p1, n1 = I.box_partition(shape, box)
        p2, n2 = capi.amgdd_box_partition(shape, box)
        assert n1 == n2 and np.array_equal(p1, p2)


def test_validation_errors():
    rp, ci, v = I.poisson2d(8, 8)
    part, nsub = I.box_partition((8, 8), (4, 4))
    bad = v.copy()
    bad[1] += 0.5                                   # break symmetry
    with pytest.raises(capi.AmgddError) as e:
        Solver(rp, ci, bad, part, nsub, 1, host_only=True)
    assert e.value.status == 2
    p2 = part.copy()
    p2[0] = nsub                                     # out of range
    with pytest.raises(capi.AmgddError) as e:
        Solver(rp, ci, v, p2, nsub, 1, host_only=True)
    assert e.value.status == 1
    with pytest.raises(capi.AmgddError) as e:       # empty subdomain
        Solver(rp, ci, v, part, nsub + 1, 1, host_only=True)
    assert e.value.status == 1
    ci2 = ci.copy()
    ci2[0], ci2[1] = ci[1], ci[0]                    # unsorted row
    with pytest.raises(capi.AmgddError) as e:
        Solver(rp, ci2, v, part, nsub, 1, host_only=True)
    assert e.value.status == 1
    with pytest.raises(capi.AmgddError) as e:       # coarsening option out of range
        Solver(rp, ci, v, part, nsub, 1, host_only=True, coarsen=2)
    assert e.value.status == 1
    s = Solver(rp, ci, v, part, nsub, 1, host_only=True)
    with pytest.raises(capi.AmgddError) as e:       # no device side
        capi.amgdd_iterate(s.h, None, None)
    assert e.value.status in (1, 9)


def test_hybrid_layouts_validate_on_host():
    """The composite grids of every sub-hierarchy (hybrid AMG-DD, Algorithm 3)
    pass the device-index range checks without a GPU; bad levels are refused."""
    rp, ci, v = I.poisson3d(20, 20, 20)
    part, nsub = I.box_partition((20, 20, 20), (10, 10, 5))
    s0 = Solver(rp, ci, v, part, nsub, 2, host_only=1)
    for lt in range(1, s0.nlev):
        s = Solver(rp, ci, v, part, nsub, 2, host_only=2, hybrid_level=lt)
        s.close()
    with pytest.raises(capi.AmgddError) as e:
        Solver(rp, ci, v, part, nsub, 2, host_only=2, hybrid_level=s0.nlev)
    assert e.value.status == 1


@pytest.mark.parametrize("precision,coarsen", [(0, "rs"), (1, "rs"), (0, "hmis")])
def test_streamed_layout_matches_whole_layout(precision, coarsen):
    """A device setup packs the composite-grid layout in chunks of grids and
    drops each chunk once it is checked and copied; host_only = 3 runs that
    same streamed packing and its per-chunk range checks without a GPU. With
    512 grids the layout spans several chunks; the streamed and the whole
    layout agree in every per-level entry count and in the FMA count."""
    rp, ci, v = I.poisson3d(40, 40, 40)
    part, nsub = I.box_partition((40, 40, 40), (5, 5, 5))
    whole = Solver(rp, ci, v, part, nsub, 2, host_only=2, precision=precision, coarsen=coarsen)
    streamed = Solver(rp, ci, v, part, nsub, 2, host_only=3, precision=precision, coarsen=coarsen)
    a, b = whole.stats, streamed.stats
    assert a.fac_fma == b.fac_fma > 0
    assert a.fac_entry_bytes == b.fac_entry_bytes == (6 if precision else 10)
    for l in range(a.num_levels):
        assert a.comp_nnz_A[l] == b.comp_nnz_A[l] > 0
        assert a.comp_nnz_P[l] == b.comp_nnz_P[l]
        assert a.comp_nnz_R[l] == b.comp_nnz_R[l]
    whole.close()
    streamed.close()


def test_streamed_layout_uneven_batch():
    """Block-diagonal batch of independent systems of different sizes (uneven
    boxes at the far ends): the streamed packing passes its checks, with the
    hybrid sub-hierarchy streamed as well."""
    rp, ci, v, part, nsub, B, picks, offs = I.batched_poisson(3, edges=(18, 24, 30), box=8, nrhs=1, seed=3)
    assert len(rp) - 1 == offs[-1] and nsub == sum(-(-e // 8) ** 3 for e in picks)
    s = Solver(rp, ci, v, part, nsub, 2, host_only=3, precision=1, hybrid_level=1)
    assert s.stats.fac_fma > 0
    s.close()
    # the same with HMIS: its composite grids pass the device-index checks too
    s = Solver(rp, ci, v, part, nsub, 2, host_only=3, precision=1, hybrid_level=1, coarsen="hmis")
    assert s.stats.fac_fma > 0
    s.close()


def test_fac_operation_count_only_extra_matvec():
    """Algorithm 4's only mat-vec beyond a V-cycle's is the coarse-residual
    recalculation f_{l+1} -= A_{l+1} u_{l+1}: skipped on the first downsweep
    (u_{l+1} = 0) and never on the finest grid. The library's executed-fma
    count over all composite grids must therefore be W1 + (n_fac - 1) W with
    W - W1 = the stored entries of A_l's real rows on every level l >= 1."""
    rp, ci, v = I.poisson3d(20, 20, 20)
    part, nsub = I.box_partition((20, 20, 20), (10, 10, 5))
    fma = {}
    for nfac in (1, 2, 3):
        s = Solver(rp, ci, v, part, nsub, 2, n_fac=nfac, host_only=2)
        st = s.stats
        fma[nfac] = st.fac_fma
        extra = sum(st.comp_nnz_A[l] for l in range(1, st.num_levels))
        s.close()
    assert extra > 0
    W1 = fma[1]
    W = fma[2] - fma[1]
    assert fma[3] - fma[2] == W
    assert W - W1 == extra


def test_device_entry_points_refuse_host_only_handles():
    """Every solve-phase entry point returns AMGDD_ERR_NOT_ON_DEVICE (9) on a
    handle set up with host_only, and option values out of range are refused
    at setup with AMGDD_ERR_INVALID_ARG (1); nothing needs a GPU."""
    import ctypes as C
    rp, ci, v = I.poisson2d(16, 16)
    part, nsub = I.box_partition((16, 16), (8, 8))
    s = Solver(rp, ci, v, part, nsub, 1, host_only=True)
    lib = capi.load()
    null = None
    calls = [
        lambda: lib.amgdd_fac(s.h, null, null, null),
        lambda: lib.amgdd_fac_multi(s.h, null, null, 4, null),
        lambda: lib.amgdd_iterate_multi(s.h, null, null, 4, null),
        lambda: lib.amgdd_solve_multi(s.h, null, null, 4, 1e-8, 10, null, null),
        lambda: lib.amgdd_set_fac_kernel(s.h, 1, 15),
        lambda: lib.amgdd_autotune(s.h, 1, 1, 0, null, null, null),
        lambda: lib.amg_vcycle(s.h, null, null, null),
        lambda: lib.amg_hybrid_cycle(s.h, null, null, null),
    ]
    for k, call in enumerate(calls):
        assert call() == 9, k
    assert lib.amgdd_autotune(None, 1, 1, 0, null, null, null) == 1
    s.close()
    for kw in ({"interp": 2}, {"p_max": -1}, {"precision": 2}, {"n_fac": 0}):
        with pytest.raises(capi.AmgddError) as e:
            Solver(rp, ci, v, part, nsub, 1, host_only=True, **kw)
        assert e.value.status == 1, kw


@pytest.mark.slow
def test_hmis_exti_hierarchy_and_maps_bit_exact_at_128cubed():
    """The paper's hierarchy flavour (HMIS over the 512 subdomains, extended+i
    truncated to 4) at the full size of the 128^3 benchmark workload: every
    level's operators and every composite grid's maps equal the oracle's."""
    w = I.workload("poisson3d_128")
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], coarsen="hmis", interp="exti")
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], host_only=1, coarsen="hmis",
               interp="exti")
    assert s.level_n == o.level_n
    for l in range(o.nlev):
        for which in ("A", "P", "R") if l < o.nlev - 1 else ("A",):
            a, b = o.matrix(l, which), capi.amgdd_get_operator(s.h, l, which)
            assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), (l, which)
    for p in range(w["nsub"]):
        for l in range(o.nlev):
            g1, k1 = o.comp_map(p, l)
            g2, k2 = capi.amgdd_get_maps(s.h, p, l)
            assert np.array_equal(g1, g2) and np.array_equal(k1, k2), (p, l)
    assert s.stats.assumption_violations == o.violations() == 0
    s.close()
