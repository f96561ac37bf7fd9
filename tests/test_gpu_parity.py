"""GPU parity: every solve-phase step through the C ABI against the CPU oracle.

Both sides compute each sparse row product as the ascending fma chain, use
the same hierarchy (checked bit for bit on the host) and the same operation
order in Algorithms 1, 2 and 4, so iterates, residuals, restricted residuals
and AlgFAC states must be IDENTICAL. Only the residual norm is reduced in a
different order: its history is compared at 1e-12 relative, far inside the
1e-10-per-iteration target.
"""
import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import Solver, capi  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _case(name):
    if name == "poisson2d_64":
        w = I.workload("poisson2d_64", seed=0)
        return w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], w["b"]
    if name == "ragged2d":   # boxes that do not divide the grid, eta = 2
        rp, ci, v = I.poisson2d(45, 37)
        part, nsub = I.box_partition((45, 37), (9, 10))
        return rp, ci, v, part, nsub, 2, I.uniform_rhs(45 * 37, 1)
    if name == "poisson3d_24":
        rp, ci, v = I.poisson3d(24, 24, 24)
        part, nsub = I.box_partition((24, 24, 24), (8, 8, 8))
        return rp, ci, v, part, nsub, 2, I.uniform_rhs(24 ** 3, 2)
    if name == "kappa3d":    # variable coefficient, per-level padding
        rp, ci, v = I.diffusion3d(I.checkerboard_kappa(20, 4, 3))
        part, nsub = I.box_partition((20, 20, 20), (10, 10, 5))
        return rp, ci, v, part, nsub, [2, 1], I.uniform_rhs(8000, 3)
    if name == "one_grid":   # nsub = 1: the composite grid is the whole hierarchy
        rp, ci, v = I.poisson2d(33, 30)
        return rp, ci, v, np.zeros(990, np.int32), 1, 1, I.uniform_rhs(990, 4)
    if name == "eta0":       # no padding: D_0 = owned set
        rp, ci, v = I.poisson2d(40, 40)
        part, nsub = I.box_partition((40, 40), (10, 10))
        return rp, ci, v, part, nsub, 0, I.uniform_rhs(1600, 5)
    if name == "aniso2d":    # rotated anisotropic diffusion (theta = 3 pi / 16, eps = 1e-3), 9-point
        rp, ci, v = I.rotated_anisotropic2d(48, 40)
        part, nsub = I.box_partition((48, 40), (12, 10))
        return rp, ci, v, part, nsub, 2, I.uniform_rhs(48 * 40, 7)
    if name == "batch3":     # three independent systems, block diagonal, uneven boxes
        rp, ci, v, part, nsub, B, picks, offs = I.batched_poisson(3, edges=(12, 16, 20), box=8, nrhs=1, seed=5)
        return rp, ci, v, part, nsub, 2, B[:, 0].copy()
    if name == "single_level":  # n <= max_coarse: only the coarsest solve
        rp, ci, v = I.poisson2d(4, 3)
        part, nsub = I.box_partition((4, 3), (2, 3))
        return rp, ci, v, part, nsub, 1, I.uniform_rhs(12, 6)
    raise KeyError(name)


CASES = ["poisson2d_64", "ragged2d", "poisson3d_24", "kappa3d", "one_grid", "eta0", "single_level", "aniso2d"]


@pytest.fixture(scope="module", params=CASES)
def pair(request):
    rp, ci, v, part, nsub, pad, b = _case(request.param)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2)
    yield request.param, o, s, b
    s.close()


def test_residual_bit_exact(pair):
    _, o, s, b = pair
    x = np.random.default_rng(7).standard_normal(s.n)
    r = torch.empty(s.n, dtype=torch.float64, device="cuda")
    nrm2 = capi.amgdd_residual(s.h, _dev(b), _dev(x), r)
    ro = o.residual(b, x)
    assert np.array_equal(_host(r), ro)
    assert np.isclose(nrm2, ro @ ro, rtol=1e-13)


def test_restriction_bit_exact(pair):
    _, o, s, b = pair
    r_all = torch.zeros(int(s.offsets[-1]), dtype=torch.float64, device="cuda")
    r_all[:s.n] = _dev(b)
    capi.amgdd_restrict(s.h, r_all)
    got = _host(r_all)
    ref = np.concatenate(o.restrict_all(b))
    assert np.array_equal(got, ref)


def test_fac_states_and_update_bit_exact(pair):
    name, o, s, b = pair
    rl = o.restrict_all(b)
    r_all = _dev(np.concatenate(rl))
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_fac(s.h, r_all, x)
    for p in range(s.nsub):
        uo, fo = o.algfac(p, rl, 2)
        for l in range(s.nlev):
            g, k = capi.amgdd_get_maps(s.h, p, l)
            ug, fg = capi.amgdd_get_fac_state(s.h, p, l, len(g))
            assert np.array_equal(ug, uo[l][g]), (name, p, l)
            real = k < 2
            assert np.array_equal(fg[real], fo[l][g[real]]), (name, p, l)
    xo = o.amgdd_iteration(b, np.zeros(s.n), 2)
    assert np.array_equal(_host(x), xo)


def test_amgdd_solve_matches_oracle(pair):
    name, o, s, b = pair
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    info = s.solve(_dev(b), x, tol=1e-8, max_iter=100)
    xo, ho = o.amgdd_solve(b, 2, tol=1e-8, maxit=100)
    assert info["converged"] and info["iterations"] == len(ho) - 1
    assert np.array_equal(_host(x), xo)
    assert np.allclose(info["history"], ho, rtol=1e-12, atol=0)


def _expected_launches(s, iters):
    """Launches of an AMG-DD solve: |b|^2 (two launches), the first residual
    and restriction and the convergence check, then per iteration the FAC
    launch, the residual, the restriction and the check. Restrictions R_l
    with at most 4096 rows (n_{l+1}) run in one cluster launch; a fine level
    of at most 4096 rows has its residual, its norm and the check done by
    that launch too."""
    n = s.level_n
    if n[0] <= 4096:     # the chain launch also does the check
        return 3 + iters * 2
    big = sum(1 for l in range(len(n) - 1) if n[l + 1] > 4096)
    pre = 2 + big + (1 if big < len(n) - 1 else 0)
    return 3 + pre + iters * (2 + pre)


@pytest.mark.parametrize("name", ["poisson2d_64", "poisson3d_24"])
def test_iteration_launch_count(name):
    rp, ci, v, part, nsub, pad, b = _case(name)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2)
    try:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        info = s.solve(_dev(b), x, tol=1e-8, max_iter=100)
        assert info["kernel_launches"] == _expected_launches(s, info["iterations"])
        if name == "poisson2d_64":   # 64^2: two launches per iteration
            assert info["kernel_launches"] == 3 + 2 * info["iterations"]
    finally:
        s.close()


def test_vcycle_matches_oracle(pair):
    name, o, s, b = pair
    x0 = np.random.default_rng(8).standard_normal(s.n)
    x = _dev(x0)
    capi.amg_vcycle(s.h, _dev(b), x)
    assert np.array_equal(_host(x), o.vcycle_apply(b, x0))
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    info = s.vcycle_solve(_dev(b), x, tol=1e-8, max_iter=200)
    xo, ho = o.vcycle_solve(b, tol=1e-8, maxit=200)
    assert info["iterations"] == len(ho) - 1
    assert np.array_equal(_host(x), xo)
    assert np.allclose(info["history"], ho, rtol=1e-12, atol=0)


def test_zero_rhs_uses_initial_residual():
    rp, ci, v, part, nsub, pad, b = _case("poisson2d_64")
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad)
    x0 = np.random.default_rng(0).uniform(-1, 1, s.n)
    x = _dev(x0)
    info = s.solve(torch.zeros(s.n, dtype=torch.float64, device="cuda"), x, tol=1e-6)
    xo, ho = o.amgdd_solve(np.zeros(s.n), 2, x0=x0, tol=1e-6)
    assert info["history"][0] == 1.0 and info["iterations"] == len(ho) - 1
    assert np.array_equal(_host(x), xo)
    s.close()


def test_no_convergence_status_and_last_iterate():
    rp, ci, v, part, nsub, pad, b = _case("poisson2d_64")
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.AmgddError) as e:
        s.solve(_dev(b), x, tol=1e-30, max_iter=3)
    assert e.value.status == 6
    xo = np.zeros(s.n)
    for _ in range(3):
        xo = o.amgdd_iteration(b, xo, 2)
    assert np.array_equal(_host(x), xo)
    s.close()


@pytest.mark.parametrize("method", ["amgdd", "vcycle"])
def test_solve_graph_limits_and_recapture(method):
    """A whole solve is one graph whose iterations run in a device-side while
    node: max_iter = 0 runs no iteration (x unchanged, history[0] only, no
    convergence unless x_0 already meets tol); a solve is re-captured when
    tol or max_iter change, and each stops exactly where the oracle's history
    first meets its tolerance; a larger max_iter than any before grows the
    device history."""
    rp, ci, v, part, nsub, pad, b = _case("poisson2d_64")
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad)
    solve = s.solve if method == "amgdd" else s.vcycle_solve
    if method == "amgdd":
        _, ho = o.amgdd_solve(b, 2, tol=1e-12, maxit=300)
    else:
        _, ho = o.vcycle_solve(b, tol=1e-12, maxit=300)
    bd = _dev(b)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.AmgddError) as e:
        solve(bd, x, tol=1e-8, max_iter=0)
    assert e.value.status == 6 and not _host(x).any()
    for tol, max_iter in ((1e-4, 100), (1e-8, 100), (1e-8, 300), (1e-12, 300)):
        x.zero_()
        info = solve(bd, x, tol=tol, max_iter=max_iter)
        k = next(i for i, h in enumerate(ho) if h <= tol)
        assert info["iterations"] == k, (tol, max_iter)
        assert np.allclose(info["history"][:k + 1], ho[:k + 1], rtol=1e-12, atol=0)
        assert info["final_relres"] == info["history"][k]
    s.close()


@pytest.mark.parametrize("case", ["poisson3d_24", "ragged2d", "kappa3d"])
@pytest.mark.parametrize("schedule", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_fac_schedules_identical(schedule, case):
    """Every kernel variant (residency, unrolling, cp.async staging depth)
    gives the oracle's bits, states included."""
    rp, ci, v, part, nsub, pad, b = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=3, schedule=schedule)
    rl = o.restrict_all(b)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_fac(s.h, _dev(np.concatenate(rl)), x)
    xo = o.amgdd_iteration(b, np.zeros(s.n), 3)
    assert np.array_equal(_host(x), xo)
    for p in (0, nsub - 1):
        uo, fo = o.algfac(p, rl, 3)
        for l in range(s.nlev):
            g, k = capi.amgdd_get_maps(s.h, p, l)
            ug, fg = capi.amgdd_get_fac_state(s.h, p, l, len(g))
            assert np.array_equal(ug, uo[l][g]), (p, l)
            assert np.array_equal(fg[k < 2], fo[l][g[k < 2]]), (p, l)
    s.close()


def test_solve_twice_and_new_buffers_recapture():
    """The captured iteration graph is keyed by its vectors: new buffers
    re-capture, repeated calls reuse it; results stay identical."""
    rp, ci, v, part, nsub, pad, b = _case("poisson2d_64")
    s = Solver(rp, ci, v, part, nsub, pad)
    bd = _dev(b)
    outs = []
    for _ in range(2):
        for _ in range(2):
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            info = s.solve(bd, x, tol=1e-8)
            outs.append((_host(x), info["iterations"]))
        bd = _dev(b)
    for xo, it in outs[1:]:
        assert it == outs[0][1] and np.array_equal(xo, outs[0][0])
    s.close()


@pytest.mark.parametrize("case", ["poisson2d_64", "poisson3d_24", "kappa3d", "ragged2d"])
def test_mixed_precision_fac_and_solve_bit_exact(case):
    """FP32 AlgFAC inside FP64 refinement: GPU states, iterates and iteration
    count equal the oracle's mixed-precision path bit for bit."""
    rp, ci, v, part, nsub, pad, b = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, precision=1)
    rl = o.restrict_all(b)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_fac(s.h, _dev(np.concatenate(rl)), x)
    for p in range(s.nsub):
        uo, fo = o.algfac32(p, rl, 2)
        for l in range(s.nlev):
            g, k = capi.amgdd_get_maps(s.h, p, l)
            ug, fg = capi.amgdd_get_fac_state(s.h, p, l, len(g))
            assert np.array_equal(ug, uo[l][g]), (p, l)
            assert np.array_equal(fg[k < 2], fo[l][g[k < 2]]), (p, l)
    assert np.array_equal(_host(x), o.amgdd_iteration32(b, np.zeros(s.n), 2))
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    info = s.solve(_dev(b), x, tol=1e-8, max_iter=100)
    xo, ho = o.amgdd_solve(b, 2, tol=1e-8, maxit=100, mixed=True)
    assert info["iterations"] == len(ho) - 1
    assert np.array_equal(_host(x), xo)
    assert np.allclose(info["history"], ho, rtol=1e-12, atol=0)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nrhs", [2, 4])
@pytest.mark.parametrize("case", ["poisson2d_64", "poisson3d_24", "kappa3d", "batch3"])
def test_multi_rhs_columns_equal_single_column_solves(case, nrhs, precision):
    """Columns solved together follow exactly the single-column arithmetic:
    each column's iterate after k iterations equals the oracle's k
    iterations on that column alone."""
    rp, ci, v, part, nsub, pad, _ = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, precision=precision)
    n = s.n
    Bh = np.stack([I.uniform_rhs(n, 10 + j) for j in range(nrhs)], axis=1)
    B = torch.from_numpy(np.ascontiguousarray(Bh)).cuda()
    X = torch.zeros((n, nrhs), dtype=torch.float64, device="cuda")
    capi.amgdd_iterate_multi(s.h, B, X)
    Xh = _host(X)
    step = o.amgdd_iteration32 if precision else (lambda b, x, nf: o.amgdd_iteration(b, x, nf))
    for j in range(nrhs):
        assert np.array_equal(Xh[:, j], step(Bh[:, j], np.zeros(n), 2)), j
    X.zero_()
    info = s.solve_multi(B, X, tol=1e-8, max_iter=100)
    Xh = _host(X)
    k = info["iterations"]
    for j in range(nrhs):
        xo = np.zeros(n)
        for _ in range(k):
            xo = step(Bh[:, j], xo, 2)
        assert np.array_equal(Xh[:, j], xo), j
        _, ho = o.amgdd_solve(Bh[:, j], 2, tol=0.0, maxit=k, mixed=bool(precision))
        assert np.allclose(info["history"][j], ho, rtol=1e-12, atol=0), j
    assert info["converged"] and info["history"][:, -1].max() <= 1e-8
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["batch3", "kappa3d"])
def test_fac_multi_equals_oracle_corrections(case, precision):
    """The several-column FAC launch alone: from the restricted residuals of
    b_j (the residual of x = 0), column j of the correction equals the
    oracle's AMG-DD iteration on b_j from zero."""
    rp, ci, v, part, nsub, pad, _ = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, precision=precision)
    n = s.n
    Bh = np.stack([I.uniform_rhs(n, 20 + j) for j in range(4)], axis=1)
    Rh = np.stack([np.concatenate(o.restrict_all(Bh[:, j])) for j in range(4)], axis=1)
    assert Rh.shape[0] == int(s.offsets[-1])
    R = torch.from_numpy(np.ascontiguousarray(Rh)).cuda()
    X = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    capi.amgdd_fac_multi(s.h, R, X)
    Xh = _host(X)
    step = o.amgdd_iteration32 if precision else (lambda b, x, nf: o.amgdd_iteration(b, x, nf))
    for j in range(4):
        assert np.array_equal(Xh[:, j], step(Bh[:, j], np.zeros(n), 2)), j
    s.close()


@pytest.mark.parametrize("case", ["poisson2d_64", "poisson3d_24", "kappa3d", "ragged2d", "aniso2d"])
def test_hybrid_amgdd_bit_exact(case):
    """Hybrid AMG-DD (Algorithm 3) on every switch level equals the oracle's
    hybrid cycle; switching on the coarsest level is the plain V-cycle."""
    rp, ci, v, part, nsub, pad, b = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    L = o.nlev - 1
    x0 = np.random.default_rng(9).standard_normal(o.n)
    for lt in range(1, L + 1):
        s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, hybrid_level=lt)
        x = _dev(x0)
        capi.amg_hybrid_cycle(s.h, _dev(b), x)
        ref = o.hybrid_apply(lt, b, x0, 2)
        assert np.array_equal(_host(x), ref), lt
        if lt == L:
            assert np.array_equal(ref, o.vcycle_apply(b, x0))
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        info = s.hybrid_solve(_dev(b), x, tol=1e-8, max_iter=200)
        xo, ho = o.hybrid_solve(lt, b, 2, tol=1e-8, maxit=200)
        assert info["iterations"] == len(ho) - 1, lt
        assert np.array_equal(_host(x), xo), lt
        assert np.allclose(info["history"], ho, rtol=1e-12, atol=0), lt
        s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["poisson3d_24", "kappa3d", "batch3", "poisson2d_64"])
def test_every_fac_kernel_candidate_is_bit_exact(case, precision):
    """Every FAC kernel the autotuner may choose (the single-column schedules,
    the several-column kernel's variants, the kernel holding each grid's work
    vectors in shared memory and the one cycling each grid with a cluster of
    blocks, for 1, 2 and 4 columns) gives the oracle's iterate bit for bit;
    the autotuner keeps one of them and the solve after it is unchanged. On
    the 64^2 case every grid's vectors fit shared memory at every width and
    precision; the 3D cases take both paths of that kernel (on chip for one
    FP32 column, in global memory at four columns)."""
    rp, ci, v, part, nsub, pad, _ = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, precision=precision)
    n = s.n
    step = o.amgdd_iteration32 if precision else (lambda b, x, nf: o.amgdd_iteration(b, x, nf))
    Bh = np.stack([I.uniform_rhs(n, 30 + j) for j in range(4)], axis=1)
    ref = [step(Bh[:, j], np.zeros(n), 2) for j in range(4)]
    b = _dev(Bh[:, 0])
    single = [0, 7] if precision else list(range(9))
    several = list(range(9, 18)) + list(range(20, capi.FAC_CANDIDATES))
    exact = single + several    # 18, 19 reorder row sums: tested below
    for k in exact:
        capi.amgdd_set_fac_kernel(s.h, 1, k)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.amgdd_iterate(s.h, b, x)
        assert np.array_equal(_host(x), ref[0]), k
    for nrhs in (2, 4):
        B = torch.from_numpy(np.ascontiguousarray(Bh[:, :nrhs])).cuda()
        for k in several:
            capi.amgdd_set_fac_kernel(s.h, nrhs, k)
            X = torch.zeros((n, nrhs), dtype=torch.float64, device="cuda")
            capi.amgdd_iterate_multi(s.h, B, X)
            Xh = _host(X)
            for j in range(nrhs):
                assert np.array_equal(Xh[:, j], ref[j]), (nrhs, k, j)
    for k in ([1, 2, 3, 4, 5, 6, 8] if precision else []) + [capi.FAC_CANDIDATES, -1]:
        with pytest.raises(capi.AmgddError):
            capi.amgdd_set_fac_kernel(s.h, 1, k)
    with pytest.raises(capi.AmgddError):
        capi.amgdd_set_fac_kernel(s.h, 2, 3)      # single-column schedules take one column
    for nrhs in (1, 4):
        best, ms = capi.amgdd_autotune(s.h, nrhs, reps=2)
        applies = ms >= 0
        assert applies[best] and ms[best] <= 1.01 * ms[applies].min()
        assert not (applies[:best] & (ms[:best] <= 1.01 * ms[applies].min())).any()
        assert applies[9:18].all() and applies[20:].all() and not applies[18:20].any()
        assert applies[:9].any() == (nrhs == 1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    info = s.solve(b, x, tol=1e-8, max_iter=100)
    xo = np.zeros(n)
    for _ in range(info["iterations"]):
        xo = step(Bh[:, 0], xo, 2)
    assert np.array_equal(_host(x), xo)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["poisson3d_24", "kappa3d", "batch3"])
def test_group_per_row_candidates_within_tolerance(case, precision):
    """Candidates 18 and 19 (g lanes per row, the group adding its partial sums
    by an xor butterfly) reorder every row sum, so they are compared with the
    oracle within rounding: one AMG-DD iteration to 1e-12 relative (FP64) or
    1e-4 (FP32 composite grids), and a solve with the same number of
    iterations (FP64) whose relative residuals differ from the oracle's by at
    most 1e-10 (absolute; near 1e-8 a rounding-level change of the iterate,
    about 1e-16 |A| |x|, moves the relative residual by a few parts in 1e5 of
    itself, so a relative bound on the history would not hold for any other
    operation order). Columns solved together equal the one-column result of
    the same candidate bit for bit."""
    rp, ci, v, part, nsub, pad, _ = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, precision=precision)
    n = s.n
    step = o.amgdd_iteration32 if precision else (lambda b, x, nf: o.amgdd_iteration(b, x, nf))
    Bh = np.stack([I.uniform_rhs(n, 40 + j) for j in range(4)], axis=1)
    tol1 = 1e-4 if precision else 1e-12
    B = torch.from_numpy(np.ascontiguousarray(Bh)).cuda()
    for k in (18, 19):
        capi.amgdd_set_fac_kernel(s.h, 1, k)
        capi.amgdd_set_fac_kernel(s.h, 4, k)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        capi.amgdd_iterate(s.h, B[:, 0].contiguous(), x)
        xg = _host(x)
        xo = step(Bh[:, 0], np.zeros(n), 2)
        assert np.linalg.norm(xg - xo) <= tol1 * np.linalg.norm(xo), k
        X = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
        capi.amgdd_iterate_multi(s.h, B, X)
        assert np.array_equal(_host(X)[:, 0], xg), k
        x.zero_()
        info = s.solve(B[:, 0].contiguous(), x, tol=1e-8, max_iter=100)
        _, ho = o.amgdd_solve(Bh[:, 0], 2, tol=1e-8, maxit=100, mixed=bool(precision))
        assert info["converged"]
        if precision:
            assert abs(info["iterations"] - (len(ho) - 1)) <= 1, k
        else:
            assert info["iterations"] == len(ho) - 1, k
            assert np.all(np.abs(info["history"] - ho) <= 1e-10), k
            assert np.allclose(info["history"], ho, rtol=1e-4, atol=0), k
    best, ms = capi.amgdd_autotune(s.h, 1, reps=2, allow_reordered=True)
    assert ms[18] > 0 and ms[19] > 0 and ms[best] <= 1.01 * ms[ms >= 0].min()
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["aniso2d", "poisson3d_24", "batch3"])
def test_extended_i_hierarchy_solve_bit_exact(case, precision):
    """With extended+i interpolation (truncated to 4 per row) the GPU solve
    equals the oracle's on the same hierarchy bit for bit, FP64 and mixed."""
    rp, ci, v, part, nsub, pad, b = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad, interp="exti", pmax=4)
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, precision=precision, interp="exti", p_max=4)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    info = s.solve(_dev(b), x, tol=1e-8, max_iter=200)
    xo, ho = o.amgdd_solve(b, 2, tol=1e-8, maxit=200, mixed=bool(precision))
    assert info["converged"] and info["iterations"] == len(ho) - 1
    assert np.array_equal(_host(x), xo)
    assert np.allclose(info["history"], ho, rtol=1e-12, atol=0)
    xv = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    iv = s.vcycle_solve(_dev(b), xv, tol=1e-8, max_iter=400)
    xvo, hvo = o.vcycle_solve(b, tol=1e-8, maxit=400)
    assert iv["iterations"] == len(hvo) - 1 and np.array_equal(_host(xv), xvo)
    s.close()


@pytest.mark.parametrize("interp", ["direct", "exti"])
@pytest.mark.parametrize("case", ["poisson2d_64", "poisson3d_24", "kappa3d"])
def test_hmis_hierarchy_bit_exact(case, interp):
    """HMIS coarsening over the subdomains (the hierarchy of the hypre
    defaults that Section 6 names), with direct and extended+i interpolation:
    AlgFAC states of every grid and level, the AMG-DD solve (with the default
    FAC kernel and with candidate 15, the benchmark's) and the V-cycle solve
    equal the oracle's on the same hierarchy bit for bit."""
    rp, ci, v, part, nsub, pad, b = _case(case)
    o = Oracle(rp, ci, v, part, nsub, pad, interp=interp, pmax=4, coarsen="hmis")
    s = Solver(rp, ci, v, part, nsub, pad, n_fac=2, interp=interp, p_max=4, coarsen="hmis")
    assert s.level_n == o.level_n
    rl = o.restrict_all(b)
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    capi.amgdd_fac(s.h, _dev(np.concatenate(rl)), x)
    for p in range(s.nsub):
        uo, fo = o.algfac(p, rl, 2)
        for l in range(s.nlev):
            g, k = capi.amgdd_get_maps(s.h, p, l)
            ug, fg = capi.amgdd_get_fac_state(s.h, p, l, len(g))
            assert np.array_equal(ug, uo[l][g]), (p, l)
            assert np.array_equal(fg[k < 2], fo[l][g[k < 2]]), (p, l)
    assert np.array_equal(_host(x), o.amgdd_iteration(b, np.zeros(s.n), 2))
    xo, ho = o.amgdd_solve(b, 2, tol=1e-8, maxit=300)
    for cand in (7, 15):
        capi.amgdd_set_fac_kernel(s.h, 1, cand)
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        info = s.solve(_dev(b), x, tol=1e-8, max_iter=300)
        assert info["converged"] and info["iterations"] == len(ho) - 1, cand
        assert np.array_equal(_host(x), xo), cand
        assert np.allclose(info["history"], ho, rtol=1e-12, atol=0), cand
    xv = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    iv = s.vcycle_solve(_dev(b), xv, tol=1e-8, max_iter=400)
    xvo, hvo = o.vcycle_solve(b, tol=1e-8, maxit=400)
    assert iv["iterations"] == len(hvo) - 1 and np.array_equal(_host(xv), xvo)
    s.close()


def test_assumption_violating_hierarchy_on_device():
    """The hand-derived chain whose composite grids break the connectivity
    assumption of Sections 4.2 and 4.5 (tests/golden/assumption_chain17.json):
    with strict_assumption the device setup is refused with
    AMGDD_ERR_HIERARCHY_ASSUMPTION and leaves no device memory behind;
    without it, both sides drop the same points and the GPU solve equals the
    oracle's bit for bit at padding 0, 1 and 2."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "assumption_chain17.json")))
    rp, ci, v = I.weak_link_chain(8, 8)
    part = np.asarray(gold["part"], np.int32)
    nsub = gold["nsub"]
    b = I.uniform_rhs(len(rp) - 1, 3)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        with pytest.raises(capi.AmgddError) as e:
            Solver(rp, ci, v, part, nsub, 1, max_coarse=gold["max_coarse"], strict_assumption=1)
        assert e.value.status == 3
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for eta in (0, 1, 2):
        o = Oracle(rp, ci, v, part, nsub, eta, max_coarse=gold["max_coarse"])
        s = Solver(rp, ci, v, part, nsub, eta, max_coarse=gold["max_coarse"], n_fac=2)
        assert s.stats.assumption_violations == len(gold["violations"][str(eta)]) == o.violations()
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        info = s.solve(_dev(b), x, tol=1e-8, max_iter=100)
        xo, ho = o.amgdd_solve(b, 2, tol=1e-8, maxit=100)
        assert info["iterations"] == len(ho) - 1, eta
        assert np.array_equal(_host(x), xo), eta
        s.close()
