"""Parity at the full 3D workload (128^3 Poisson, 512 subdomains of 16^3,
padding 2), in the launch configuration the benchmark times.

The oracle cannot run every composite grid in seconds at this size, so the
check samples: the composite maps of every subdomain and level (host), the
whole residual and restriction chain, and one AMG-DD iteration whose update
is compared on the owned points of sampled subdomains (interior, face, edge
and corner boxes) against the oracle's AlgFAC for exactly those subdomains.
The iteration runs with the FAC kernel the benchmark times (the autotuner's
choice; candidates 15 and 31, the one-block-per-grid kernel and the
work-sized warp teams, are its choices on this workload) as well as with the
single-column kernel (schedule 8).
"""
import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import Solver, capi  # noqa: E402


@pytest.fixture(scope="module")
def full():
    w = I.workload("poisson3d_128", seed=0)
    o = Oracle(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"])
    s = Solver(w["rowptr"], w["col"], w["val"], w["part"], w["nsub"], w["padding"], n_fac=2)
    yield w, o, s
    s.close()


def test_fullsize_maps_bit_exact(full):
    w, o, s = full
    assert s.level_n == o.level_n
    for p in range(w["nsub"]):
        for l in range(s.nlev):
            g1, k1 = o.comp_map(p, l)
            g2, k2 = capi.amgdd_get_maps(s.h, p, l)
            assert np.array_equal(g1, g2) and np.array_equal(k1, k2), (p, l)


def test_fullsize_one_iteration_sampled(full):
    w, o, s = full
    b = w["b"]
    bd = torch.from_numpy(b).cuda()
    tuned, _ = capi.amgdd_autotune(s.h, 1, reps=2)
    kernels = sorted({7, 15, 31, tuned})    # 7: the single-column kernel (schedule 8)
    xs = {}
    for k in kernels:
        capi.amgdd_set_fac_kernel(s.h, 1, k)
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        capi.amgdd_iterate(s.h, bd, x)
        torch.cuda.synchronize()
        xs[k] = x.cpu().numpy()
    # residual + restriction: whole vectors
    r_all = torch.zeros(int(s.offsets[-1]), dtype=torch.float64, device="cuda")
    capi.amgdd_residual(s.h, bd, torch.zeros_like(bd), r_all[:s.n])
    capi.amgdd_restrict(s.h, r_all)
    rl = o.restrict_all(o.residual(b, np.zeros(s.n)))
    assert np.array_equal(r_all.cpu().numpy(), np.concatenate(rl))
    # sampled subdomains: corner, edge, face, interior boxes
    nb = 8
    sample = [0, 3, 3 + nb * 3, 3 + nb * (3 + nb * 3), 511, 7 + nb * 4]
    xo = o.amgdd_iteration(b, np.zeros(s.n), 2, subset=sample)
    for k, xg in xs.items():
        for p in sample:
            own = np.nonzero(w["part"] == p)[0]
            assert np.array_equal(xg[own], xo[own]), (k, p)
        # everything outside the sample was updated once by its own grid, and
        # every kernel gives the same bits there too
        assert np.count_nonzero(xg) > 0.99 * s.n
        assert np.array_equal(xg, xs[kernels[0]]), k
