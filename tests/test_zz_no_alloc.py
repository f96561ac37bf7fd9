"""The allocation-free residual entry point against the oracle and against
the handle-based residual.

amgdd_residual_csr_noalloc exists for callers that cannot call cudaMalloc when
they need a residual (processes whose device memory was handed to their own
pool allocator, where a raw allocation fails or breaks the budget; loops that
cannot pay for an allocation's latency): it takes a device CSR the caller owns
and keeps its reduction scratch in a static device array. Every check runs
two calls in a row (the scratch keeps the previous call's partial sums):

* r equals the CPU oracle's residual bit for bit (each row is the same
  ascending fma chain) and the squared norm equals r.r within 1e-12
  relative (the reduction order differs), on a 2D Poisson matrix of
  1,229,881 rows: 301 blocks of 4096 rows, the last one partial;
* on a 3D case, r equals amgdd_residual of a set-up handle bit for bit;
* n = 0 gives a squared norm of exactly 0; n above the 16,777,216-row limit
  is refused before anything runs.
This file is collected last, so a failure here comes after every other test.
"""
import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import Solver, capi  # noqa: E402


def _dev_csr(rp, ci, v):
    return (torch.from_numpy(rp.astype(np.int32)).cuda(), torch.from_numpy(ci.astype(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(v, np.float64)).cuda())


def test_noalloc_residual_matches_oracle_twice_with_partial_last_block():
    rp, ci, v = I.poisson2d(1109, 1109)
    n = len(rp) - 1
    assert n % 4096 != 0 and n // 4096 + 1 >= 300
    o = Oracle(rp, ci, v)
    A = _dev_csr(rp, ci, v)
    rng = np.random.default_rng(12)
    for call in range(2):
        bh = rng.uniform(-1, 1, n)
        xh = rng.standard_normal(n)
        r = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        nrm = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        capi.amgdd_residual_csr_noalloc(n, *A, torch.from_numpy(bh).cuda(), torch.from_numpy(xh).cuda(), r, nrm)
        torch.cuda.synchronize()
        ro = o.residual(bh, xh)
        assert np.array_equal(r.cpu().numpy(), ro), call
        assert np.isclose(nrm.item(), ro @ ro, rtol=1e-12, atol=0), call


def test_noalloc_residual_matches_handle_residual_twice():
    rp, ci, v = I.poisson3d(40, 36, 30)
    part, nsub = I.box_partition((40, 36, 30), (10, 12, 10))
    n = len(rp) - 1
    s = Solver(rp, ci, v, part, nsub, 1)
    A = _dev_csr(rp, ci, v)
    rng = np.random.default_rng(11)
    for call in range(2):
        b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        r_ref = torch.empty_like(b)
        nrm_ref = capi.amgdd_residual(s.h, b, x, r_ref)
        r = torch.full_like(b, np.nan)
        nrm = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        capi.amgdd_residual_csr_noalloc(n, *A, b, x, r, nrm)
        torch.cuda.synchronize()
        assert torch.equal(r, r_ref), call
        assert np.isclose(nrm.item(), nrm_ref, rtol=1e-12, atol=0), call
    s.close()


def test_noalloc_empty_matrix_gives_zero_norm_twice():
    one_i = torch.zeros(1, dtype=torch.int32, device="cuda")
    one_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        nrm = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        capi.amgdd_residual_csr_noalloc(0, one_i, one_i, one_d, one_d, one_d, one_d, nrm)
        torch.cuda.synchronize()
        assert nrm.item() == 0.0


def test_noalloc_rejects_too_many_rows():
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    ti = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.AmgddError) as e:
        capi.amgdd_residual_csr_noalloc(16_777_217, ti, ti, t, t, t, t, t)
    assert e.value.status == 1
    assert "16,777,216" in str(e.value)
