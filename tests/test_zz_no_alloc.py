"""The allocation-free residual entry point against the handle-based one.

amgdd_residual_csr_noalloc exists for callers that cannot call cudaMalloc when
they need a residual (processes whose device memory was handed to their own
pool allocator, where a raw allocation fails or breaks the budget; loops that
cannot pay for an allocation's latency): it takes a device CSR the caller owns
and keeps its reduction scratch in a static device array. Two calls in a
row must each match amgdd_residual of a set-up handle: r bit for bit (same
ascending fma chain per row), the squared norm to 1e-12 relative (the block
partition of the reduction differs).
"""
import numpy as np
import pytest

import amgdd_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import Solver, capi  # noqa: E402


def test_noalloc_residual_matches_handle_residual_twice():
    rp, ci, v = I.poisson3d(40, 36, 30)
    part, nsub = I.box_partition((40, 36, 30), (10, 12, 10))
    n = len(rp) - 1
    s = Solver(rp, ci, v, part, nsub, 1)
    A_rp = torch.from_numpy(rp.astype(np.int32)).cuda()
    A_ci = torch.from_numpy(ci.astype(np.int32)).cuda()
    A_v = torch.from_numpy(v).cuda()
    rng = np.random.default_rng(11)
    for call in range(2):
        b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
        x = torch.from_numpy(rng.standard_normal(n)).cuda()
        r_ref = torch.empty_like(b)
        nrm_ref = capi.amgdd_residual(s.h, b, x, r_ref)
        r = torch.full_like(b, np.nan)
        nrm = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        capi.amgdd_residual_csr_noalloc(n, A_rp, A_ci, A_v, b, x, r, nrm)
        torch.cuda.synchronize()
        assert torch.equal(r, r_ref), call
        assert np.isclose(nrm.item(), nrm_ref, rtol=1e-12, atol=0), call
    s.close()


def test_noalloc_rejects_too_many_rows():
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    ti = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.AmgddError) as e:
        capi.amgdd_residual_csr_noalloc(16_777_217, ti, ti, t, t, t, t, t)
    assert e.value.status == 1
    assert "16,777,216" in str(e.value)
