"""Failure paths of the setup, driven from the host: no GPU fault is involved.

AMGDD_FAULT_ALLOC=k makes the k-th device or pinned allocation of one
amgdd_setup call fail as if memory were exhausted. Walking k over every
allocation of a setup, each call must return AMGDD_ERR_OOM with a message,
free what it had allocated (device free memory back where it started), and
leave the library usable: the next setup without injection solves to the
oracle's iterates.
"""
import os

import numpy as np
import pytest

import amgdd_inputs as I
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1906_10575_gb300 import Solver, capi  # noqa: E402


def test_every_setup_allocation_failure_is_clean():
    rp, ci, v = I.poisson2d(40, 36)
    part, nsub = I.box_partition((40, 36), (10, 12))
    b = I.uniform_rhs(40 * 36, 3)
    Solver(rp, ci, v, part, nsub, 1, hybrid_level=2).close()     # context and modules loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for k in range(1, 2000):
            os.environ["AMGDD_FAULT_ALLOC"] = str(k)
            try:
                s = Solver(rp, ci, v, part, nsub, 1, hybrid_level=2)
            except capi.AmgddError as e:
                assert e.status == 4, (k, str(e))            # AMGDD_ERR_OOM
                assert str(e), k
                failed += 1
                continue
            s.close()                                        # k past the last allocation
            break
    finally:
        os.environ.pop("AMGDD_FAULT_ALLOC", None)
    assert failed >= 20, failed                              # every allocation site was reached
    torch.cuda.synchronize()
    # a leak would keep at least one 1 MB staging buffer per failed setup
    assert torch.cuda.mem_get_info()[0] >= free0 - (16 << 20)
    o = Oracle(rp, ci, v, part, nsub, 1)
    s = Solver(rp, ci, v, part, nsub, 1)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    capi.amgdd_iterate(s.h, torch.from_numpy(b).cuda(), x)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), o.amgdd_iteration(b, np.zeros(len(b)), 2))
    s.close()
