"""Host tests of the team plan of FAC candidate 31 (amgdd_plan_teams; no GPU).

The teams kernel splits blocks of 1024 threads (32 warps) into teams of
whole warps that wait on named barriers 1..15; a plan that gave a block more
than 15 teams or 32 warps, overlapping warps, or a grid twice or not at all
would hang or fault the kernel or skip work, so these invariants are checked
here on the host (setup also checks them before any launch).
"""
import numpy as np
import pytest

from paper_1906_10575_gb300 import capi


def _check_invariants(plan, nsub):
    seen = np.zeros(nsub, np.int64)
    for teams in plan:
        assert len(teams) <= 15
        end = 0
        for w0, nw, grids in teams:
            assert nw >= 1 and w0 >= end and w0 + nw <= 32
            end = w0 + nw
            for g in grids:
                seen[g] += 1
    assert (seen == 1).all()


def _box_work(nb):
    """Per-grid work of an nb^3 box partition: interior boxes 1000, each
    clipped side takes a share away (a face box, an edge box, a corner box)."""
    w = []
    for i in range(nb):
        for j in range(nb):
            for k in range(nb):
                sides = sum(c in (0, nb - 1) for c in (i, j, k))
                w.append(1000 - 150 * sides)
    return np.array(w, np.int64)


def test_one_grid_per_team_balances_work():
    w = _box_work(8)                       # 512 grids: 16^3 boxes of a 128^3 grid
    nblocks = 304                          # two blocks of 1024 threads per SM
    plan = capi.amgdd_plan_teams(w, nblocks)
    _check_invariants(plan, len(w))
    per_warp = []
    for teams in plan:
        if teams:
            assert sum(nw for _, nw, _ in teams) == 32     # no warp of a used block idle
        for _, nw, grids in teams:
            assert len(grids) == 1
            per_warp.append(w[grids[0]] / nw)
    # the largest per-warp load is below that of one 512-thread block per grid
    # (16 warps for the largest grid) and not below the ideal spread
    ideal = w.sum() / (32 * nblocks)
    assert ideal <= max(per_warp) < 0.95 * w.max() / 16
    # within a block, more work never gets fewer warps
    for teams in plan:
        ws = [(w[g[0]], nw) for _, nw, g in teams]
        for a in ws:
            for b in ws:
                if a[0] > b[0]:
                    assert a[1] >= b[1]


def test_many_grids_get_lists_on_two_teams_per_block():
    rng = np.random.default_rng(1)
    w = rng.integers(100, 2000, size=6083).astype(np.int64)
    plan = capi.amgdd_plan_teams(w, 304)
    _check_invariants(plan, len(w))
    loads = []
    for teams in plan:
        assert [(w0, nw) for w0, nw, _ in teams] == [(0, 16), (16, 16)]
        for _, _, grids in teams:
            loads.append(w[grids].sum())
            # largest grids first within a list
            assert (np.diff(w[grids]) <= 0).all()
    # longest-processing-time order: loads differ by at most one grid's work
    assert max(loads) - min(loads) <= w.max()


@pytest.mark.parametrize("nsub,nblocks", [(1, 1), (1, 304), (2, 1), (3, 1), (15, 8), (608, 304), (609, 304)])
def test_edge_sizes(nsub, nblocks):
    w = np.arange(1, nsub + 1, dtype=np.int64) * 7
    plan = capi.amgdd_plan_teams(w, nblocks)
    _check_invariants(plan, nsub)


def test_zero_work_grids_still_planned():
    w = np.zeros(40, np.int64)
    _check_invariants(capi.amgdd_plan_teams(w, 16), 40)


def test_invalid_arguments():
    with pytest.raises(capi.AmgddError):
        capi.amgdd_plan_teams(np.zeros(0, np.int64), 4)
    with pytest.raises(capi.AmgddError):
        capi.amgdd_plan_teams(np.array([1, -1], np.int64), 4)
    with pytest.raises(capi.AmgddError):
        capi.amgdd_plan_teams(np.array([1, 2], np.int64), 0)
