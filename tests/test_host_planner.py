"""The batch engine's launch planner (host logic, no GPU): pending phases of a
batch share one launch, cut into tiers of teams.  Checked on random batches
through the testing hook cd_debug_plan_launch."""
import numpy as np
import pytest

from paper_1304_4453_gb300 import cd


def _need(work, quantum, grid):
    q = -(-work // quantum)
    t = 1
    while t < q and t < grid:
        t <<= 1
    return min(t, grid)


def _check_plan(work, quantum, team_min, grid_max):
    grid, tiers, order = cd.cd_debug_plan_launch(work, quantum, team_min, grid_max)
    n = len(work)
    assert 1 <= grid <= grid_max
    assert sorted(order) == list(range(n))
    # tiers tile the grid and the run order, in sequence
    blk = team = run = 0
    for t in tiers:
        assert t["begin"] == blk and t["team0"] == team and t["first"] == run
        assert t["blocks"] >= 1 and t["team_size"] >= 1 and t["count"] >= 1
        assert t["blocks"] % t["team_size"] == 0
        blk += t["blocks"]
        team += t["blocks"] // t["team_size"]
        run += t["count"]
    assert blk == grid and run == n
    # runs in decreasing need, then decreasing work; one need per tier
    needs = [_need(work[i], quantum, grid_max) for i in order]
    keyed = [(needs[k], work[i]) for k, i in enumerate(order)]
    assert keyed == sorted(keyed, key=lambda x: (-x[0], -x[1]))
    for t in tiers:
        tier_needs = set(needs[t["first"]:t["first"] + t["count"]])
        assert len(tier_needs) == 1
        need = tier_needs.pop()
        # a team is as large as the tier's need unless the tier has fewer
        # blocks than its graphs (up to team_min of them) would need side by
        # side
        if t["blocks"] >= need * min(t["count"], team_min):
            assert t["team_size"] >= need
    return grid, tiers, order


@pytest.mark.parametrize("grid_max", [1, 2, 7, 152, 608, 1216])
@pytest.mark.parametrize("team_min", [1, 8, 32])
def test_random_batches(grid_max, team_min):
    rng = np.random.default_rng(grid_max * 100 + team_min)
    for trial in range(40):
        n = int(rng.integers(1, 600))
        work = (10 ** rng.uniform(1, 8.5, n)).astype(np.int64).tolist()
        quantum = int(2 ** rng.integers(10, 23))
        _check_plan(work, quantum, team_min, grid_max)


def test_single_graph_spans_the_grid():
    grid, tiers, order = _check_plan([120_000_000], 1 << 18, 8, 608)
    assert grid == 608 and len(tiers) == 1 and tiers[0]["team_size"] == 608


def test_equal_graphs_share_the_grid_in_teams_of_their_need():
    grid, tiers, order = _check_plan([1 << 20] * 512, 1 << 18, 8, 608)
    assert len(tiers) == 1 and tiers[0]["team_size"] == 4 and grid == 608


def test_blocks_follow_the_work():
    # one heavy tier and one light tier: the heavy one gets most blocks
    grid, tiers, order = _check_plan([1 << 27] + [1000] * 64, 1 << 18, 8, 608)
    heavy = [t for t in tiers if order[t["first"]] == 0][0]
    assert heavy["blocks"] > 500


def test_invalid_arguments():
    for args in (([], 1, 1, 1), ([5], 0, 1, 1), ([5], 1, 0, 1), ([5], 1, 1, 0)):
        with pytest.raises(cd.CDError):
            cd.cd_debug_plan_launch(*args)
