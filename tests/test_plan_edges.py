"""Size of the fused plan's dependency graph (host only).

Phase 1 of a tile column (Algorithm 2: L_ii^-1 and the U blocks) may start only
when every block of that column of L is final. Written as one dependency per
(phase-1 task, L block) pair, that costs (phase-1 tasks) x (L blocks) edges per
column, and each edge is one device atomic when its source task completes. The
fused plan joins each column once instead, so its graph stays within the factor
and selected-inversion plans' edges plus one edge per L block and one per
phase-1 task."""
import pytest

from paper_2504_19171_gb300 import stiles as S


@pytest.mark.parametrize("shape", [(4, 256, 1, 16), (4, 1024, 1, 64), (6, 1024, 2, 64), (3, 1024, 1, 0)])
def test_fused_edges_stay_linear(shape):
    fac = S.stiles_plan_stats(*shape, S.PLAN_FACTOR)
    sel = S.stiles_plan_stats(*shape, S.PLAN_SELINV)
    fus = S.stiles_plan_stats(*shape, S.PLAN_FUSED)
    # joins add at most one edge per L block (counted by the factor plan's
    # tasks, which write every L block) and one per phase-1 task
    assert fus["edges"] <= fac["edges"] + sel["edges"] + fac["tasks"] + sel["tasks"], (shape, fus, fac, sel)
    assert fus["edges"] < 8 * fus["tasks"], (shape, fus)


def test_edges_per_task_do_not_grow_with_tile_size():
    """Per-(task, L block) column waits would grow edges per task with the
    square of the blocks per tile; the joined graph does not."""
    ratios = []
    for b in (256, 512, 1024):
        st = S.stiles_plan_stats(4, b, 1, b // 16, S.PLAN_FUSED)
        ratios.append(st["edges"] / st["tasks"])
    assert max(ratios) < 2.0 * min(ratios), ratios


def test_edges_reported_for_every_plan_kind():
    """Every plan kind reports its edges; a plan with more than one task has
    at least one (the selected-inversion plan's panel waits, on counters with
    many writers, give it more edges per task than the fused plan)."""
    for which in (S.PLAN_FACTOR, S.PLAN_SELINV, S.PLAN_FUSED):
        st = S.stiles_plan_stats(3, 640, 1, 16, which)
        assert st["tasks"] > 1 and st["edges"] > 0, (which, st)
