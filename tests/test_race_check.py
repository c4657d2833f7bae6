"""Host race check of the task tables (no GPU): every two task parts that
touch the same element, one of them writing it, are ordered by the
dependency graph the persistent kernel releases tasks from, and parts of one
task never conflict. Shapes cover ragged blocks (b not a multiple of 64),
several 64-blocks per tile (the split critical-path tasks), arrows, wide
bands; plans cover factor / selinv / fused, the reduced precisions (32 x 32
tensor parts), tuning codes and column-selected plans. A planted race (the
predecessors of one POTRF removed) must be found."""
import pytest

from paper_2504_19171_gb300 import stiles as S

SHAPES = [(6, 128, 2, 24), (4, 192, 1, 40), (8, 64, 3, 16), (3, 100, 2, 37), (5, 256, 1, 0), (1, 130, 0, 9),
          (7, 96, 6, 5)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kind", ["factor", "selinv", "fused"])
def test_plans_race_free(shape, kind):
    which = {"factor": S.PLAN_FACTOR, "selinv": S.PLAN_SELINV, "fused": S.PLAN_FUSED}[kind]
    assert S.stiles_debug_race_check(*shape, which) == S.STILES_OK


@pytest.mark.parametrize("precision", [S.STILES_EMU64, S.STILES_FP32X])
@pytest.mark.parametrize("tuning", [0, 64, 1 + 4 + 16, 2 + 8 + 64, 3])
def test_reduced_precision_and_tuned_plans_race_free(precision, tuning):
    for shape in [(6, 128, 2, 24), (3, 192, 1, 40)]:
        assert S.stiles_debug_race_check(*shape, S.PLAN_FUSED + 256 * tuning, precision) == S.STILES_OK, shape


def test_column_selected_plans_race_free():
    for shape in [(6, 128, 2, 24), (5, 192, 1, 8)]:
        for first in (1, 3, shape[0]):
            for kind in (S.PLAN_FUSED, S.PLAN_SELINV):
                assert S.stiles_debug_race_check(*shape, kind + (first << 16)) == S.STILES_OK, (shape, first)


@pytest.mark.parametrize("shape", [(6, 128, 2, 24), (4, 192, 1, 40), (3, 64, 1, 0)])
def test_planted_race_is_found(shape):
    for kind in (S.PLAN_FACTOR, S.PLAN_FUSED):
        assert S.stiles_debug_race_check(*shape, kind, plant=1) == S.STILES_ERR_PLAN


@pytest.mark.parametrize("shape", [(3, 640, 1, 16), (4, 576, 2, 9), (3, 200, 1, 0)])
@pytest.mark.parametrize("precision", [S.STILES_FP64, S.STILES_EMU64, S.STILES_FP32X])
def test_column_join_carries_the_phase1_order(shape, precision):
    """In a fused plan, phase 1 of a tile column follows that column of L only
    through the column's join task: with the edges into the first join
    removed, the column's first phase-1 read of L is unordered after its
    writer, and the check finds it."""
    assert S.stiles_debug_race_check(*shape, S.PLAN_FUSED, precision=precision) == S.STILES_OK
    assert S.stiles_debug_race_check(*shape, S.PLAN_FUSED, precision=precision, plant=2) == S.STILES_ERR_PLAN


def test_bad_arguments():
    assert S.stiles_debug_race_check(4, 64, 1, 0, S.PLAN_FUSED, plant=3) == S.STILES_ERR_INVALID_ARG
    assert S.stiles_debug_race_check(0, 64, 1, 0, S.PLAN_FUSED) == S.STILES_ERR_INVALID_ARG
    # factor and selected-inversion plans have no join task to plant a race in
    for kind in (S.PLAN_FACTOR, S.PLAN_SELINV):
        assert S.stiles_debug_race_check(4, 64, 1, 0, kind, plant=2) == S.STILES_ERR_INVALID_ARG


@pytest.mark.parametrize("shape", [(6, 128, 2, 24), (4, 192, 1, 40), (3, 100, 2, 37), (2, 64, 1, 0)])
@pytest.mark.parametrize("precision", [S.STILES_FP64, S.STILES_EMU64])
def test_serve_templates_race_free(shape, precision):
    """Request-server templates: the request's A is built in place in L by
    PREP tasks; every task touching a tile column of L (including the tasks
    that zero L's strict upper part) must come after that column's PREP."""
    assert S.stiles_debug_race_check_serve(*shape, precision) == S.STILES_OK


def test_serve_template_planted_race_is_found():
    assert S.stiles_debug_race_check_serve(4, 192, 1, 40, plant=1) == S.STILES_ERR_PLAN


@pytest.mark.parametrize("precision", [S.STILES_FP64, S.STILES_EMU64, S.STILES_FP32X])
def test_batch_tables_race_free(precision):
    """Merged batch tables: every matrix's tasks at its own offsets; no
    conflict inside a matrix or across matrices, with per-matrix tuning codes."""
    shapes = [(3, 128, 1, 16), (4, 64, 2, 0), (2, 192, 1, 40), (5, 96, 3, 7)]
    assert S.stiles_debug_race_check_batch(shapes, precision) == S.STILES_OK
    assert S.stiles_debug_race_check_batch(shapes, precision, tuning=[0, 4 + 16, 2 + 8, 1]) == S.STILES_OK


def test_batch_planted_race_is_found():
    shapes = [(3, 128, 1, 16), (2, 192, 1, 40)]
    assert S.stiles_debug_race_check_batch(shapes, plant=1) == S.STILES_ERR_PLAN
