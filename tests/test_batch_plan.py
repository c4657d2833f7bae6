"""Merged task tables of a batch of uneven matrices (host only): every access
stays inside the batch buffers, queue capacities hold, every task is
released once; and the merged table is exactly the union of the solo ones."""
import pytest

from paper_2504_19171_gb300 import stiles as S
from paper_2504_19171_gb300 import workloads as W

SMALL = [(16, 64, 1, 16), (5, 100, 2, 37), (3, 200, 2, 1), (30, 1, 1, 0), (4, 3, 1, 2), (1, 50, 0, 5), (7, 40, 4, 0)]


@pytest.mark.parametrize("prec", [S.STILES_FP64, S.STILES_EMU64, S.STILES_FP32X])
def test_batch_plan_validates(prec):
    assert S.stiles_debug_validate_batch(SMALL, prec) == S.STILES_OK


def test_batch_plan_validates_drawn_shapes():
    shapes = [(nt // 8 + 2, b // 8, w, a // 4) for nt, b, w, a in W.batch_shapes(12, seed=3)]
    assert S.stiles_debug_validate_batch(shapes, S.STILES_FP64) == S.STILES_OK


def test_batch_rejects_bad_shapes():
    assert S.stiles_debug_validate_batch([(0, 4, 1, 1)], 0) == S.STILES_ERR_INVALID_ARG
    assert S.stiles_debug_validate_batch([(3, 4, 1, -1)], 0) == S.STILES_ERR_INVALID_ARG


@pytest.mark.parametrize("tune", [0, 1, 2, 3, 4, 8, 16, 4 + 16, 3 + 8 + 16, 64, 64 + 3 + 8 + 16])
@pytest.mark.parametrize("prec", [S.STILES_FP64, S.STILES_EMU64])
def test_tuned_plans_validate_and_keep_the_work(tune, prec):
    for sh in [(7, 150, 2, 70), (16, 64, 1, 16), (3, 200, 2, 1)]:
        which = S.PLAN_FUSED + 16 * prec + 256 * tune
        assert S.stiles_debug_validate(*sh, which) == S.STILES_OK
        a = S.stiles_plan_stats(*sh, which, 152)
        b = S.stiles_plan_stats(*sh, S.PLAN_FUSED + 16 * prec, 152)
        assert a["flops"] == b["flops"] and a["tile_gemms"] == b["tile_gemms"]


def test_invalid_tuning_codes_are_rejected():
    for tune in (12, 32, 48, 128, 64 + 12, -1):
        assert S.stiles_debug_validate(7, 64, 1, 8, S.PLAN_FUSED + 256 * tune) == S.STILES_ERR_INVALID_ARG
    assert S.stiles_debug_validate_batch([(4, 64, 1, 8)], 0, [12]) == S.STILES_ERR_INVALID_ARG
    assert S.stiles_debug_validate_batch([(4, 64, 1, 8), (5, 30, 2, 3)], 0, [3, 8 + 16]) == S.STILES_OK


@pytest.mark.parametrize("shape", [(6, 64, 1, 16), (5, 100, 2, 37), (9, 40, 3, 0), (1, 50, 0, 5), (4, 3, 1, 2)])
@pytest.mark.parametrize("prec", [S.STILES_FP64, S.STILES_EMU64])
def test_serve_template_validates(shape, prec):
    """Request-server table: in bounds (the PREP tasks read the base values
    and the row-sum vectors behind them), PREP tasks are the only roots."""
    assert S.stiles_debug_validate_serve(*shape, prec, 0) == S.STILES_OK
    assert S.stiles_debug_validate_serve(*shape, prec, 2 + 8 + 16) == S.STILES_OK


def test_diagonal_tile_updates_stay_fp64_by_default():
    """In a reduced-precision plan the block updates inside each diagonal
    tile (the steps of that tile's POTRF) stay FP64 unless tuning bit 6
    lowers them: the lowered share is then exactly the diagonal tiles'
    POTRF work minus its block POTRF and block TRSM sweeps."""
    nt, b, w, a = 6, 192, 1, 40
    which = S.PLAN_FACTOR + 16 * S.STILES_EMU64
    keep = S.stiles_plan_stats(nt, b, w, a, which, 152)["flops_lowered"]
    low = S.stiles_plan_stats(nt, b, w, a, which + 256 * 64, 152)["flops_lowered"]
    R = b // 64  # blocks per diagonal tile; SYRK of a diagonal block m^2 k, GEMM of the others 2 m n k
    syrk = sum(64 ** 3 * r for r in range(R))  # block (r, r) receives r updates of m^2 k
    gemm = sum(2 * 64 ** 3 * c for r in range(R) for c in range(r))  # block (r, c), r > c, receives c updates
    assert low - keep == nt * (syrk + gemm)
    assert S.stiles_plan_stats(nt, b, w, a, S.PLAN_FACTOR, 152)["flops_lowered"] == 0
