"""The flop count behind every TFLOP/s figure.

The closed form (``oracle/flops.py``) is pinned to textbook counts and to a
count by hand of the n = 204,864 benchmark matrix; the library's planner
(``stiles_plan_stats``, whose count the bench divides by the measured time)
must reproduce it for every plan kind on shapes with ragged tiles, clipped
bands, no arrow and a full band."""
import pytest

from oracle import flops as F
from paper_2504_19171_gb300 import build as B


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_2504_19171_gb300 import stiles
    return stiles


@pytest.mark.parametrize("nt,b", [(1, 7), (3, 5), (6, 64), (9, 33)])
def test_full_band_gives_dense_counts(nt, b):
    # a full band without an arrow is a dense SPD matrix of order n = nt b:
    # Cholesky n^3/3 (LAPACK POTRF), inverse from the factor 2 n^3/3 (TRTRI + LAUUM)
    n = nt * b
    assert F.flops(nt, b, nt - 1, 0, "factor") == pytest.approx(n ** 3 / 3, rel=1e-15)
    assert F.flops(nt, b, nt - 1, 0, "selinv") == pytest.approx(2 * n ** 3 / 3, rel=1e-15)
    # the arrow of height b is one more dense tile row: still dense, order n + b
    assert F.flops(nt, b, nt - 1, b, "factor") == pytest.approx((n + b) ** 3 / 3, rel=1e-15)
    assert F.flops(nt, b, nt - 1, b, "selinv") == pytest.approx(2 * (n + b) ** 3 / 3, rel=1e-15)


def test_block_diagonal_counts():
    # independent diagonal tiles: one POTRF and one TRTRI + LAUUM each
    assert F.flops(10, 12, 0, 0, "factor") == pytest.approx(10 * 12 ** 3 / 3)
    assert F.flops(10, 12, 0, 0, "selinv") == pytest.approx(10 * 2 * 12 ** 3 / 3)


def test_benchmark_matrix_by_hand():
    # n = 204,864 (nt 200, b 1024, w 1, a 64), counted by hand per tile column:
    # 199 columns with one band tile below and the arrow, the last with the arrow only
    b, a = 1024, 64
    col_f = lambda nb: b**3 / 3 + (nb * b + a) * b * b + (nb * b * b + a * a) * b + 2 * b * (nb * a * b)
    col_s = lambda nb: 2 * b**3 / 3 + (nb * b + a) * b * b + 2 * b * (nb * b + a) ** 2 + b * b * (nb * b + a)
    fac = 199 * col_f(1) + col_f(0) + a**3 / 3
    sel = 199 * col_s(1) + col_s(0) + 2 * a**3 / 3
    assert F.flops(200, b, 1, a, "factor") == pytest.approx(fac, rel=1e-15)
    assert F.flops(200, b, 1, a, "selinv") == pytest.approx(sel, rel=1e-15)
    assert round(F.flops(200, b, 1, a)) == 1_619_706_249_216
    assert round(F.flops(200, b, 1, a, "factor") / 1e9, 1) == 539.9
    assert round(F.flops(200, b, 4, a) / 1e12, 2) == 13.27


def test_gemm_terms_grow_with_pairs():
    # one more band tile below every column adds its products with every other
    # band tile and the arrow: the difference between w = 2 and w = 1 at nt = 3
    # (one column gains a tile) is worked out term by term
    b, a = 4, 3
    d = F.flops(3, b, 2, a, "selinv") - F.flops(3, b, 1, a, "selinv")
    m1, m2 = b + a, 2 * b + a  # rows below column 0 at w = 1 and w = 2
    assert d == pytest.approx((m2 - m1) * b * b + 2 * b * (m2**2 - m1**2) + b * b * (m2 - m1))


SHAPES = [(16, 64, 1, 16), (7, 100, 3, 37), (5, 10, 0, 0), (1, 8, 0, 3), (3, 5, 2, 0), (10, 33, 9, 5),
          (6, 64, 5, 64), (12, 96, 4, 70), (40, 1024, 4, 64)]


@pytest.mark.parametrize("shape", SHAPES)
def test_planner_count_matches_closed_form(S, shape):
    for which, kind in ((S.PLAN_FACTOR, "factor"), (S.PLAN_SELINV, "selinv"), (S.PLAN_FUSED, "fused")):
        got = S.stiles_plan_stats(*shape, which, workers=152)["flops"]
        want = F.flops(*shape, kind)
        assert abs(got - want) <= 2 + 1e-12 * want, (shape, kind, got, want)


def test_planner_count_benchmark_matrix(S):
    got = S.stiles_plan_stats(200, 1024, 1, 64, S.PLAN_FUSED, workers=152)["flops"]
    assert abs(got - 1_619_706_249_216) <= 2
