"""General selections (Sec. III-B, Fig. 2): pruning a selection to the tile
columns it needs, and the full inverse (case 6) as the pattern with the band
widened to every tile. Host-side checks and oracle pins (no GPU)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import stiles as S
from paper_2504_19171_gb300 import workloads as W


def test_sigma_of_later_columns_does_not_depend_on_earlier_columns_of_L():
    """The pruning rule, pinned on the oracle: Sigma tiles of columns >= i0
    are unchanged when every L tile of columns < i0 is replaced."""
    M = W.random_arrowhead(7, 5, 2, 3, seed=11)
    L = O.cholesky(M)
    S_ref = O.selinv_from_factor(M, L)
    i0 = 3
    L2 = {k: v.copy() for k, v in L.items()}
    rng = np.random.default_rng(0)
    for (i, k), T in L2.items():
        if k < i0:
            T[...] = rng.standard_normal(T.shape) + (np.eye(*T.shape) * 5 if i == k else 0)
    S2 = O.selinv_from_factor(M, L2)
    for (i, k), T in S_ref.items():
        if k >= i0:
            assert np.array_equal(S2[(i, k)], T), (i, k)
    assert any(not np.array_equal(S2[key], S_ref[key]) for key in S_ref if key[1] < i0)


def test_full_pattern_is_the_dense_inverse():
    """Case 6 on the oracle: with the band widened to every tile the method
    returns the whole inverse."""
    M = W.random_arrowhead(6, 4, 1, 3, seed=2)
    F = S.widen_band(M)
    _, Sf, _ = O.selinv(F)
    inv = np.linalg.inv(M.to_dense())
    for (i, k), T in Sf.items():
        r0, c0 = i * M.b, k * M.b
        assert np.allclose(T, inv[r0:r0 + T.shape[0], c0:c0 + T.shape[1]], atol=1e-13, rtol=0)


@pytest.mark.parametrize("shape", [(9, 130, 1, 70), (16, 64, 1, 16), (7, 40, 4, 0)])
def test_selected_plans_validate_and_shrink(shape):
    nt, b, w, a = shape
    last = nt if a > 0 else nt - 1
    prev = None
    for sel0 in range(0, last + 1, max(1, last // 4)):
        which = S.PLAN_FUSED + 65536 * sel0
        assert S.stiles_debug_validate(*shape, which) == S.STILES_OK
        st = S.stiles_plan_stats(*shape, which, 152)
        if prev is not None:
            assert st["tasks"] < prev["tasks"] and st["flops"] < prev["flops"]
        prev = st
    assert S.stiles_plan_stats(*shape, S.PLAN_FUSED, 152) == S.stiles_plan_stats(*shape, S.PLAN_FUSED + 0, 152)
    assert S.stiles_debug_validate(*shape, S.PLAN_FUSED + 65536 * (last + 1)) == S.STILES_ERR_INVALID_ARG


def test_first_column_for_entries():
    nt, b = 10, 8
    assert S.first_column_for([(79, 3), (40, 41)], nt, b) == 0
    assert S.first_column_for([(47, 41), (60, 80)], nt, b) == 5
    assert S.first_column_for([(85, 83)], nt, b) == nt  # arrow x arrow: the corner column only


def test_update_runs_only_in_full_fused_plans():
    """The planner merges far one-block-column update terms into runs only in
    a fused plan of every column: that plan has fewer tasks than the factor
    and selected-inversion plans together, while a column-selected fused plan
    has exactly their sum (single terms) plus one join task per selected column
    of L (tile columns first .. nt-1 and the arrow column: the point where that
    column of L is final). Every one of these plans validates (satisfiable
    waits, in-bounds accesses)."""
    from paper_2504_19171_gb300 import stiles as S
    for shape in [(3, 640, 1, 16), (4, 576, 2, 9), (2, 1024, 1, 8)]:
        fac = S.stiles_plan_stats(*shape, S.PLAN_FACTOR)["tasks"]
        fused = S.stiles_plan_stats(*shape, S.PLAN_FUSED)["tasks"]
        sel = S.stiles_plan_stats(*shape, S.PLAN_SELINV)["tasks"]
        assert fused < fac + sel, shape
        assert S.stiles_debug_validate(*shape, S.PLAN_FUSED) == S.STILES_OK, shape
        for first in (1, shape[0]):
            which = first << 16
            f = S.stiles_plan_stats(*shape, S.PLAN_FUSED + which)["tasks"]
            s = S.stiles_plan_stats(*shape, S.PLAN_SELINV + which)["tasks"]
            assert f == fac + s + (shape[0] + 1 - first), (shape, first)
            assert S.stiles_debug_validate(*shape, S.PLAN_FUSED + which) == S.STILES_OK, (shape, first)
