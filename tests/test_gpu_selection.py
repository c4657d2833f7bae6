"""General selections on the GPU: a selected plan's Sigma columns are
bit-identical to the full selected inversion on shapes where both plans run
the same update tasks (and agree to rounding where the full plan merges far
update terms into runs), earlier columns are not written; the full inverse
(band widened to every tile) against the dense inverse."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu, rel_err, run_gpu


@pytest.mark.gpu
@pytest.mark.parametrize("shape,first", [((9, 130, 1, 70), 4), ((16, 64, 1, 16), 16), ((7, 40, 4, 0), 1),
                                         ((12, 64, 3, 64), 11)])
def test_selected_columns_match_full_and_skip_the_rest(shape, first):
    S = need_gpu()
    import torch
    M = W.random_arrowhead(*shape, seed=sum(shape) + first)
    _, S_full, ld_full, _ = run_gpu(M, "fused")
    st = S.Stiles(*shape, wait_budget_s=5.0, first_column=first).upload(M)
    try:
        st.S.fill_(float("nan"))
        st.factor_selinv()
        torch.cuda.synchronize()
        assert st.status()[0] == S.STILES_OK
        assert st.logdet() == ld_full
        Ssel = st.sigma_tiles()
    finally:
        st.close()
    for (i, k), T in S_full.items():
        if k >= first:
            assert np.array_equal(Ssel[(i, k)], T), (i, k)
        else:
            assert np.all(np.isnan(Ssel[(i, k)])), (i, k)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(6, 64, 1, 16), (5, 30, 2, 7), (8, 16, 1, 0)])
def test_full_inverse_case6(shape):
    need_gpu()
    M = W.random_arrowhead(*shape, seed=3)
    F = __import__("paper_2504_19171_gb300.stiles", fromlist=["widen_band"]).widen_band(M)
    _, Sg, _, status = run_gpu(F, "fused")
    assert status[0] == 0
    inv = np.linalg.inv(M.to_dense())
    ref = {}
    for (i, k), T in Sg.items():
        r0, c0 = i * M.b, k * M.b
        ref[(i, k)] = inv[r0:r0 + T.shape[0], c0:c0 + T.shape[1]]
    assert rel_err(Sg, ref) < FP64_TOL
    _, Sr, _ = O.selinv(F)
    assert rel_err(Sg, Sr) < FP64_TOL


@pytest.mark.gpu
def test_selected_columns_where_the_full_plan_merges_update_runs():
    """(3, 640, 1, 16): the full fused plan merges far update terms into runs,
    a selected plan keeps single terms; its columns agree with the full run's
    to rounding and with the oracle."""
    S = need_gpu()
    import torch
    shape, first = (3, 640, 1, 16), 1
    M = W.random_arrowhead(*shape, seed=77)
    _, S_full, _, _ = run_gpu(M, "fused")
    _, Sr, ldr = O.selinv(M)
    st = S.Stiles(*shape, wait_budget_s=5.0, first_column=first).upload(M)
    try:
        st.S.fill_(float("nan"))
        st.factor_selinv()
        torch.cuda.synchronize()
        assert st.status()[0] == S.STILES_OK
        assert abs(st.logdet() - ldr) < 1e-10 * abs(ldr)
        Ssel = st.sigma_tiles()
    finally:
        st.close()
    sel = {key: T for key, T in Ssel.items() if key[1] >= first}
    assert rel_err(sel, {key: S_full[key] for key in sel}) < 1e-13
    assert rel_err(sel, {key: Sr[key] for key in sel}) < FP64_TOL
    assert all(np.all(np.isnan(T)) for key, T in Ssel.items() if key[1] < first)
