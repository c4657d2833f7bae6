"""Failure detection on the GPU without faulting it: non-SPD input reported
LAPACK-style, a dependency that never arrives ends the launch with a TIMEOUT
status after a short wait budget (the GPU stays usable), bad arguments are
rejected before any launch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu, rel_err, run_gpu


@pytest.mark.gpu
@pytest.mark.parametrize("tile,local", [(0, 0), (2, 5), (3, 70), (6, 3)])
def test_not_spd_reports_first_failing_column(tile, local):
    S = need_gpu()
    M = W.random_arrowhead(6, 100, 1, 9, seed=3)
    M.tiles[(tile, tile)][local, local] = -5.0
    col = tile * M.b + local
    with pytest.raises(O.OracleNotSPD) as e:
        O.cholesky(M)
    assert e.value.info == col + 1
    for mode in ("fused", "split"):
        _, _, _, status = run_gpu(M, mode)
        assert status[0] == S.STILES_ERR_NOT_SPD
        assert status[1] == col + 1


@pytest.mark.gpu
def test_nan_input_is_not_spd():
    S = need_gpu()
    M = W.random_arrowhead(4, 64, 1, 8, seed=1)
    M.tiles[(1, 1)][3, 3] = np.nan
    _, _, _, status = run_gpu(M, "fused")
    assert status[0] == S.STILES_ERR_NOT_SPD and status[1] == 64 + 3 + 1


@pytest.mark.gpu
@pytest.mark.parametrize("which", [0, 2])
def test_stuck_dependency_times_out_and_gpu_recovers(which):
    S = need_gpu()
    import torch
    M = W.random_arrowhead(6, 64, 1, 8, seed=2)
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=0.5).upload(M)
    try:
        S.stiles_debug_break_plan(st.h, which)
        st.factor() if which == 0 else st.factor_selinv()
        code, info, done = st.status()
        assert code == S.STILES_ERR_TIMEOUT
        assert S.stiles_logdet(st.h)[0] == S.STILES_ERR_TIMEOUT
    finally:
        st.close()
    torch.cuda.synchronize()
    # the device is still healthy: a fresh handle computes the right answer
    Lr, Sr, ldr = O.selinv(M)
    L, Sg, ld, status = run_gpu(M, "fused")
    assert status[0] == 0 and rel_err(Sg, Sr) < FP64_TOL


@pytest.mark.gpu
def test_bad_arguments_are_rejected():
    S = need_gpu()
    import torch
    st = S.Stiles(3, 8, 1, 2)
    try:
        with pytest.raises(S.StilesError) as e:
            S.stiles_factor(st.h, 0, st.L.data_ptr(), st.scratch.data_ptr(), 0)
        assert e.value.code == S.STILES_ERR_INVALID_ARG
        with pytest.raises(S.StilesError):
            S.stiles_selinv(st.h, st.L.data_ptr(), st.L.data_ptr(), st.scratch.data_ptr(), 0)
        with pytest.raises(S.StilesError):
            S.stiles_selinv(st.h, st.L.data_ptr(), st.S.data_ptr(), st.scratch.data_ptr() + 8, 0)
        with pytest.raises(S.StilesError):
            S.stiles_set_option(st.h, S.STILES_OPT_WAIT_BUDGET_NS, 0)
    finally:
        st.close()
    with pytest.raises(S.StilesError) as e:
        S.stiles_create(0, 8, 1, 2)
    assert e.value.code == S.STILES_ERR_INVALID_ARG
    with pytest.raises(S.StilesError) as e:
        S.stiles_create(3, 8, 1, 2, precision=7)
    assert e.value.code == S.STILES_ERR_UNSUPPORTED


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("value", [np.nan, np.inf])
@pytest.mark.parametrize("where", ["band", "arrow"])
def test_nonfinite_off_diagonal_entry_is_reported(prec, value, where):
    """A NaN or Inf in an off-diagonal tile of A (made on the host) reaches a
    pivot through the factor's products in every precision mode: the launch
    reports NOT_SPD instead of a finite, wrong Sigma. The emulated-FP64 digit
    split turns a non-finite operand row or column into NaN products."""
    S = need_gpu()
    M = W.random_arrowhead(6, 100, 1, 9, seed=7)
    if where == "band":
        M.tiles[(1, 0)][17, 40] = value  # row 17 of L_10: reaches the pivots of tile 1 through SYRK
    else:
        M.tiles[(M.nt, 0)][3, 70] = value  # row 3 of the arrow: reaches the corner's pivots
    _, _, _, status = run_gpu(M, "fused", precision=prec)
    assert status[0] == S.STILES_ERR_NOT_SPD, (prec, where, status)
