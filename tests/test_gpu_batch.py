"""Batched launch (many uneven matrices, one persistent graph launch):
every matrix against the oracle, every matrix bit-identical to its solo run
(same precision and tiling: the result of a block never depends on the
schedule), per-matrix NOT_SPD isolation, graph re-use across launches."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu, rel_err, run_gpu

SHAPES = [(16, 64, 1, 16), (5, 100, 2, 37), (9, 130, 1, 70), (4, 3, 1, 2), (1, 50, 0, 5), (7, 40, 4, 0),
          (30, 1, 1, 0), (12, 64, 3, 64)]
EMU_TOL = 1e-12


def _batch(mats, precision=0, budget_s=5.0):
    S = need_gpu()
    import torch
    bt = S.StilesBatch([(M.nt, M.b, M.w, M.a) for M in mats], wait_budget_s=budget_s, precision=precision)
    bt.upload(mats)
    bt.factor_selinv()
    torch.cuda.synchronize()
    Sh, Lh = bt.S.cpu().numpy(), bt.L.cpu().numpy()
    return bt, Sh, Lh


@pytest.mark.gpu
def test_batch_against_oracle_and_solo():
    mats = [W.random_arrowhead(*sh, seed=10 + m) for m, sh in enumerate(SHAPES)]
    bt, Sh, Lh = _batch(mats)
    try:
        lds = bt.logdet()
        for m, M in enumerate(mats):
            assert bt.status(m) == (0, 0)
            Lr, Sr, ldr = O.selinv(M)
            Sg, Lg = bt.sigma_tiles(m, Sh), bt.L_tiles(m, Lh)
            assert rel_err(Sg, Sr) < FP64_TOL
            assert rel_err(Lg, Lr) < FP64_TOL
            assert abs(lds[m] - ldr) < FP64_TOL * max(1.0, abs(ldr))
            L1, S1, ld1, st1 = run_gpu(M, "fused")
            for key in S1:
                assert np.array_equal(S1[key], Sg[key]), (m, key)
                assert np.array_equal(L1[key], Lg[key]), (m, key)
            assert ld1 == lds[m]
    finally:
        bt.close()


@pytest.mark.gpu
def test_batch_emulated_fp64_matches_solo_and_oracle():
    mats = [W.random_arrowhead(*sh, seed=40 + m) for m, sh in enumerate(SHAPES[:5])]
    bt, Sh, _ = _batch(mats, precision=1)
    try:
        for m, M in enumerate(mats):
            assert bt.status(m) == (0, 0)
            Sg = bt.sigma_tiles(m, Sh)
            _, Sr, _ = O.selinv(M)
            assert rel_err(Sg, Sr) < EMU_TOL
            _, S1, _, _ = run_gpu(M, "fused", precision=1)
            for key in S1:
                assert np.array_equal(S1[key], Sg[key]), (m, key)
    finally:
        bt.close()


@pytest.mark.gpu
def test_batch_not_spd_is_reported_per_matrix():
    S = need_gpu()
    mats = [W.random_arrowhead(6, 100, 1, 9, seed=3 + m) for m in range(4)]
    mats[2].tiles[(3, 3)][70, 70] = -5.0  # matrix 2 fails at global column 3*100+70
    bt, Sh, _ = _batch(mats)
    try:
        for m in range(4):
            code, info = bt.status(m)
            if m == 2:
                assert code == S.STILES_ERR_NOT_SPD and info == 3 * 100 + 70 + 1
            else:
                assert (code, info) == (0, 0)
                _, Sr, _ = O.selinv(mats[m])
                assert rel_err(bt.sigma_tiles(m, Sh), Sr) < FP64_TOL
        ld = bt.logdet()
        assert np.isnan(ld[2]) and np.all(np.isfinite(ld[[0, 1, 3]]))
    finally:
        bt.close()


@pytest.mark.gpu
def test_batch_graph_relaunch_and_new_buffers():
    import torch
    mats = [W.random_arrowhead(*sh, seed=70 + m) for m, sh in enumerate(SHAPES[:4])]
    bt, S_first, _ = _batch(mats)

    def same_as_first():  # every pattern tile (padding and unused slots are never written)
        now = bt.S.cpu().numpy()
        for m in range(len(mats)):
            a, b = bt.sigma_tiles(m, now), bt.sigma_tiles(m, S_first)
            assert all(np.array_equal(a[k], b[k]) for k in b), m

    try:
        bt.factor_selinv()  # same pointers: the graph is re-used
        torch.cuda.synchronize()
        same_as_first()
        bt.S = torch.full_like(bt.S, np.nan)  # new output buffer: a new graph
        bt.factor_selinv()
        torch.cuda.synchronize()
        same_as_first()
        for m in range(len(mats)):
            assert bt.status(m) == (0, 0)
    finally:
        bt.close()


@pytest.mark.gpu
def test_batch_counts_are_the_sum_of_solo_plans():
    S = need_gpu()
    stats = [S.stiles_plan_stats(*sh, S.PLAN_FUSED, 152) for sh in SHAPES]
    h = S.stiles_batch_create(SHAPES)
    try:
        bs = S.stiles_batch_stats(h)
    finally:
        S.stiles_batch_destroy(h)
    assert bs["tasks"] == sum(s["tasks"] for s in stats)
    assert bs["flops"] == pytest.approx(sum(s["flops"] for s in stats), rel=1e-12)
    assert bs["tile_gemms"] == sum(s["tile_gemms"] for s in stats)


@pytest.mark.gpu
@pytest.mark.parametrize("tune", [4, 8, 16, 8 + 16, 1, 2 + 8])
def test_tuning_codes_keep_the_results(tune):
    """Bits 2-5 re-partition blocks among CTAs: bit-identical; bits 0-1
    regroup update terms: equal to rounding (and to the oracle)."""
    S = need_gpu()
    import torch
    M = W.random_arrowhead(9, 130, 2, 70, seed=5)
    _, S0, ld0, _ = run_gpu(M, "fused")
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=5.0, tuning=tune).upload(M)
    try:
        st.factor_selinv()
        torch.cuda.synchronize()
        assert st.status()[0] == S.STILES_OK
        St = st.sigma_tiles()
    finally:
        st.close()
    if tune & 3 == 0:
        assert all(np.array_equal(St[k], S0[k]) for k in S0)
    else:
        _, Sr, _ = O.selinv(M)
        assert rel_err(St, Sr) < FP64_TOL


@pytest.mark.gpu
def test_autotuner_picks_a_candidate_and_caches(tmp_path):
    need_gpu()
    from paper_2504_19171_gb300 import autotune as AT
    path = str(tmp_path / "tune.json")
    tuner = AT.Autotuner(path, nt_probe=3, copies=2, reps=1, candidates=(0, 8, 16))
    code = tuner.best(128, 1, 20, 0)
    assert code in (0, 8, 16)
    again = AT.Autotuner(path)
    assert again.best(128, 1, 20, 0) == code  # from the cache, no probe
