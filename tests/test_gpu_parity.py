"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle,
element by element on the same seeded inputs, for shapes that span several
fine blocks per tile, ragged tile and arrow edges, and the degenerate cases
(one tile column, no arrow, no band, scalar tiles)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu, rel_err, run_gpu

SHAPES = [
    (16, 64, 1, 16),   # the n = 1040 configuration
    (5, 100, 2, 37),   # ragged tiles (64 + 36) and arrow (37)
    (9, 130, 1, 70),   # three row blocks per tile (64 + 64 + 2), arrow 64 + 6
    (4, 3, 1, 2),      # tiles smaller than one fine block
    (1, 50, 0, 5),     # a single band tile column
    (6, 64, 0, 0),     # block diagonal, no arrow
    (7, 40, 4, 0),     # wide band, no arrow
    (3, 200, 2, 1),    # arrow of width 1
    (12, 64, 3, 64),
    (30, 1, 1, 0),     # scalar tridiagonal
    (10, 2, 3, 1),
]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", ["fused", "split"])
def test_parity_against_oracle(shape, mode):
    M = W.random_arrowhead(*shape, seed=sum(shape))
    Lr, Sr, ldr = O.selinv(M)
    L, S, ld, status = run_gpu(M, mode)
    assert status[0] == 0
    assert rel_err(L, Lr) < FP64_TOL
    assert rel_err(S, Sr) < FP64_TOL
    assert abs(ld - ldr) < FP64_TOL * max(1.0, abs(ldr))
    for i in range(M.nt + (1 if M.a else 0)):
        T = S[(i, i)]
        assert np.array_equal(T, T.T)
        assert np.all(np.triu(L[(i, i)], 1) == 0)


@pytest.mark.gpu
def test_inplace_factor():
    M = W.random_arrowhead(8, 96, 2, 20, seed=4)
    Lr, Sr, ldr = O.selinv(M)
    L, S, ld, status = run_gpu(M, "inplace")
    assert status[0] == 0
    assert rel_err(L, Lr) < FP64_TOL and rel_err(S, Sr) < FP64_TOL


@pytest.mark.gpu
def test_spatiotemporal_small_against_oracle():
    M = W.spatiotemporal(nt=12, side=8, a=16, rho=0.9, tau=1.0, seed=0)  # b = 64
    Lr, Sr, ldr = O.selinv(M)
    L, S, ld, status = run_gpu(M, "fused")
    assert status[0] == 0
    assert rel_err(S, Sr) < FP64_TOL
    assert abs(ld - ldr) < FP64_TOL * abs(ldr)


@pytest.mark.gpu
def test_kron_closed_form_band4():
    side, nt, rho = 8, 10, 0.6
    M = W.spatiotemporal(nt=nt, side=side, a=0, rho=rho, tau=0.0, band_power=4)
    L, S, ld, status = run_gpu(M, "fused")
    assert status[0] == 0
    Qs_inv = np.linalg.inv(W.laplacian2d_plus_identity(side))
    R = np.array([[rho ** abs(s - t) / (1 - rho * rho) for t in range(nt)] for s in range(nt)])
    R4 = np.linalg.matrix_power(R, 4)
    ref = {(i, k): R4[i, k] * Qs_inv for (i, k) in S}
    kappa = np.linalg.cond(M.to_dense())
    assert rel_err(S, ref) < max(1e-12, 50 * kappa * np.finfo(float).eps)


@pytest.mark.gpu
def test_bitwise_repeatable():
    """Every block is reduced in a fixed order, so the dynamic claim order
    does not change a single bit."""
    M = W.random_arrowhead(10, 128, 2, 33, seed=8)
    _, S1, ld1, _ = run_gpu(M, "fused")
    _, S2, ld2, _ = run_gpu(M, "fused")
    _, S3, ld3, _ = run_gpu(M, "split")
    for key in S1:
        assert np.array_equal(S1[key], S2[key]) and np.array_equal(S1[key], S3[key])
    assert ld1 == ld2 == ld3



@pytest.mark.gpu
@pytest.mark.parametrize("buffers", ["pinned", "pageable", "same_pinned"])
def test_host_buffer_entry_point(buffers):
    """stiles_factor_selinv_host returns the same bits as the device-buffer
    call, and Sigma matches the oracle, in both of its ways: separate pinned
    buffers (the kernel reads A and writes the final Sigma blocks over the
    host link), and pageable or shared buffers (copies before and after)."""
    import torch
    M = W.random_arrowhead(9, 96, 2, 20, seed=21)
    _, S_dev, ld_dev, _ = run_gpu(M, "fused")
    S = need_gpu()
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=5.0)
    try:
        packed = torch.from_numpy(st.layout.pack(M.tiles, np.zeros(st.doubles)))
        if buffers == "pinned":
            A_host = packed.pin_memory()
            S_host = torch.full((st.doubles,), np.nan, dtype=torch.float64).pin_memory()
        elif buffers == "pageable":
            A_host = packed.clone()
            S_host = torch.full((st.doubles,), np.nan, dtype=torch.float64)
        else:
            A_host = S_host = packed.pin_memory()
        for rep in range(2):  # a second call on the same handle and buffers
            if buffers == "same_pinned" and rep:
                A_host.copy_(packed)
            ld = st.factor_selinv_host(A_host, S_host)
            assert st.status()[0] == S.STILES_OK
            got = st.layout.unpack(S_host.numpy())
            for key in S_dev:
                assert np.array_equal(got[key], S_dev[key]), (buffers, rep, key)
            assert ld == ld_dev
    finally:
        st.close()
    _, Sref, _ = O.selinv(M)
    assert rel_err(got, Sref) < FP64_TOL


EMU_TOL = 1e-12  # emulated-FP64 target against the FP64 oracle
PREC_SHAPES = [(16, 64, 1, 16), (5, 100, 2, 37), (9, 130, 1, 70), (4, 3, 1, 2), (7, 40, 4, 0), (12, 64, 3, 64)]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", PREC_SHAPES)
@pytest.mark.parametrize("mode", ["fused", "split"])
def test_emulated_fp64_parity(shape, mode):
    S = need_gpu()
    M = W.random_arrowhead(*shape, seed=sum(shape) + 1)
    Lr, Sr, ldr = O.selinv(M)
    L, Sg, ld, status = run_gpu(M, mode, precision=S.STILES_EMU64)
    assert status[0] == 0
    assert rel_err(L, Lr) < EMU_TOL
    assert rel_err(Sg, Sr) < EMU_TOL
    assert abs(ld - ldr) < EMU_TOL * max(1.0, abs(ldr))
    for i in range(M.nt + (1 if M.a else 0)):
        assert np.array_equal(Sg[(i, i)], Sg[(i, i)].T)


@pytest.mark.gpu
def test_emulated_fp64_spatiotemporal():
    S = need_gpu()
    M = W.spatiotemporal(nt=12, side=8, a=16, rho=0.9, tau=1.0, seed=0)
    Lr, Sr, ldr = O.selinv(M)
    L, Sg, ld, status = run_gpu(M, "fused", precision=S.STILES_EMU64)
    assert status[0] == 0
    assert rel_err(Sg, Sr) < EMU_TOL and abs(ld - ldr) < EMU_TOL * abs(ldr)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", PREC_SHAPES)
def test_fp32_class_error_is_reported(shape):
    """FP32-class products: the error against the FP64 oracle is reported
    (printed) and must stay at FP32 level for these well-conditioned cases."""
    S = need_gpu()
    M = W.random_arrowhead(*shape, seed=sum(shape) + 2)
    Lr, Sr, ldr = O.selinv(M)
    L, Sg, ld, status = run_gpu(M, "fused", precision=S.STILES_FP32X)
    assert status[0] == 0
    err = rel_err(Sg, Sr)
    print(f"FP32-class {shape}: Sigma rel err {err:.3e}, L rel err {rel_err(L, Lr):.3e}, logdet abs err {abs(ld - ldr):.3e}")
    assert err < 1e-4


MERGED_RUN_SHAPES = [(3, 640, 1, 16), (4, 576, 2, 9)]  # blocks far enough apart for update runs


@pytest.mark.gpu
@pytest.mark.parametrize("shape", MERGED_RUN_SHAPES)
def test_update_runs_parity(shape):
    """Shapes whose fused plan merges far update terms into runs: the fused
    FP64 and EMU64 results against the oracle, and against the factor +
    selinv calls (single terms), which agree to rounding."""
    M = W.random_arrowhead(*shape, seed=sum(shape) + 5)
    _, Sr, ldr = O.selinv(M)
    _, S_fused, ld_fused, st_fused = run_gpu(M, "fused")
    _, S_split, ld_split, st_split = run_gpu(M, "split")
    _, S_emu, ld_emu, st_emu = run_gpu(M, "fused", precision=1)
    assert st_fused[0] == 0 and st_split[0] == 0 and st_emu[0] == 0
    assert rel_err(S_fused, Sr) < FP64_TOL
    assert rel_err(S_split, Sr) < FP64_TOL
    assert rel_err(S_fused, S_split) < 1e-13
    assert rel_err(S_emu, Sr) < 1e-12
    for ld in (ld_fused, ld_split, ld_emu):
        assert abs(ld - ldr) < 1e-10 * abs(ldr)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["fused", "split", "inplace"])
@pytest.mark.parametrize("precision", [0, 1])
def test_strict_upper_of_diagonal_tiles(mode, precision):
    """L's strict upper part in every diagonal tile is written as zero, and
    A's is never read: both start as NaN (the whole L buffer, and the strict
    upper triangles of A's diagonal tiles), the results still match the
    oracle and L's strict upper triangles come out exactly zero."""
    S = need_gpu()
    import torch
    M = W.random_arrowhead(6, 192, 2, 24, seed=11)  # three 64-column blocks per tile
    Lr, Sr, ldr = O.selinv(M)
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=5.0, precision=precision).upload(M)
    try:
        lay = st.layout
        for i in range(M.nt + (1 if M.a else 0)):
            T = lay.tile_view(st.A, i, i)
            T.copy_(torch.where(torch.ones_like(T, dtype=torch.bool).triu(1), torch.full_like(T, float("nan")), T))
        st.L.fill_(float("nan"))
        if mode == "fused":
            st.factor_selinv()
        else:
            st.factor(inplace=(mode == "inplace"))
            st.selinv()
        torch.cuda.synchronize()
        assert st.status()[0] == 0
        L, Sg = st.L_tiles(), st.sigma_tiles()
    finally:
        st.close()
    tol = FP64_TOL if precision == 0 else 1e-12
    assert rel_err(L, Lr) < tol and rel_err(Sg, Sr) < tol
    for i in range(M.nt + (1 if M.a else 0)):
        U = np.triu(L[(i, i)], 1)
        assert np.all(U == 0), (i, np.argwhere(U != 0)[:3])
