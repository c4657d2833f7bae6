"""Parity at the benchmark's full size and launch configuration (one fused
persistent launch of the n = 204,864 spatio-temporal arrowhead matrix,
nt = 200 tiles of 1024, bandwidth 1, arrow 64).

The scalar oracle cannot finish this size in test time, so the checks use
what the oracle can compute one by one or what holds at any size:
* sampled columns of A^{-1} from the oracle's conjugate-gradient probe,
  compared with every selected entry of Sigma in those columns;
* the Kronecker closed form of the same shape (tau = 0, arrow decoupled):
  Sigma_st = (rho^|s-t| / (1 - rho^2)) Q_s^{-1}, corner = I, and
  logdet = b log(1 - rho^2) + nt logdet(Q_s);
* exact symmetry and positivity of diag(Sigma)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu

NT, SIDE, A = 200, 32, 64
B = SIDE * SIDE


def run_full(M):
    S = need_gpu()
    import torch
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=10.0).upload(M)
    try:
        st.factor_selinv()
        torch.cuda.synchronize()
        status = st.status()
        ld = st.logdet() if status[0] == 0 else float("nan")
        Sig = st.S.cpu().numpy()
        return st.layout, Sig, ld, status
    finally:
        st.close()


@pytest.mark.gpu
def test_full_size_columns_against_cg_probe():
    M = W.spatiotemporal(nt=NT, side=SIDE, a=A, rho=0.9, tau=1.0, seed=0)
    lay, Sig, ld, status = run_full(M)
    assert status[0] == 0, status
    n = M.n
    cols = [0, 517, 1023, 1024 + 300, 99 * B + 777, (NT - 1) * B + 1023, NT * B + 5, n - 1]
    X, relres = O.sigma_columns_cg(M, cols, tol=1e-14, sparse=True)
    assert np.all(relres < 1e-12), relres
    worst, scale = 0.0, np.abs(X).max()
    for t, c in enumerate(cols):
        kc = min(c // B, NT)
        cc = c - kc * B
        for (i, k) in lay.pattern():
            T = lay.tile_view(Sig, i, k)
            if k == kc:
                ref = X[i * B:i * B + T.shape[0], t]
                worst = max(worst, np.abs(T[:, cc] - ref).max())
            elif i == kc:
                ref = X[k * B:k * B + T.shape[1], t]
                worst = max(worst, np.abs(T[cc, :] - ref).max())
    assert worst < FP64_TOL * scale, worst / scale
    # exact symmetry and positive diagonal of every diagonal tile
    for i in range(NT + 1):
        T = np.asarray(lay.tile_view(Sig, i, i))
        assert np.array_equal(T, T.T)
        assert np.all(np.diag(T) > 0)


@pytest.mark.gpu
def test_full_size_kronecker_closed_form():
    rho = 0.9
    M = W.spatiotemporal(nt=NT, side=SIDE, a=A, rho=rho, tau=0.0, couple_arrow=False)
    lay, Sig, ld, status = run_full(M)
    assert status[0] == 0, status
    Qs = W.laplacian2d_plus_identity(SIDE)
    Qs_inv = np.linalg.inv(Qs)
    scale = np.abs(Qs_inv).max() / (1 - rho * rho)
    worst = 0.0
    for (i, k) in lay.pattern():
        T = lay.tile_view(Sig, i, k)
        if i == NT:
            ref = np.eye(A) if k == NT else 0.0
        else:
            ref = (rho ** abs(i - k) / (1 - rho * rho)) * Qs_inv
        worst = max(worst, np.abs(T - ref).max())
    assert worst < FP64_TOL * scale, worst / scale
    ref_ld = B * math.log(1 - rho * rho) + NT * np.linalg.slogdet(Qs)[1]
    assert abs(ld - ref_ld) < FP64_TOL * abs(ref_ld)
