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


def run_full(M, precision=0):
    S = need_gpu()
    import torch
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=10.0, precision=precision).upload(M)
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


EMU_TOL = 1e-12  # emulated-FP64 target


def ar1_covariance(nt, rho):
    """R = Q_t^{-1} of the AR(1) precision with unit innovations:
    R_st = rho^|s-t| / (1 - rho^2) (the closed form, not a solve)."""
    idx = np.arange(nt)
    return rho ** np.abs(idx[:, None] - idx[None, :]) / (1 - rho * rho)


def kron_closed_form_error(lay, Sig, ld, w, rho):
    """max |Sigma - Sigma_exact| / max |Sigma_exact| over every selected tile
    and the relative logdet error, for A = kron(Q_t^w, Q_s) with the arrow
    decoupled (corner I): Sigma tile (i, k) = (R^w)_ik Q_s^{-1} with R the
    AR(1) covariance, logdet = w b log(1 - rho^2) + nt logdet(Q_s)."""
    Rw = np.linalg.matrix_power(ar1_covariance(NT, rho), w)
    Qs_inv = np.linalg.inv(W.laplacian2d_plus_identity(SIDE))
    scale = np.abs(Rw).max() * np.abs(Qs_inv).max()
    worst = 0.0
    for (i, k) in lay.pattern():
        T = lay.tile_view(Sig, i, k)
        if i == NT:
            ref = np.eye(A) if k == NT else 0.0
        else:
            ref = Rw[i, k] * Qs_inv
        worst = max(worst, np.abs(T - ref).max())
    ref_ld = w * B * math.log(1 - rho * rho) + NT * np.linalg.slogdet(W.laplacian2d_plus_identity(SIDE))[1]
    return worst / scale, abs(ld - ref_ld) / abs(ref_ld)


# (tile bandwidth, rho, precision, Sigma tolerance, logdet tolerance); None: reported only.
# rho keeps kron(Q_t^w, Q_s) well conditioned (AR(1) precision eigenvalues
# in [(1 - rho)^2, (1 + rho)^2]): at w = 4, rho = 0.4 gives a condition number
# near that of the w = 1, rho = 0.9 case (about 8e3 against 3e3), so the
# FP64 rounding of the method stays well inside the bars.
KRON_CASES = [
    (4, 0.4, 0, FP64_TOL, FP64_TOL),
    (4, 0.4, 1, EMU_TOL, EMU_TOL),
    (1, 0.9, 1, EMU_TOL, EMU_TOL),
    (1, 0.9, 2, None, None),
    (4, 0.4, 2, None, None),
]


@pytest.mark.gpu
@pytest.mark.parametrize("w,rho,prec,tol,ld_tol", KRON_CASES)
def test_full_size_kronecker_closed_form_band_and_precisions(w, rho, prec, tol, ld_tol):
    """The benchmark's size (nt = 200 tiles of 1024, arrow 64) at tile
    bandwidth 1 and 4, in FP64, emulated FP64 and FP32-class, against the
    Kronecker closed form (an independent reference: no oracle run, no GPU
    result): FP64 within 1e-10, emulated FP64 within 1e-12, FP32-class
    printed and bounded at FP32 level."""
    M = W.spatiotemporal(nt=NT, side=SIDE, a=A, rho=rho, tau=0.0, couple_arrow=False, band_power=w)
    lay, Sig, ld, status = run_full(M, precision=prec)
    assert status[0] == 0, status
    err, ld_err = kron_closed_form_error(lay, Sig, ld, w, rho)
    print(f"kron closed form w={w} rho={rho} precision={prec}: Sigma err {err:.3e}, logdet rel err {ld_err:.3e}")
    if tol is None:
        assert err < 1e-4 and ld_err < 1e-5
    else:
        assert err < tol, err
        assert ld_err < ld_tol, ld_err
