"""Pins for the CPU FP64 oracle: each check compares it with something other
than itself (a library inverse, a closed form, a printed table, an invariant
of SPD inverses, an independent iterative solve).

Error metric used throughout (the reading of "max relative error"): the
largest absolute deviation over the selected entries divided by the largest
absolute reference entry.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sel_err(M, S, Ref):
    """max |S - Ref| / max |Ref| over the selected tiles (Ref dense n x n)."""
    num, den = 0.0, np.abs(Ref).max()
    for (i, k), T in S.items():
        r0, c0 = i * M.b, k * M.b
        num = max(num, np.abs(T - Ref[r0:r0 + T.shape[0], c0:c0 + T.shape[1]]).max(initial=0.0))
    return num / den


# ---------------------------------------------------------------- P1 -----
TINY = list(itertools.product([1, 2, 3, 5, 8], [1, 2, 3, 5, 8], [0, 1, 2, 4], [0, 1, 4]))


@pytest.mark.parametrize("nt,b,w,a", TINY)
def test_dense_inverse_tiny(nt, b, w, a):
    M = W.random_arrowhead(nt, b, w, a, seed=nt * 1000 + b * 100 + w * 10 + a)
    L, S, ld = O.selinv(M)
    A = M.to_dense()
    assert sel_err(M, S, np.linalg.inv(A)) < 1e-13
    assert abs(ld - np.linalg.slogdet(A)[1]) < 1e-12 * max(1.0, abs(ld))


# ---------------------------------------------------------------- P2 -----
@pytest.mark.parametrize("rho", [0.5, 0.9])
def test_ar1_closed_form(rho):
    n = 200
    M = W.ar1_tridiagonal(n, rho)
    L, S, ld = O.selinv(M)
    for (i, k), T in S.items():
        assert abs(T[0, 0] - rho ** abs(i - k) / (1 - rho * rho)) < 1e-13 / (1 - rho * rho)
    assert abs(ld - math.log(1 - rho * rho)) < 1e-12


def test_toeplitz_closed_form():
    n = 60
    M = W.toeplitz_tridiagonal(n)
    L, S, ld = O.selinv(M)
    for (i, k), T in S.items():
        # 1-based (p <= q): Sigma_pq = p (n + 1 - q) / (n + 1)
        p, q = k + 1, i + 1
        assert abs(T[0, 0] - p * (n + 1 - q) / (n + 1)) < 1e-12 * n
    assert abs(ld - math.log(n + 1)) < 1e-12


# ---------------------------------------------------------------- P3 -----
@pytest.mark.parametrize("rho,power,a", [(0.5, 1, 0), (0.9, 1, 0), (0.9, 1, 3), (0.7, 4, 0), (0.7, 2, 5)])
def test_kron_closed_form(rho, power, a):
    side, nt = 4, 12
    M = W.spatiotemporal(nt=nt, side=side, a=a, rho=rho, tau=0.0, band_power=power, couple_arrow=False)
    L, S, ld = O.selinv(M)
    Qs = W.laplacian2d_plus_identity(side)
    Qs_inv = np.linalg.inv(Qs)
    # AR(1) covariance in closed form, then its power for Q_t^p
    R = np.array([[rho ** abs(s - t) / (1 - rho * rho) for t in range(nt)] for s in range(nt)])
    Rp = np.linalg.matrix_power(R, power)
    scale = np.abs(Rp).max() * np.abs(Qs_inv).max()
    # Cholesky-based inversion is accurate to about kappa(A) * eps relative
    kappa = np.linalg.cond(M.to_dense())
    tol = max(1e-13, 20 * kappa * np.finfo(float).eps)
    for (i, k), T in S.items():
        if i == nt:
            ref = np.eye(a) if k == nt else np.zeros((a, side * side))
        else:
            ref = Rp[i, k] * Qs_inv
        assert np.abs(T - ref).max() < tol * scale, (i, k)
    b = side * side
    ref_ld = b * power * math.log(1 - rho * rho) + nt * np.linalg.slogdet(Qs)[1]
    assert abs(ld - ref_ld) < 1e-11 * abs(ref_ld)


# ---------------------------------------------------------------- P4 -----
def test_arrow_corner_schur():
    M = W.random_arrowhead(6, 5, 1, 4, seed=3, scale=0.3)
    L, S, ld = O.selinv(M)
    A = M.to_dense()
    nb = M.nt * M.b
    Ab, B, C = A[:nb, :nb], A[:nb, nb:], A[nb:, nb:]
    ref = np.linalg.inv(C - B.T @ np.linalg.solve(Ab, B))
    assert np.abs(S[(M.nt, M.nt)] - ref).max() < 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------- P5 -----
def test_cg_probe_against_inverse():
    M = W.random_arrowhead(5, 6, 2, 3, seed=11)
    Ainv = np.linalg.inv(M.to_dense())
    cols = [0, 7, 19, M.n - 1]
    X, relres = O.sigma_columns_cg(M, cols)
    assert np.all(relres < 1e-13)
    assert np.abs(X - Ainv[:, cols]).max() < 1e-13 * np.abs(Ainv).max()


def test_oracle_against_cg_columns():
    M = W.random_arrowhead(20, 32, 2, 8, seed=5)
    L, S, ld = O.selinv(M)
    rng = np.random.default_rng(0)
    cols = sorted(rng.choice(M.n, size=6, replace=False).tolist()) + [M.n - 1]
    X, relres = O.sigma_columns_cg(M, cols)
    assert np.all(relres < 1e-13)
    worst = 0.0
    for t, c in enumerate(cols):
        kc = min(c // M.b, M.nt)
        cc = c - kc * M.b
        for (i, k), T in S.items():
            r0 = i * M.b
            if k == kc:          # column c of tile (i, kc)
                worst = max(worst, np.abs(T[:, cc] - X[r0:r0 + T.shape[0], t]).max())
            elif i == kc:        # row c of tile (kc, k) = column c of its transpose
                worst = max(worst, np.abs(T[cc, :] - X[k * M.b:k * M.b + T.shape[1], t]).max())
    assert worst < 1e-13 * np.abs(X).max()


# ---------------------------------------------------------------- P6 -----
@pytest.mark.parametrize("shape", [(16, 64, 1, 16), (9, 7, 3, 5), (4, 20, 0, 2)])
def test_logdet_against_slogdet(shape):
    M = W.random_arrowhead(*shape, seed=2)
    L, S, ld = O.selinv(M)
    sign, ref = np.linalg.slogdet(M.to_dense())
    assert sign > 0
    assert abs(ld - ref) < 1e-12 * abs(ref)


# ---------------------------------------------------------------- P7 -----
def test_invariants():
    M = W.random_arrowhead(10, 12, 2, 6, seed=9)
    L, S, ld = O.selinv(M)
    for i in range(M.nt + 1):
        T = S[(i, i)]
        assert np.array_equal(T, T.T)                    # exact symmetry after mirroring
        d = np.diag(T)
        assert np.all(d > 0)
        assert np.all(d * np.diag(M.tiles[(i, i)]) >= 1 - 1e-14)  # (A^{-1})_ii A_ii >= 1
        np.linalg.cholesky(T)                            # Sigma_ii is positive definite
    for (i, k), T in L.items():
        if i == k:
            assert np.all(np.triu(T, 1) == 0)


def test_not_spd_reports_first_column():
    M = W.random_arrowhead(5, 4, 1, 3, seed=1)
    bad = 2 * M.b + 1                                   # global column 9 (0-based)
    T = M.tiles[(2, 2)]
    T[1, 1] = -1.0
    with pytest.raises(O.OracleNotSPD) as e:
        O.cholesky(M)
    assert e.value.info == bad + 1


# ------------------------------------------------- paper worked example -----
def test_paper_three_by_three_tile_equations():
    """The six tile equations of Sec. III-A for a 3 x 3 tile matrix, with L
    from numpy's Cholesky (independent of the oracle's factorization)."""
    b = 4
    M = W.random_arrowhead(2, b, 1, b, seed=21, scale=0.3)  # tiles 0, 1 and the arrow 2: a full 3 x 3 tile matrix
    A = M.to_dense()
    Lf = np.linalg.cholesky(A)
    Lt = {(i, j): Lf[i * b:(i + 1) * b, j * b:(j + 1) * b] for i in range(3) for j in range(3)}
    inv = np.linalg.inv
    S22 = inv(Lt[2, 2]).T @ inv(Lt[2, 2])
    S21 = -S22 @ Lt[2, 1] @ inv(Lt[1, 1])
    S11 = -inv(Lt[1, 1]).T @ Lt[2, 1].T @ S21 + inv(Lt[1, 1]).T @ inv(Lt[1, 1])
    S20 = -S21 @ Lt[1, 0] @ inv(Lt[0, 0]) - S22 @ Lt[2, 0] @ inv(Lt[0, 0])
    S10 = -S11 @ Lt[1, 0] @ inv(Lt[0, 0]) - S21.T @ Lt[2, 0] @ inv(Lt[0, 0])
    S00 = -inv(Lt[0, 0]).T @ Lt[1, 0].T @ S10 - inv(Lt[0, 0]).T @ Lt[2, 0].T @ S20 + inv(Lt[0, 0]).T @ inv(Lt[0, 0])
    ref = {(2, 2): S22, (2, 1): S21, (1, 1): S11, (2, 0): S20, (1, 0): S10, (0, 0): S00}
    L, S, ld = O.selinv(M)
    scale = max(np.abs(v).max() for v in ref.values())
    for key, R in ref.items():
        assert np.abs(S[key] - R).max() < 1e-13 * scale, key


# ------------------------------------------------------------ P8 (oracle) --
def n_gemm_formula(N, B):
    """Appendix A closed form for the selected-inversion GEMM count."""
    return (N - B) * B + B * (B - 1) // 2 + B * B * (N - B - 1) + B * (B + 1) * (2 * B + 1) // 6


def test_phase2_gemm_counts_match_paper_table():
    g = json.load(open(os.path.join(GOLDEN, "gemm_counts.json")))
    for row in g["table"]:
        N, B = row["N"], row["B"]
        M = W.random_arrowhead(N - 1, 2, B - 1, 2, seed=0)
        O.selinv(M)
        assert O.last_phase2_gemm_count() == row["gemm"], row


@pytest.mark.parametrize("N", range(2, 13))
def test_phase2_gemm_counts_match_formula(N):
    for B in range(1, N + 1):
        M = W.random_arrowhead(N - 1, 1, B - 1, 1, seed=0)
        O.selinv(M)
        assert O.last_phase2_gemm_count() == n_gemm_formula(N, B), (N, B)


# ------------------------------------------------------ planted mistakes --
def _pins_pass() -> bool:
    try:
        for shape in [(6, 3, 1, 2), (5, 2, 3, 1), (4, 3, 2, 0)]:
            M = W.random_arrowhead(*shape, seed=1)
            L, S, ld = O.selinv(M)
            A = M.to_dense()
            if sel_err(M, S, np.linalg.inv(A)) > 1e-13:
                return False
            if abs(ld - np.linalg.slogdet(A)[1]) > 1e-12 * max(1, abs(ld)):
                return False
        return True
    except Exception:
        return False


@pytest.mark.parametrize("mutant", range(1, 8))
def test_pins_catch_planted_mistakes(mutant):
    assert _pins_pass()
    O.set_mutant(mutant)
    try:
        assert not _pins_pass(), f"planted mistake {mutant} went unnoticed"
    finally:
        O.set_mutant(0)
