"""Algorithmic flop count of the method in closed form.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and the
bench's CPU-oracle arm use it; the library never does, and nothing here
imports the CUDA package.

Counting convention (one fixed rule for every TFLOP/s figure): POTRF, TRTRI
and LAUUM of an m x m tile m^3/3; TRSM and TRMM m k^2; SYRK m^2 k; GEMM
2 m n k; the symmetric update of a diagonal Sigma tile m^2 k per term (only
its lower triangle is needed, as for SYRK).

The tile operations are those of the factorization (Sec. III, taken from
sTiles: POTRF / TRSM / SYRK / GEMM on the tiles of the band + arrow pattern)
and of the two-phase selected inversion (Algorithm 2: TRTRI, LAUUM, TRMM of
every tile column; Algorithm 3 with the recurrences of Sec. III-A: one
Sigma_jk U_ki product per pair (j, k) of struct(i), and one update of
Sigma_ii per k). Tile column k < nt has n_k = min(w, nt - 1 - k) band tiles
below its diagonal plus the arrow tile (a rows) when a > 0, so its cost
depends on n_k only: nt - w columns have n_k = w and one column each has
n_k = w - 1, ..., 0. The arrow corner (a x a) adds its POTRF and its TRTRI +
LAUUM.

Independent checks (tests): a full band (w = nt - 1, a = 0) gives the
textbook dense counts n^3/3 for the Cholesky factorization and 2 n^3/3 for
the inverse from the factor (TRTRI + LAUUM); a block-diagonal matrix gives
nt b^3/3 and 2 nt b^3/3.
"""
from __future__ import annotations

from fractions import Fraction


def _factor_column(n: int, b: int, a: int) -> Fraction:
    """Factor work of one band tile column with n band tiles below it."""
    m = n * b + a                                  # rows below the diagonal tile
    potrf = Fraction(b ** 3, 3)
    trsm = m * b * b                               # L_ik = A_ik L_kk^{-T}, i in struct(k)
    syrk = (n * b * b + a * a) * b                 # A_ii -= L_ik L_ik^T
    gemm = 2 * b * (b * b * n * (n - 1) // 2 + n * a * b)  # A_ij -= L_ik L_jk^T, i > j
    return potrf + trsm + syrk + gemm


def _selinv_column(n: int, b: int, a: int) -> Fraction:
    """Selected-inversion work of one band tile column with n band tiles below it."""
    m = n * b + a
    trtri_lauum = Fraction(2 * b ** 3, 3)
    trmm = m * b * b                               # U_ki = L_ki Linv_ii
    products = 2 * b * m * m                       # Sigma_ji = -sum_k S_jk U_ki, j, k in struct(i)
    diag = b * b * m                               # Sigma_ii -= Sigma_ki^T U_ki (lower triangle)
    return trtri_lauum + trmm + products + diag


def flops(nt: int, b: int, w: int, a: int, kind: str = "fused") -> float:
    """Algorithmic flops of one factorization ("factor"), one selected
    inversion ("selinv"), or both ("fused") of the (nt, b, w, a) pattern."""
    if nt < 1 or b < 1 or w < 0 or a < 0:
        raise ValueError("nt >= 1, b >= 1, w >= 0, a >= 0")
    if kind not in ("factor", "selinv", "fused"):
        raise ValueError(kind)
    w = min(w, nt - 1)
    counts = [(w, nt - w)] + [(q, 1) for q in range(w)]
    total = Fraction(0)
    for n, c in counts:
        if kind != "selinv":
            total += c * _factor_column(n, b, a)
        if kind != "factor":
            total += c * _selinv_column(n, b, a)
    if a > 0:
        if kind != "selinv":
            total += Fraction(a ** 3, 3)
        if kind != "factor":
            total += Fraction(2 * a ** 3, 3)
    return float(total)
