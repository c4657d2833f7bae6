"""Python entry to the plain C FP64 oracle (``stiles_oracle.c``) and the
independent column probe.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline may use this module; the library never does. Nothing here imports
the CUDA package, and the C oracle shares no code with it.

Functions (each cites what it follows):

* :func:`cholesky` -- tiled Cholesky A = L L^T on the arrowhead tile pattern
  (Sec. III: the factorization selected inversion starts from).
* :func:`selinv` -- two-phase selected inversion: phase 1 (Algorithm 2),
  phase 2 (Algorithm 3 with the tile recurrences of Sec. III-A).
* :func:`logdet` -- 2 * sum log diag(L) (plain definition).
* :func:`sigma_columns_cg` -- columns of A^{-1} by conjugate gradients on
  the matrix itself: the definition Sigma = A^{-1} reached by a different
  algorithm, used to check sampled entries at sizes the scalar oracle cannot
  finish.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Iterable, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stiles_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs = {}
_mutant = 0


def _lib_path(mutant: int) -> str:
    return os.path.join(_BUILD, "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so")


def build(force: bool = False, mutant: int = 0) -> str:
    """Compile the C oracle with gcc (-O2 -ffp-contract=off). ``mutant`` > 0
    builds a planted-mistake variant for the tests that check the pins."""
    path = _lib_path(mutant)
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               f"-DORACLE_MUTANT={int(mutant)}", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def set_mutant(mutant: int) -> None:
    """Route the functions below to a planted-mistake build (0 = the oracle)."""
    global _mutant
    _mutant = int(mutant)


def _load():
    with _lock:
        if _mutant not in _libs:
            lib = ctypes.CDLL(build(mutant=_mutant))
            i32, dp = ctypes.c_int, ctypes.POINTER(ctypes.c_double)
            lib.oracle_layout_size.restype = ctypes.c_long
            lib.oracle_layout_size.argtypes = [i32] * 4
            lib.oracle_tile_offset.restype = ctypes.c_long
            lib.oracle_tile_offset.argtypes = [i32] * 6
            lib.oracle_cholesky.restype = i32
            lib.oracle_cholesky.argtypes = [i32] * 4 + [dp]
            lib.oracle_logdet.restype = ctypes.c_double
            lib.oracle_logdet.argtypes = [i32] * 4 + [dp]
            lib.oracle_selinv.restype = i32
            lib.oracle_selinv.argtypes = [i32] * 4 + [dp, dp]
            lib.oracle_last_phase2_gemms.restype = ctypes.c_long
            lib.oracle_last_phase2_gemms.argtypes = []
            _libs[_mutant] = lib
        return _libs[_mutant]


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pattern(nt: int, w: int, a: int) -> Iterable[Tuple[int, int]]:
    for k in range(nt):
        yield (k, k)
        for i in range(k + 1, min(k + w, nt - 1) + 1):
            yield (i, k)
        if a > 0:
            yield (nt, k)
    if a > 0:
        yield (nt, nt)


class _Packed:
    """A tile dictionary packed into the oracle's own row-major layout."""

    def __init__(self, nt: int, b: int, w: int, a: int):
        lib = _load()
        self.shape = (nt, b, w, a)
        self.buf = np.zeros(lib.oracle_layout_size(nt, b, w, a))
        self.offsets = {}
        for i, k in _pattern(nt, w, a):
            off = lib.oracle_tile_offset(nt, b, w, a, i, k)
            assert off >= 0
            r = a if i == nt else b
            c = a if k == nt else b
            self.offsets[(i, k)] = (off, r, c)

    def view(self, key) -> np.ndarray:
        off, r, c = self.offsets[key]
        return self.buf[off:off + r * c].reshape(r, c)

    def load(self, tiles: Dict[Tuple[int, int], np.ndarray]) -> "_Packed":
        for key in self.offsets:
            self.view(key)[...] = tiles[key]
        return self

    def unload(self) -> Dict[Tuple[int, int], np.ndarray]:
        return {key: self.view(key).copy() for key in self.offsets}


class OracleNotSPD(ArithmeticError):
    def __init__(self, info: int):
        super().__init__(f"matrix is not SPD: first failing pivot at global column {info} (1-based)")
        self.info = info


def cholesky(M) -> Dict[Tuple[int, int], np.ndarray]:
    """Tile factor L of an :class:`ArrowheadTiles` (upper part of diagonal
    tiles zero). Raises :class:`OracleNotSPD` with the LAPACK-style column."""
    nt, b, w, a = M.nt, M.b, M.w, M.a
    P = _Packed(nt, b, w, a).load(M.tiles)
    info = _load().oracle_cholesky(nt, b, w, a, _ptr(P.buf))
    if info < 0:
        raise ValueError("bad shape")
    if info > 0:
        raise OracleNotSPD(info)
    return P.unload()


def logdet(M, L: Dict[Tuple[int, int], np.ndarray]) -> float:
    P = _Packed(M.nt, M.b, M.w, M.a).load(L)
    return float(_load().oracle_logdet(M.nt, M.b, M.w, M.a, _ptr(P.buf)))


def selinv_from_factor(M, L: Dict[Tuple[int, int], np.ndarray]) -> Dict[Tuple[int, int], np.ndarray]:
    nt, b, w, a = M.nt, M.b, M.w, M.a
    PL = _Packed(nt, b, w, a).load(L)
    PS = _Packed(nt, b, w, a)
    if _load().oracle_selinv(nt, b, w, a, _ptr(PL.buf), _ptr(PS.buf)) != 0:
        raise RuntimeError("oracle_selinv failed")
    return PS.unload()


def last_phase2_gemm_count() -> int:
    """Tile GEMMs performed by phase 2 of the most recent selinv call."""
    return int(_load().oracle_last_phase2_gemms())


def selinv(M):
    """(L, Sigma, logdet) for an :class:`ArrowheadTiles`."""
    L = cholesky(M)
    return L, selinv_from_factor(M, L), logdet(M, L)


def sparse_tiles(M) -> Dict[Tuple[int, int], object]:
    """The tiles as scipy CSR matrices (exact copies of the nonzeros), for a
    fast matvec when the tiles themselves are sparse (Kronecker workloads)."""
    import scipy.sparse as sp
    cache = {}
    out = {}
    for key, T in M.tiles.items():
        tid = id(T)
        if tid not in cache:
            cache[tid] = sp.csr_matrix(T)
        out[key] = cache[tid]
    return out


def matvec(M, X: np.ndarray, tiles=None) -> np.ndarray:
    """A @ X using the tiles (lower pattern plus its transpose)."""
    Y = np.zeros_like(X)
    for (i, k), T in (tiles or M.tiles).items():
        r0, c0 = i * M.b, k * M.b
        Y[r0:r0 + T.shape[0]] += T @ X[c0:c0 + T.shape[1]]
        if i != k:
            Y[c0:c0 + T.shape[1]] += T.T @ X[r0:r0 + T.shape[0]]
    return Y


def sigma_columns_cg(M, cols, tol: float = 1e-15, maxiter: int = 5000, sparse: bool = False) -> Tuple[np.ndarray, np.ndarray]:
    """Columns ``cols`` of A^{-1} by diagonally (Jacobi) preconditioned
    conjugate gradients, one independent CG per column run side by side.

    Returns (X, relres): X[:, t] solves A x = e_{cols[t]} and relres[t] is
    ||e - A x|| / ||e|| at exit. ``sparse=True`` multiplies with CSR copies
    of the tiles (same values, fewer operations).
    """
    tiles = sparse_tiles(M) if sparse else None
    cols = np.asarray(cols, dtype=np.int64)
    n = M.n
    E = np.zeros((n, len(cols)))
    E[cols, np.arange(len(cols))] = 1.0
    dinv = np.zeros(n)
    for i in range(M.nt + (1 if M.a > 0 else 0)):
        r0 = i * M.b
        d = np.diag(M.tiles[(i, i)])
        dinv[r0:r0 + d.size] = 1.0 / d
    X = np.zeros_like(E)
    R = E.copy()
    Z = dinv[:, None] * R
    P = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    for _ in range(maxiter):
        AP = matvec(M, P, tiles)
        alpha = rz / np.einsum("ij,ij->j", P, AP)
        X += alpha * P
        R -= alpha * AP
        res = np.linalg.norm(R, axis=0)
        if np.all(res <= tol):
            break
        Z = dinv[:, None] * R
        rz_new = np.einsum("ij,ij->j", R, Z)
        P = Z + (rz_new / rz) * P
        rz = rz_new
    relres = np.linalg.norm(E - matvec(M, X, tiles), axis=0)
    return X, relres
