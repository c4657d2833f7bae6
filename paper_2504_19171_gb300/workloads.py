"""Seeded synthetic SPD block-arrowhead inputs.

This module only *generates* matrices; it holds none of the selected-inversion
arithmetic. Both the CUDA path and the CPU oracle receive its output, so it is
the one piece of Python they share.

A matrix is an :class:`ArrowheadTiles`: the lower tile pattern of an SPD
block-arrowhead matrix (Sec. I, Fig. 2 case 7 of the sTiles selected
inversion paper): ``nt`` band tile columns of size ``b``, lower bandwidth
``w`` tiles, and an arrow tile row of height ``a`` (tile index ``nt``).
Tile ``(i, k)`` with ``i >= k`` is a dense float64 array of shape
``(rows(i), rows(k))``; diagonal tiles are stored full and symmetric.

Recipes (all use ``numpy.random.default_rng(seed)``):

* :func:`random_arrowhead` -- off-diagonal entries N(0,1) * scale, symmetric,
  diagonal = 1 + row absolute sum (strictly diagonally dominant, so SPD).
* :func:`spatiotemporal` -- kron(Q_t, Q_s) + tau*I with Q_t an AR(1)
  precision (rho) and Q_s the 2-D 5-point Laplacian plus identity, and a dense
  arrow of N(0,1) entries whose corner is made diagonally dominant over its
  full row. This stands in for the INLA-style spatio-temporal models the
  paper's matrices come from (their arrow = fixed effects, band = random
  effects); the paper's own matrices are not available.
* :func:`sweep_arrowhead` -- a fixed random base pattern rescaled per request
  by (tau, rho), diagonally dominant for every tau > 0.
* :func:`ar1_tridiagonal`, :func:`toeplitz_tridiagonal` -- scalar (b = 1)
  tridiagonal cases with closed-form inverses.
* :func:`batch_shapes` -- shape draws for uneven batches.
* :func:`random_arrowhead_packed` -- the :func:`random_arrowhead` recipe
  drawn on a torch device straight into the packed band+arrow layout (for
  batches of many large matrices; its random stream is torch's, not numpy's).
* :func:`sweep_base`, :func:`sweep_base_packed` -- the fixed part of a sweep
  shape (base values and band / arrow absolute row sums) for the request
  server, on the host or drawn on a torch device.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Iterator, List, Tuple

import numpy as np

TileKey = Tuple[int, int]


@dataclass
class ArrowheadTiles:
    nt: int
    b: int
    w: int
    a: int
    tiles: Dict[TileKey, np.ndarray] = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nt * self.b + self.a

    def rows(self, i: int) -> int:
        return self.a if i == self.nt else self.b

    def row_start(self, i: int) -> int:
        return i * self.b

    def nsub(self, k: int) -> int:
        return min(self.w, self.nt - 1 - k)

    def struct(self, k: int) -> List[int]:
        """Off-diagonal tile rows of tile column k (band, then the arrow)."""
        if k == self.nt:
            return []
        s = list(range(k + 1, k + self.nsub(k) + 1))
        if self.a > 0:
            s.append(self.nt)
        return s

    def pattern(self) -> Iterator[TileKey]:
        """Lower tile pattern, column by column, diagonal first, corner last."""
        for k in range(self.nt):
            yield (k, k)
            for i in self.struct(k):
                yield (i, k)
        if self.a > 0:
            yield (self.nt, self.nt)

    def nbytes(self) -> int:
        return sum(self.rows(i) * self.rows(k) * 8 for i, k in self.pattern())

    def to_dense(self) -> np.ndarray:
        """Full symmetric dense matrix (small cases only)."""
        n = self.n
        A = np.zeros((n, n))
        for (i, k), T in self.tiles.items():
            r0, c0 = self.row_start(i), self.row_start(k)
            A[r0:r0 + T.shape[0], c0:c0 + T.shape[1]] = T
            if i != k:
                A[c0:c0 + T.shape[1], r0:r0 + T.shape[0]] = T.T
        return A

    @staticmethod
    def from_dense(A: np.ndarray, nt: int, b: int, w: int, a: int) -> "ArrowheadTiles":
        M = ArrowheadTiles(nt, b, w, a)
        for i, k in M.pattern():
            r0, c0 = M.row_start(i), M.row_start(k)
            M.tiles[(i, k)] = np.array(A[r0:r0 + M.rows(i), c0:c0 + M.rows(k)], dtype=np.float64)
        return M


def _set_dominant_diagonal(M: ArrowheadTiles, shift: np.ndarray | float) -> None:
    """diag(A) <- shift + (sum of |off-diagonal| over the full symmetric row)."""
    rowabs = np.zeros(M.n)
    for (i, k), T in M.tiles.items():
        r0, c0 = M.row_start(i), M.row_start(k)
        if i == k:
            off = np.abs(T).sum(axis=1) - np.abs(np.diag(T))
            rowabs[r0:r0 + T.shape[0]] += off
        else:
            absT = np.abs(T)
            rowabs[r0:r0 + T.shape[0]] += absT.sum(axis=1)
            rowabs[c0:c0 + T.shape[1]] += absT.sum(axis=0)
    diag = shift + rowabs
    for i in range(M.nt + (1 if M.a > 0 else 0)):
        r0 = M.row_start(i)
        T = M.tiles[(i, i)]
        np.fill_diagonal(T, diag[r0:r0 + T.shape[0]])


def random_arrowhead(nt: int, b: int, w: int, a: int, seed: int = 0, scale: float = 0.1) -> ArrowheadTiles:
    """Random strictly diagonally dominant SPD arrowhead matrix.

    Off-diagonal entries of every pattern tile are N(0,1)*scale (diagonal
    tiles symmetrised from their lower triangle); the diagonal is then set to
    1 + the row's absolute off-diagonal sum over the full symmetric matrix.
    Tiles are drawn in pattern order, so a seed fixes the matrix.
    """
    if nt < 1 or b < 1 or w < 0 or a < 0:
        raise ValueError("need nt >= 1, b >= 1, w >= 0, a >= 0")
    rng = np.random.default_rng(seed)
    M = ArrowheadTiles(nt, b, w, a)
    for i, k in M.pattern():
        T = rng.standard_normal((M.rows(i), M.rows(k))) * scale
        if i == k:
            T = np.tril(T, -1)
            T = T + T.T
        M.tiles[(i, k)] = T
    _set_dominant_diagonal(M, 1.0)
    return M


def ar1_precision(nt: int, rho: float) -> np.ndarray:
    """AR(1) precision with unit innovation variance: tridiagonal,
    diag [1, 1+rho^2, ..., 1+rho^2, 1], off-diagonal -rho. Its inverse is
    rho^|i-j| / (1 - rho^2)."""
    Q = np.zeros((nt, nt))
    for i in range(nt):
        Q[i, i] = 1.0 + rho * rho if 0 < i < nt - 1 else 1.0
        if i + 1 < nt:
            Q[i, i + 1] = Q[i + 1, i] = -rho
    if nt == 1:
        Q[0, 0] = 1.0 - rho * rho
    return Q


def laplacian2d_plus_identity(side: int) -> np.ndarray:
    """Dense side^2 x side^2 matrix: 2-D 5-point Dirichlet Laplacian (4 on
    the diagonal, -1 to grid neighbours) plus the identity."""
    m = side * side
    Q = np.zeros((m, m))
    for y in range(side):
        for x in range(side):
            p = y * side + x
            Q[p, p] = 5.0
            if x + 1 < side:
                Q[p, p + 1] = Q[p + 1, p] = -1.0
            if y + 1 < side:
                Q[p, p + side] = Q[p + side, p] = -1.0
    return Q


def spatiotemporal(nt: int = 200, side: int = 32, a: int = 64, rho: float = 0.9, tau: float = 1.0,
                   seed: int = 0, band_power: int = 1, couple_arrow: bool = True) -> ArrowheadTiles:
    """Spatio-temporal arrowhead: A_band = kron(Q_t^p, Q_s) + tau*I.

    Q_t is the AR(1) precision (``rho``); ``band_power`` p > 1 replaces it
    with Q_t^p (bandwidth p tiles). The tile size is b = side^2 and the tile
    bandwidth is w = p. The arrow is ``a`` columns of N(0,1) entries; its
    a x a corner has symmetric N(0,1) off-diagonal entries and diagonal
    1 + the full row's absolute sum (corner and band columns). With
    ``couple_arrow=False`` the arrow tiles are zero and the corner is the
    identity, which decouples the arrow (closed-form tests).
    """
    if band_power < 1:
        raise ValueError("band_power >= 1")
    Qt = ar1_precision(nt, rho)
    Qtp = np.linalg.matrix_power(Qt, band_power)
    Qs = laplacian2d_plus_identity(side)
    b = side * side
    w = min(band_power, nt - 1)
    M = ArrowheadTiles(nt, b, w, a)
    rng = np.random.default_rng(seed)
    eye = np.eye(b)
    for k in range(nt):
        for i in [k] + [j for j in M.struct(k) if j != nt]:
            T = Qtp[i, k] * Qs
            if i == k:
                T = T + tau * eye
            M.tiles[(i, k)] = T
    if a > 0:
        if couple_arrow:
            for k in range(nt):
                M.tiles[(nt, k)] = rng.standard_normal((a, b))
            C = np.tril(rng.standard_normal((a, a)), -1)
            C = C + C.T
            rowabs = np.abs(C).sum(axis=1)
            for k in range(nt):
                rowabs += np.abs(M.tiles[(nt, k)]).sum(axis=1)
            np.fill_diagonal(C, 1.0 + rowabs)
            M.tiles[(nt, nt)] = C
        else:
            for k in range(nt):
                M.tiles[(nt, k)] = np.zeros((a, b))
            M.tiles[(nt, nt)] = np.eye(a)
    return M


def sweep_arrowhead(nt: int, b: int, w: int, a: int, tau: float, rho: float, seed: int = 0) -> ArrowheadTiles:
    """One request of a hyperparameter sweep on a fixed pattern.

    The base off-diagonal values are N(0,1)*0.1 drawn from ``seed`` (fixed per
    shape). Per request the band off-diagonals are multiplied by ``rho``, the
    arrow entries are kept, and the diagonal is tau + row absolute sum, so the
    matrix stays strictly diagonally dominant (SPD) for every tau > 0.
    """
    base = random_arrowhead(nt, b, w, a, seed=seed)
    M = ArrowheadTiles(nt, b, w, a)
    for (i, k), T in base.tiles.items():
        T = T.copy()
        if i == k:
            np.fill_diagonal(T, 0.0)
        if i != nt:
            T *= rho
        M.tiles[(i, k)] = T
    _set_dominant_diagonal(M, tau)
    return M


def sweep_base(nt: int, b: int, w: int, a: int, seed: int = 0):
    """The fixed part of a sweep shape, as a request server takes it: the base
    matrix of :func:`sweep_arrowhead` (off-diagonal values, zero diagonal)
    and its band / arrow absolute row sums ``rb``, ``ra`` over the full
    symmetric matrix, so that request (tau, rho) is band x rho, arrow as is,
    diagonal tau + rho rb + ra."""
    base = random_arrowhead(nt, b, w, a, seed=seed)
    M = ArrowheadTiles(nt, b, w, a)
    rb, ra = np.zeros(M.n), np.zeros(M.n)
    for (i, k), T in base.tiles.items():
        T = T.copy()
        if i == k:
            np.fill_diagonal(T, 0.0)
        M.tiles[(i, k)] = T
        acc = ra if (i == nt) else rb
        r0, c0 = M.row_start(i), M.row_start(k)
        absT = np.abs(T)
        acc[r0:r0 + T.shape[0]] += absT.sum(axis=1)
        if i != k:
            acc[c0:c0 + T.shape[1]] += absT.sum(axis=0)
    return M, rb, ra


def ar1_tridiagonal(n: int, rho: float) -> ArrowheadTiles:
    """Scalar AR(1) precision as a b = 1, w = 1, a = 0 arrowhead."""
    return ArrowheadTiles.from_dense(ar1_precision(n, rho), n, 1, 1, 0)


def toeplitz_tridiagonal(n: int) -> ArrowheadTiles:
    """tridiag(-1, 2, -1) of order n as a b = 1, w = 1, a = 0 arrowhead."""
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return ArrowheadTiles.from_dense(A, n, 1, 1, 0)


def batch_shapes(count: int = 64, seed: int = 0, nt_range=(20, 200), b_choices=(128, 256, 512),
                 w_range=(1, 4), a_range=(8, 128)) -> List[Tuple[int, int, int, int]]:
    """Shapes (nt, b, w, a) for an uneven batch: nt, w, a uniform on their
    integer ranges, b drawn from ``b_choices``."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        b = int(rng.choice(b_choices))
        w = int(rng.integers(w_range[0], w_range[1] + 1))
        a = int(rng.integers(a_range[0], a_range[1] + 1))
        out.append((nt, b, w, a))
    return out


def random_arrowhead_packed(nt: int, b: int, w: int, a: int, seed: int, out, scale: float = 0.1) -> None:
    """Fill the float64 torch tensor ``out`` (at least nt*colstride + a*a
    elements, any device) with a random strictly diagonally dominant SPD
    arrowhead matrix in the packed band+arrow layout: column-major tiles,
    tile column k at k*colstride with colstride = (1+w) b^2 + a b, tiles
    (k,k), (k+1,k) .. (k+w,k), (nt,k) in that slot, the corner at
    nt*colstride. Same recipe as :func:`random_arrowhead` (off-diagonal
    N(0,1)*scale, diagonal tiles symmetric, diagonal 1 + full-row absolute
    sum), drawn with a torch generator seeded by ``seed``."""
    import torch

    w = min(w, nt - 1)
    dev = out.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    colstride = (1 + w) * b * b + a * b
    n = nt * b + a
    rows = lambda i: a if i == nt else b  # noqa: E731
    start = lambda i: i * b  # noqa: E731  (the arrow starts at nt*b)

    def view(i, k):
        if k == nt:
            off = nt * colstride
        elif i == nt:
            off = k * colstride + (1 + w) * b * b
        else:
            off = k * colstride + (i - k) * b * b
        r, c = rows(i), rows(k)
        return out[off:off + r * c].view(c, r).t()

    pattern = []
    for k in range(nt):
        pattern.append((k, k))
        pattern += [(i, k) for i in range(k + 1, min(k + w, nt - 1) + 1)]
        if a > 0:
            pattern.append((nt, k))
    if a > 0:
        pattern.append((nt, nt))
    rowabs = torch.zeros(n, dtype=torch.float64, device=dev)
    for i, k in pattern:
        r, c = rows(i), rows(k)
        T = torch.randn((r, c), generator=gen, dtype=torch.float64, device=dev) * scale
        if i == k:
            T = torch.tril(T, -1)
            T = T + T.t()
            rowabs[start(i):start(i) + r] += T.abs().sum(dim=1)
        else:
            absT = T.abs()
            rowabs[start(i):start(i) + r] += absT.sum(dim=1)
            rowabs[start(k):start(k) + c] += absT.sum(dim=0)
        view(i, k).copy_(T)
    for i in range(nt + (1 if a > 0 else 0)):
        r = rows(i)
        view(i, i).diagonal().copy_(1.0 + rowabs[start(i):start(i) + r])


def sweep_base_packed(nt: int, b: int, w: int, a: int, seed: int, out, scale: float = 0.1):
    """Base matrix of a sweep shape drawn on a torch device into ``out`` (the
    packed layout, as :func:`random_arrowhead_packed`): off-diagonal entries
    N(0,1)*scale, zero diagonal. Returns (rb, ra): the band and arrow absolute
    row sums over the full symmetric matrix (float64 tensors of length n on
    ``out``'s device)."""
    import torch

    w = min(w, nt - 1)
    dev = out.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    colstride = (1 + w) * b * b + a * b
    n = nt * b + a
    rb = torch.zeros(n, dtype=torch.float64, device=dev)
    ra = torch.zeros(n, dtype=torch.float64, device=dev)
    for k in range(nt + (1 if a > 0 else 0)):
        rows_k = a if k == nt else b
        tiles = [(k, k)] if k == nt else ([(k, k)] + [(i, k) for i in range(k + 1, min(k + w, nt - 1) + 1)] +
                                          ([(nt, k)] if a > 0 else []))
        for i, kk in tiles:
            r = a if i == nt else b
            if kk == nt:
                off = nt * colstride
            elif i == nt:
                off = kk * colstride + (1 + w) * b * b
            else:
                off = kk * colstride + (i - kk) * b * b
            T = torch.randn((r, rows_k), generator=gen, dtype=torch.float64, device=dev) * scale
            if i == kk:
                T = torch.tril(T, -1)
                T = T + T.t()
            acc = ra if i == nt else rb
            absT = T.abs()
            acc[i * b:i * b + r] += absT.sum(dim=1)
            if i != kk:
                acc[kk * b:kk * b + rows_k] += absT.sum(dim=0)
            out[off:off + r * rows_k].view(rows_k, r).t().copy_(T)
    return rb, ra
