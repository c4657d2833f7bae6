"""The synthetic generators (no method arithmetic): the packed device-side
recipe produces a symmetric, strictly diagonally dominant (hence SPD) matrix
in the packed band+arrow layout and leaves unused slots untouched."""
import numpy as np
import pytest

from paper_2504_19171_gb300 import workloads as W


@pytest.mark.parametrize("shape", [(5, 7, 2, 3), (1, 4, 0, 0), (6, 3, 1, 0), (3, 2, 4, 5)])
def test_packed_generator_is_spd_and_dominant(shape):
    torch = pytest.importorskip("torch")
    nt, b, w, a = shape
    w = min(w, nt - 1)
    colstride = (1 + w) * b * b + a * b
    x = torch.full((nt * colstride + a * a,), float("nan"), dtype=torch.float64)
    W.random_arrowhead_packed(nt, b, w, a, 7, x)
    M = W.ArrowheadTiles(nt, b, w, a)
    flat = x.numpy()
    for i, k in M.pattern():
        r, c = M.rows(i), M.rows(k)
        off = nt * colstride if k == nt else (k * colstride + (1 + w) * b * b if i == nt else k * colstride + (i - k) * b * b)
        M.tiles[(i, k)] = flat[off:off + r * c].reshape(c, r).T
    D = M.to_dense()
    assert np.all(np.isfinite(D))
    assert np.array_equal(D, D.T)
    off = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.all(np.diag(D) > off)
    assert np.linalg.eigvalsh(D).min() > 0
    # a second draw with the same seed is identical
    y = torch.full_like(x, float("nan"))
    W.random_arrowhead_packed(nt, b, w, a, 7, y)
    assert torch.equal(torch.nan_to_num(x, 123.0), torch.nan_to_num(y, 123.0))


def test_sweep_base_packed_row_sums():
    """rb / ra are the band / arrow absolute row sums of the packed base, so a
    request (tau, rho) is strictly diagonally dominant."""
    torch = pytest.importorskip("torch")
    nt, b, w, a = 4, 5, 2, 3
    colstride = (1 + w) * b * b + a * b
    x = torch.zeros(nt * colstride + a * a, dtype=torch.float64)
    rb, ra = W.sweep_base_packed(nt, b, w, a, 3, x)
    M = W.ArrowheadTiles(nt, b, w, a)
    flat = x.numpy()
    for i, k in M.pattern():
        r, c = M.rows(i), M.rows(k)
        off = nt * colstride if k == nt else (k * colstride + (1 + w) * b * b if i == nt else k * colstride + (i - k) * b * b)
        M.tiles[(i, k)] = flat[off:off + r * c].reshape(c, r).T.copy()
    D = M.to_dense()
    assert np.all(np.diag(D) == 0) and np.array_equal(D, D.T)
    n = nt * b + a
    band = np.zeros_like(D)
    band[:nt * b, :nt * b] = D[:nt * b, :nt * b]
    arrow = D - band
    assert np.allclose(np.abs(band).sum(axis=1), rb.numpy())
    assert np.allclose(np.abs(arrow).sum(axis=1), ra.numpy())
    tau, rho = 0.5, 0.7
    A = rho * band + arrow
    A[np.diag_indices(n)] = tau + rho * rb.numpy() + ra.numpy()
    assert np.linalg.eigvalsh(A).min() > 0
