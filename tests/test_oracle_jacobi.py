"""Pins of the Jacobi-fused SpGEMM oracle, C = (I - omega D^-1 A) B (Kokkos
Kernels paper, Sec. "Jacobi-Fused SpGEMM Kernel"), against facts that do not
come from the oracle: the dense formula on tiny inputs, omega = 0, the closed
form for the 1D Laplacian times the identity, the row-sum invariant of
prolongator smoothing, and rejection of a row without a diagonal."""
import numpy as np
import pytest

import oracle as O
from oracle import jacobi as J
from paper_2103_11991_gb300 import inputs as I
from tests._util import assert_values_within, pattern_dense


def _square(m, dens, seed, **kw):
    return I.with_diagonal(I.random_sparse(m, m, dens, seed, **kw), seed + 500,
                           split=kw.get("duplicates", False))


@pytest.mark.parametrize("seed", range(10))
def test_dense_formula_random(seed):
    u = I.uniform01(seed, "jtest.dims", 3)
    m, k = 1 + int(u[0] * 30), 1 + int(u[1] * 30)
    omega = [0.5, 2.0 / 3.0, 1.3, -0.7][seed % 4]
    A = _square(m, [0.05, 0.2, 0.5][seed % 3], seed, duplicates=seed % 2 == 0,
                unsorted=seed % 3 == 0)
    B = I.random_sparse(m, k, 0.3, seed + 70, duplicates=seed % 4 == 1, unsorted=seed % 2 == 1)
    C = J.jacobi_spgemm(A, B, omega)
    Ad, Bd = A.to_dense(), B.to_dense()
    d = np.diag(Ad)
    want = Bd - omega * ((Ad @ Bd) / d[:, None])
    scale = np.abs(omega / d)[:, None] * (np.abs(Ad) @ np.abs(Bd)) + np.abs(Bd)
    # structure: that of A*B (B's own rows are inside it)
    pat = (pattern_dense(A).astype(np.int64) @ pattern_dense(B).astype(np.int64)) > 0
    assert np.array_equal(pattern_dense(C), pat)
    rows = np.repeat(np.arange(C.m), np.diff(C.rowptr))
    assert_values_within(C.vals, want[rows, C.colind], scale[rows, C.colind] + 1e-300)
    # the bound the GPU is held to: the same scale, taken over the stored
    # entries (repeated entries count each, so it can only be larger)
    ja = J.jacobi_abs(A, B, omega)
    assert np.all(ja >= scale[rows, C.colind] * (1 - 1e-12))
    if seed % 2 == 1 and seed % 4 != 1:  # no repeated entries in A or B
        assert np.allclose(ja, scale[rows, C.colind], rtol=1e-12, atol=0)


def test_omega_zero_gives_b():
    A = _square(20, 0.2, 3)
    B = I.random_sparse(20, 15, 0.3, 4)
    C = J.jacobi_spgemm(A, B, 0.0)
    rows = np.repeat(np.arange(C.m), np.diff(C.rowptr))
    Bd = B.to_dense()
    assert np.array_equal(C.vals, Bd[rows, C.colind])


def test_laplacian_1d_times_identity_closed_form():
    # A = tridiag(-1, 2, -1), B = I, omega = 1/2: C = I - A/4, exactly
    # (interior row [1/4, 1/2, 1/4], boundary rows [1/2, 1/4])
    n = 9
    A = I.laplacian_1d(n)
    C = J.jacobi_spgemm(A, I.identity(n), 0.5)
    Cd = C.to_dense()
    want = np.eye(n) - A.to_dense() / 4.0
    assert np.array_equal(Cd, want)
    assert C.nnz == 3 * n - 2


def test_prolongator_smoothing_keeps_constants_on_interior_rows():
    # 2D 5-point Laplacian (4/-1): interior rows sum to 0, so (I - w D^-1 A) 1 = 1
    # there; P (aggregation, one 1.0 per row) maps 1 to 1, so C 1 = 1 on interior rows
    g = 12
    A = I.stencil_2d(g, g, 5, 4.0, -1.0)
    rows = np.arange(g * g)
    agg = (rows % g) // 2 + (g // 2) * ((rows // g) // 2)
    P = I.ensure_csr(g * g, (g // 2) ** 2, np.arange(g * g + 1), agg, np.ones(g * g))
    C = J.jacobi_spgemm(A, P, 2.0 / 3.0)
    sums = np.add.reduceat(C.vals, C.rowptr[:-1].astype(np.int64))
    x, y = rows % g, rows // g
    interior = (x > 0) & (x < g - 1) & (y > 0) & (y < g - 1)
    assert np.allclose(sums[interior], 1.0, rtol=0, atol=1e-14)
    assert not np.allclose(sums[~interior], 1.0)


def test_missing_or_zero_diagonal_is_rejected():
    A = I.laplacian_1d(5)
    rp = A.rowptr.copy()
    # drop the diagonal of row 2
    keep = np.ones(A.nnz, dtype=bool)
    keep[rp[2] + 1] = False
    A2 = I.ensure_csr(5, 5, np.array([0, 2, 5, 7, 10, 12]) - np.array([0, 0, 0, 1, 1, 1]),
                      A.colind[keep], A.vals[keep])
    with pytest.raises(ValueError):
        J.jacobi_spgemm(A2, I.identity(5), 0.5)
    A3 = A.copy()
    A3.vals[rp[1] + 1] = 0.0
    with pytest.raises(ValueError):
        J.jacobi_spgemm(A3, I.identity(5), 0.5)
