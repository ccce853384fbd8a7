"""Pins of the SpAdd oracle, C = alpha A + beta B (Kokkos Kernels paper, Sec.
"SpAdd"), against facts that do not come from it: the dense sum on tiny
inputs, the structure of beta = 0 and of A + (-A), commutativity, and the
identity A + B = [A B] [I; I] evaluated with the Gustavson SpGEMM oracle."""
import numpy as np
import pytest

import oracle as O
from oracle import spadd as S
from paper_2103_11991_gb300 import inputs as I
from tests._util import assert_structure_equal, assert_values_within, pattern_dense


def _pair(m, n, dens, seed, **kw):
    A = I.random_sparse(m, n, dens, seed, **kw)
    B = I.random_sparse(m, n, dens, seed + 31, duplicates=kw.get("unsorted", False),
                        unsorted=kw.get("duplicates", False))
    return A, B


@pytest.mark.parametrize("seed", range(10))
def test_dense_sum(seed):
    u = I.uniform01(seed, "sa.dims", 2)
    m, n = 1 + int(u[0] * 30), 1 + int(u[1] * 30)
    A, B = _pair(m, n, [0.0, 0.1, 0.3, 0.7][seed % 4], seed, duplicates=seed % 2 == 0,
                 unsorted=seed % 3 == 0)
    al, be = [(1.0, 1.0), (2.5, -0.5), (-1.0, 3.0)][seed % 3]
    C = S.spadd(A, B, al, be)
    pat = pattern_dense(A) | pattern_dense(B)
    assert np.array_equal(pattern_dense(C), pat)
    for i in range(C.m):
        assert np.all(np.diff(C.colind[C.rowptr[i]:C.rowptr[i + 1]]) > 0)
    D = al * A.to_dense() + be * B.to_dense()
    Dabs = abs(al) * np.abs(A.to_dense()) + abs(be) * np.abs(B.to_dense())
    rows = np.repeat(np.arange(C.m), np.diff(C.rowptr))
    assert_values_within(C.vals, D[rows, C.colind], Dabs[rows, C.colind] + 1e-300)
    if seed % 2 and seed % 3:  # no repeated entries (they count each in the oracle's bound)
        assert np.allclose(S.spadd_abs(A, B, al, be), Dabs[rows, C.colind], rtol=1e-15, atol=0)


def test_beta_zero_and_cancellation_keep_structure():
    A, B = _pair(25, 20, 0.2, 3)
    C = S.spadd(A, B, 1.0, 0.0)
    assert np.array_equal(pattern_dense(C), pattern_dense(A) | pattern_dense(B))
    Bonly = pattern_dense(B) & ~pattern_dense(A)
    rows = np.repeat(np.arange(C.m), np.diff(C.rowptr))
    assert np.all(C.vals[Bonly[rows, C.colind]] == 0.0)
    Z = S.spadd(A, A, 1.0, -1.0)
    assert_structure_equal(Z.rowptr, Z.colind, O.spgemm(A, I.identity(A.n)).rowptr,
                           O.spgemm(A, I.identity(A.n)).colind)
    assert np.all(Z.vals == 0.0)


def test_commutative():
    A, B = _pair(30, 25, 0.15, 8)
    C1 = S.spadd(A, B, 1.5, -2.0)
    C2 = S.spadd(B, A, -2.0, 1.5)
    assert_structure_equal(C1.rowptr, C1.colind, C2.rowptr, C2.colind)
    assert np.array_equal(C1.vals, C2.vals)  # two terms per entry: one rounding either way


def test_sum_as_product_with_stacked_identity():
    # alpha A + beta B = [alpha A, beta B] * [I; I]
    A, B = _pair(40, 35, 0.1, 11, unsorted=True)
    al, be = 0.75, -1.25
    m, n = A.m, A.n
    ra = np.repeat(np.arange(m), np.diff(A.rowptr))
    rb = np.repeat(np.arange(m), np.diff(B.rowptr))
    rows = np.concatenate([ra, rb])
    cols = np.concatenate([A.colind.astype(np.int64), B.colind.astype(np.int64) + n])
    vals = np.concatenate([al * A.vals, be * B.vals])
    o = np.argsort(rows, kind="stable")
    AB = I._from_sorted_coo(m, 2 * n, rows[o], cols[o], vals[o])
    st = np.arange(2 * n) % n
    IS = I.ensure_csr(2 * n, n, np.arange(2 * n + 1), st, np.ones(2 * n))
    P = O.spgemm(AB, IS)
    C = S.spadd(A, B, al, be)
    assert_structure_equal(C.rowptr, C.colind, P.rowptr, P.colind)
    assert_values_within(C.vals, P.vals, S.spadd_abs(A, B, al, be) + 1e-300)
