"""Jacobi-fused SpGEMM oracle: C = (I - omega D^-1 A) B.

TEST INFRASTRUCTURE ONLY (the same rule as the rest of ``oracle/``: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it; it
imports nothing from the product path).

Written from the Kokkos Kernels paper, Sec. "Jacobi-Fused SpGEMM Kernel": A is
m x m with every diagonal entry present and nonzero, B is m x k, D = diag(A),
and row i of the result is

    E(i,:) = sum_{A(i,j) != 0} A(i,j) B(j,:)          (Eq. 1, the plain product)
    C(i,:) = B(i,:) - omega D^-1(i) E(i,:)

so C has the structure of E (B(i,:) is inside E(i,:) because A(i,i) is stored).
Steps, in that order: E from the Gustavson oracle (``oracle.spgemm``), the
diagonal D(i) as the sum of the row's stored (i,i) entries (repeated entries
add, as in every oracle here), the row factor s_i = -omega / D(i) computed
once per row, then c = s_i * e + b for every column of E(i,:), with b = B(i,c)
(repeats summed) or 0 where B(i,:) has no entry.  A row without a diagonal
entry, or whose diagonal sums to zero, is outside the method's assumption and
raises ValueError.

Parity status: pinned by ``tests/test_oracle_jacobi.py`` (dense brute force on
tiny inputs, omega = 0, the closed form for the 1D Laplacian with B = I, the
row-sum invariant of prolongator smoothing, rejection of a missing diagonal).
"""
from __future__ import annotations

import numpy as np

from . import OracleCSR, spgemm, spgemm_abs


def diagonal(A) -> np.ndarray:
    """D(i) = sum of the stored (i,i) entries of square A; ValueError if a row
    has none or they sum to zero."""
    if A.m != A.n:
        raise ValueError("Jacobi needs a square A")
    rows = np.repeat(np.arange(A.m, dtype=np.int64), np.diff(np.asarray(A.rowptr, dtype=np.int64)))
    cols = np.asarray(A.colind, dtype=np.int64)
    on = rows == cols
    d = np.zeros(A.m, dtype=np.float64)
    np.add.at(d, rows[on], np.asarray(A.vals, dtype=np.float64)[on])
    has = np.zeros(A.m, dtype=bool)
    has[rows[on]] = True
    if not has.all():
        raise ValueError(f"row {int(np.nonzero(~has)[0][0])} of A has no diagonal entry")
    if (d == 0.0).any():
        raise ValueError(f"row {int(np.nonzero(d == 0.0)[0][0])} of A has a zero diagonal")
    return d


def _b_at(B, E) -> np.ndarray:
    """B(i,c) at every entry (i,c) of E (repeats of B summed, 0 where B has none)."""
    k = np.int64(max(B.n, 1))
    brows = np.repeat(np.arange(B.m, dtype=np.int64), np.diff(np.asarray(B.rowptr, dtype=np.int64)))
    bkey = brows * k + np.asarray(B.colind, dtype=np.int64)
    ukey, inv = np.unique(bkey, return_inverse=True)
    bsum = np.zeros(len(ukey), dtype=np.float64)
    np.add.at(bsum, inv, np.asarray(B.vals, dtype=np.float64))
    erows = np.repeat(np.arange(E.m, dtype=np.int64), np.diff(E.rowptr))
    ekey = erows * k + E.colind.astype(np.int64)
    out = np.zeros(len(ekey), dtype=np.float64)
    if len(ukey):
        pos = np.searchsorted(ukey, ekey)
        pos_c = np.minimum(pos, len(ukey) - 1)
        hit = ukey[pos_c] == ekey
        out[hit] = bsum[pos_c[hit]]
        if hit.sum() != len(ukey):
            raise ValueError("B(i,:) is not inside E(i,:): a diagonal entry is missing")
    return out


def jacobi_spgemm(A, B, omega: float) -> OracleCSR:
    """C = (I - omega D^-1 A) B as CSR (int64 row pointers)."""
    d = diagonal(A)
    if A.n != B.m:
        raise ValueError("inner dimensions differ")
    E = spgemm(A, B)
    s = -float(omega) / d
    rows = np.repeat(np.arange(E.m, dtype=np.int64), np.diff(E.rowptr))
    vals = s[rows] * E.vals + _b_at(B, E)
    return OracleCSR(E.m, E.n, E.rowptr, E.colind, vals)


def jacobi_abs(A, B, omega: float) -> np.ndarray:
    """Per-entry scale of the error bound: |s_i| * sum |a_ij||b_jc| + |B(i,c)|."""
    d = diagonal(A)
    E = spgemm_abs(A, B)
    s = np.abs(float(omega) / d)
    rows = np.repeat(np.arange(E.m, dtype=np.int64), np.diff(E.rowptr))
    from types import SimpleNamespace
    Babs = SimpleNamespace(m=B.m, n=B.n, rowptr=B.rowptr, colind=B.colind, vals=np.abs(B.vals))
    return s[rows] * E.vals + _b_at(Babs, E)
