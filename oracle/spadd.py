"""Sparse matrix addition oracle: C = alpha A + beta B.

TEST INFRASTRUCTURE ONLY (the same rule as the rest of ``oracle/``).

Written from the Kokkos Kernels paper, Sec. "SpAdd": A, B and C are m x n in
CSR; every stored entry of A and of B lands in C, and entries of the same row
and column merge additively into one entry of C (for repeated columns within A
or B too).  Row i of C holds the union of the columns of A(i,:) and B(i,:), in
ascending order; the structure is structural (a sum that cancels keeps an
explicit 0.0).  Values, per (i, c): v = sum over A's entries (i, c) in storage
order of alpha * a, then sum over B's entries (i, c) in storage order of
beta * b, accumulated left to right starting from the first term.

Parity status: pinned by ``tests/test_oracle_spadd.py`` (dense brute force,
beta = 0 and A + (-A) structures, commutativity, the SpGEMM identity
A + B = [A B] [I; I] checked with the Gustavson oracle).
"""
from __future__ import annotations

import numpy as np

from . import OracleCSR


def spadd(A, B, alpha: float = 1.0, beta: float = 1.0) -> OracleCSR:
    """C = alpha A + beta B (int64 row pointers, ascending columns)."""
    if A.m != B.m or A.n != B.n:
        raise ValueError("A and B have different shapes")
    m = A.m
    rowptr = np.zeros(m + 1, dtype=np.int64)
    cols_out, vals_out = [], []
    alpha, beta = float(alpha), float(beta)
    for i in range(m):
        acc = {}
        for p in range(int(A.rowptr[i]), int(A.rowptr[i + 1])):
            c = int(A.colind[p])
            t = alpha * float(A.vals[p])
            acc[c] = acc[c] + t if c in acc else t
        for p in range(int(B.rowptr[i]), int(B.rowptr[i + 1])):
            c = int(B.colind[p])
            t = beta * float(B.vals[p])
            acc[c] = acc[c] + t if c in acc else t
        cols = sorted(acc)
        cols_out.extend(cols)
        vals_out.extend(acc[c] for c in cols)
        rowptr[i + 1] = rowptr[i] + len(cols)
    return OracleCSR(m, A.n, rowptr, np.array(cols_out, dtype=np.int32),
                     np.array(vals_out, dtype=np.float64))


def spadd_abs(A, B, alpha: float = 1.0, beta: float = 1.0) -> np.ndarray:
    """Per-entry scale of the error bound: sum |alpha a| + sum |beta b|."""
    from types import SimpleNamespace
    Aa = SimpleNamespace(m=A.m, n=A.n, rowptr=A.rowptr, colind=A.colind, vals=np.abs(A.vals))
    Ba = SimpleNamespace(m=B.m, n=B.n, rowptr=B.rowptr, colind=B.colind, vals=np.abs(B.vals))
    return spadd(Aa, Ba, abs(alpha), abs(beta)).vals
