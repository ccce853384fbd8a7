"""CPU oracle for two-phase SpGEMM and for the learned row-capacity predictor.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2103_11991_gb300``) never imports it, and
it imports nothing from the product path: it shares no code, header, helper or
constant with the CUDA library.  Its inputs come from the seeded generators in
``paper_2103_11991_gb300.inputs``, a module that holds no SpGEMM arithmetic.

Contents
--------
``spgemm_oracle.c``  Gustavson SpGEMM, Kokkos Kernels paper Sec. "Standard SpGEMM
                     Kernel", Eq. 1, symbolic and numeric phases, plain C,
                     single thread, fp64, built with -ffp-contract=off.
``mlp.py``           fp64 numpy forward/backward of the row-capacity MLP.
``features.py``      row features and capacity-bucket labels written from their
                     plain definitions (numpy).
``jacobi.py``        Jacobi-fused SpGEMM C = (I - omega D^-1 A) B, paper Sec.
                     "Jacobi-Fused SpGEMM Kernel", on top of the Gustavson oracle.
``spadd.py``         sparse matrix addition C = alpha A + beta B, paper Sec. "SpAdd"
                     (per-row merge of the two rows, plain Python).

Parity status: every function here is pinned by ``tests/test_oracle.py``,
``tests/test_oracle_mlp.py``, ``tests/test_oracle_jacobi.py`` and
``tests/test_oracle_spadd.py`` (dense brute force, closed forms, invariants,
finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spgemm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_spgemm.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no vectorisation tricks, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            i32 = ctypes.c_int32
            lib.oracle_symbolic_rows.argtypes = [i32, i32, i32, i32p, i32p, i32p, i32p, i64p]
            lib.oracle_symbolic_rows.restype = ctypes.c_int
            lib.oracle_numeric_rows.argtypes = [i32, i32, i32, i32p, i32p, f64p, i32p, i32p, f64p,
                                                i64p, i32p, f64p]
            lib.oracle_numeric_rows.restype = ctypes.c_int
            lib.oracle_row_flops.argtypes = [i32, i32, i32p, i32p, i32p, i64p]
            lib.oracle_row_flops.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleCSR:
    """Result of the oracle: int64 row pointers, int32 columns, fp64 values."""

    def __init__(self, m, n, rowptr, colind, vals):
        self.m, self.n = m, n
        self.rowptr, self.colind, self.vals = rowptr, colind, vals

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self):
        d = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        np.add.at(d, (rows, self.colind.astype(np.int64)), self.vals)
        return d


def symbolic(A, B, r0: int = 0, r1: int | None = None) -> np.ndarray:
    """Symbolic phase on rows [r0, r1): int64 counts nnz(C(i,:))."""
    if A.n != B.m:
        raise ValueError("inner dimensions differ")
    lib = _load()
    r1 = A.m if r1 is None else r1
    arp, aci = _c(A.rowptr, np.int32), _c(A.colind, np.int32)
    brp, bci = _c(B.rowptr, np.int32), _c(B.colind, np.int32)
    counts = np.zeros(max(r1 - r0, 0), dtype=np.int64)
    if r1 > r0:
        rc = lib.oracle_symbolic_rows(r0, r1, B.n, _p(arp, ctypes.c_int32), _p(aci, ctypes.c_int32),
                                      _p(brp, ctypes.c_int32), _p(bci, ctypes.c_int32),
                                      _p(counts, ctypes.c_int64))
        if rc != 0:
            raise MemoryError("oracle symbolic: scratch allocation failed")
    return counts


def numeric(A, B, counts: np.ndarray, r0: int = 0, r1: int | None = None,
            a_vals=None, b_vals=None) -> OracleCSR:
    """Numeric phase on rows [r0, r1) given the symbolic counts of those rows;
    returns the block of C as CSR (row pointers relative to the block)."""
    lib = _load()
    r1 = A.m if r1 is None else r1
    nr = max(r1 - r0, 0)
    offsets = np.zeros(nr + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    nnz = int(offsets[-1])
    colind = np.zeros(nnz, dtype=np.int32)
    vals = np.zeros(nnz, dtype=np.float64)
    arp, aci = _c(A.rowptr, np.int32), _c(A.colind, np.int32)
    brp, bci = _c(B.rowptr, np.int32), _c(B.colind, np.int32)
    av = _c(A.vals if a_vals is None else a_vals, np.float64)
    bv = _c(B.vals if b_vals is None else b_vals, np.float64)
    if nr > 0:
        rc = lib.oracle_numeric_rows(r0, r1, B.n, _p(arp, ctypes.c_int32), _p(aci, ctypes.c_int32),
                                     _p(av, ctypes.c_double), _p(brp, ctypes.c_int32),
                                     _p(bci, ctypes.c_int32), _p(bv, ctypes.c_double),
                                     _p(offsets, ctypes.c_int64), _p(colind, ctypes.c_int32),
                                     _p(vals, ctypes.c_double))
        if rc == -1:
            raise MemoryError("oracle numeric: scratch allocation failed")
        if rc == -2:
            raise ValueError("oracle numeric: counts disagree with the structure")
    return OracleCSR(nr, B.n, offsets, colind, vals)


def spgemm(A, B, r0: int = 0, r1: int | None = None) -> OracleCSR:
    """C = A*B (rows [r0, r1) of it): symbolic, scan, numeric."""
    r1 = A.m if r1 is None else r1
    return numeric(A, B, symbolic(A, B, r0, r1), r0, r1)


def spgemm_abs(A, B, r0: int = 0, r1: int | None = None) -> OracleCSR:
    """|A|*|B| on the same structure: per entry the sum of |a_ij||b_jc|, the
    scale of the per-entry error bound 1e-12 * sum |a||b|."""
    r1 = A.m if r1 is None else r1
    return numeric(A, B, symbolic(A, B, r0, r1), r0, r1, np.abs(A.vals), np.abs(B.vals))


def spgemm_rows(A, B, rows) -> dict:
    """C(i,:) for each listed row i, as {i: (cols, vals, absbound)}."""
    out = {}
    for i in np.asarray(rows, dtype=np.int64).tolist():
        c = spgemm(A, B, i, i + 1)
        ab = spgemm_abs(A, B, i, i + 1)
        out[i] = (c.colind.copy(), c.vals.copy(), ab.vals.copy())
    return out


def row_flops(A, B, r0: int = 0, r1: int | None = None) -> np.ndarray:
    """Per-row flop upper bound sum_{j in A(i,:)} nnz(B(j,:)) (int64)."""
    lib = _load()
    r1 = A.m if r1 is None else r1
    arp, aci = _c(A.rowptr, np.int32), _c(A.colind, np.int32)
    brp = _c(B.rowptr, np.int32)
    out = np.zeros(max(r1 - r0, 0), dtype=np.int64)
    if r1 > r0:
        lib.oracle_row_flops(r0, r1, _p(arp, ctypes.c_int32), _p(aci, ctypes.c_int32),
                             _p(brp, ctypes.c_int32), _p(out, ctypes.c_int64))
    return out
