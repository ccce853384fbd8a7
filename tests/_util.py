"""Helpers shared by the tests: golden fixture parsing and CSR comparison."""
import os

import numpy as np

from paper_2103_11991_gb300.inputs import CSR, _from_sorted_coo

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Per-entry value tolerance: |c - c_ref| <= REL_TOL * sum_j |a_ij| |b_jc|.
REL_TOL = 1e-12


def read_golden_rows(name):
    """Parse a golden file into {case: {row: {col: value}}}."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0].lstrip("-").isdigit():
                case, row, ents = "C", int(parts[0]), parts[1:]
            else:
                case, row, ents = parts[0], int(parts[1]), parts[2:]
            d = out.setdefault(case, {}).setdefault(row, {})
            for e in ents:
                c, v = e.split(":")
                d[int(c)] = float(v)
    return out


def csr_from_rows(rows: dict, m: int, n: int) -> CSR:
    r, c, v = [], [], []
    for i in sorted(rows):
        for col in sorted(rows[i]):
            r.append(i)
            c.append(col)
            v.append(rows[i][col])
    return _from_sorted_coo(m, n, np.array(r, np.int64), np.array(c, np.int64), np.array(v))


def pattern_dense(M) -> np.ndarray:
    d = np.zeros((M.m, M.n), dtype=bool)
    rows = np.repeat(np.arange(M.m), np.diff(np.asarray(M.rowptr, dtype=np.int64)))
    d[rows, np.asarray(M.colind, dtype=np.int64)] = True
    return d


def assert_structure_equal(rowptr, colind, ref_rowptr, ref_colind):
    rowptr = np.asarray(rowptr, dtype=np.int64)
    ref_rowptr = np.asarray(ref_rowptr, dtype=np.int64)
    assert rowptr.shape == ref_rowptr.shape
    bad = np.nonzero(rowptr != ref_rowptr)[0]
    assert len(bad) == 0, f"row pointers differ first at {bad[:5]}"
    colind = np.asarray(colind, dtype=np.int64)
    ref_colind = np.asarray(ref_colind, dtype=np.int64)
    assert colind.shape == ref_colind.shape
    bad = np.nonzero(colind != ref_colind)[0]
    assert len(bad) == 0, f"column indices differ first at {bad[:5]}"


def assert_values_within(vals, ref_vals, absbound, rel=REL_TOL):
    vals = np.asarray(vals, dtype=np.float64)
    ref_vals = np.asarray(ref_vals, dtype=np.float64)
    err = np.abs(vals - ref_vals)
    lim = rel * np.asarray(absbound, dtype=np.float64)
    bad = np.nonzero(~(err <= lim))[0]
    assert len(bad) == 0, (f"{len(bad)} values outside {rel}*sum|a||b|; first {bad[:5]}: "
                           f"got {vals[bad[:3]]} want {ref_vals[bad[:3]]} bound {lim[bad[:3]]}")
