"""GPU: the wide tier on R-MAT rows at full width.  Every 100th row of R-MAT
scale 20 whose flop bound exceeds 24,576 (1,288 rows, the rows the wide tier
takes in the full product), times the whole scale-20 matrix (k = 2^20
columns), in float64 through the C ABI, against the CPU oracle entry by entry:
structure exact, values within 1e-12 * sum |a||b| (the wide tier adds into C
with atomics in no fixed order).  The rows' values do not fit shared memory
beside their 128 KB bit vectors, so they take the kept-bit-vector path: rank
tables from the block scan, C's columns in claimed rounds, per-row piece sizes
of the entry-piece walk."""
import numpy as np
import pytest

import oracle
from paper_2103_11991_gb300 import inputs as I
from tests._gpu import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu


def _heavy_rows(R, step):
    rp = R.rowptr.astype(np.int64)
    flop = oracle.row_flops(R, R)
    rows = np.nonzero(np.asarray(flop) > 24576)[0][::step]
    cnt = np.diff(rp)[rows]
    srp = np.concatenate(([0], np.cumsum(cnt))).astype(np.int32)
    sci = np.concatenate([R.colind[rp[i]:rp[i + 1]] for i in rows]).astype(np.int32)
    sva = np.concatenate([R.vals[rp[i]:rp[i + 1]] for i in rows])
    return I.ensure_csr(len(rows), R.n, srp, sci, sva)


def test_rmat20_heavy_rows_full_width():
    R = I.config_inputs("rmat20")["A"]
    S = _heavy_rows(R, 100)
    rp, ci, va, arith, st = run_gpu(S, R, arith=1)
    assert arith == 1
    assert st["num_dense_rows"] + st["num_cta_rows"] == S.m  # every row in the wide tier
    ref = check_against_oracle(S, R, rp, ci, va)
    assert np.diff(ref.rowptr).max() > 100_000
