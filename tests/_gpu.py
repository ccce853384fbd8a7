"""GPU-side helpers for the parity tests (run the C ABI, compare with the oracle)."""
import numpy as np

import oracle
from tests._util import assert_structure_equal, assert_values_within


def run_gpu(A, B, **opts):
    from paper_2103_11991_gb300 import spgemm as K
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM(**opts) as op:
        C = op(dA, dB)
        op.sync()
        arith = op.last_arith()
        stats = op.stats()
    return (C.rowptr.cpu().numpy(), C.colind.cpu().numpy(), C.vals.cpu().numpy(), arith, stats)


def check_against_oracle(A, B, rowptr, colind, vals, exact=False):
    ref = oracle.spgemm(A, B)
    assert_structure_equal(rowptr, colind, ref.rowptr, ref.colind)
    if exact:
        assert np.array_equal(vals, ref.vals), "values differ (exact case)"
    else:
        ab = oracle.spgemm_abs(A, B)
        assert_values_within(vals, ref.vals, ab.vals)
    return ref
