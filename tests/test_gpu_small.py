"""GPU: the small-product path (options.small_max_rows; kk_small.cu): both
phases as one launch of one CTA for A of at most 4,096 rows whose rows of C
hold at most 16 columns.  Against the oracle through the C ABI: structure and
values exact (float64 in A-row storage order, the oracle's order); a row of
C with more columns hands the call to the tiered path; indices out of range
are reported; the Jacobi-fused numeric phase and numeric refreshes work on the
small path's symbolic result."""
import numpy as np
import pytest

import oracle
from oracle import jacobi as J
from paper_2103_11991_gb300 import inputs as I
from tests._gpu import check_against_oracle, run_gpu
from tests._util import assert_structure_equal, assert_values_within

pytestmark = pytest.mark.gpu


def test_stencil2d_64_takes_the_small_path():
    A = I.config_inputs("stencil2d_64")["A"]
    rp, ci, va, arith, st = run_gpu(A, A)
    assert st["small_path_rows"] == A.m and st["launches_sym"] == 1 and st["launches_num"] == 1
    assert arith == 1
    assert st["flops"] == int(np.asarray(oracle.row_flops(A, A)).sum())
    check_against_oracle(A, A, rp, ci, va, exact=True)


@pytest.mark.parametrize("seed", range(4))
def test_random_small_products_exact(seed):
    # sparse rows (about 1.2 entries), so that every row of C has at most 16
    # columns (10 to 12 here); repeated and unsorted entries in some cases
    u = I.uniform01(seed, "small.dims", 3)
    m, n, k = 50 + int(u[0] * 3000), 40 + int(u[1] * 2000), 30 + int(u[2] * 2000)
    A = I.random_sparse(m, n, 1.2 / n, seed, duplicates=seed == 1, unsorted=seed == 2)
    B = I.random_sparse(n, k, 1.2 / k, seed + 20, duplicates=seed == 3, unsorted=seed == 2)
    rp, ci, va, _, st = run_gpu(A, B)
    assert np.diff(oracle.spgemm(A, B).rowptr).max() <= 16
    assert st["small_path_rows"] == m
    check_against_oracle(A, B, rp, ci, va, exact=True)


def test_row_beyond_the_small_path_takes_the_tiered_path():
    # rows of one entry, except row 0 with ten entries far apart: its row of C
    # (ten tridiagonal rows of B) has 29 columns, beyond the path's 16, while
    # the mean flop bound (about 3) lets the small path try
    m = 500
    rows = np.concatenate([np.zeros(10, dtype=np.int64), np.arange(1, m)])
    cols = np.concatenate([np.arange(0, 200, 20), np.arange(1, m)])
    rp = np.concatenate(([0], np.cumsum(np.bincount(rows, minlength=m))))
    A = I.ensure_csr(m, m, rp, cols, I.uniform01(5, "small.a", len(cols)) * 2 - 1)
    B = I.laplacian_1d(m)
    rp_, ci, va, _, st = run_gpu(A, B, arith=1)
    assert np.diff(oracle.spgemm(A, B).rowptr).max() == 29
    assert st["small_path_rows"] == 0
    check_against_oracle(A, B, rp_, ci, va)


def test_small_path_off_and_forced_tiers():
    A = I.config_inputs("stencil2d_64")["A"]
    for opts in ({"small_max_rows": 0}, {"force_tier": 0}):
        rp, ci, va, _, st = run_gpu(A, A, arith=1, **opts)
        assert st["small_path_rows"] == 0
        check_against_oracle(A, A, rp, ci, va)


def test_small_path_refresh_and_jacobi():
    from paper_2103_11991_gb300 import spgemm as K
    A = I.stencil_2d(50, 50, 5)
    dA = K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dA)
        assert op.stats()["small_path_rows"] == A.m
        ci, va = op.numeric(dA, dA, rp, nnz)
        # new values, same structure: the numeric phase alone
        dA.vals.mul_(0.5)
        op.numeric(dA, dA, rp, nnz, ci, va)
        op.sync()
        A2 = I.ensure_csr(A.m, A.n, A.rowptr, A.colind, A.vals * 0.5)
        check_against_oracle(A2, A2, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy(), exact=True)
        # the Jacobi-fused numeric phase on the same symbolic result
        op.jacobi_numeric(dA, dA, rp, nnz, 2.0 / 3.0, ci, va)
        op.sync()
        ref = J.jacobi_spgemm(A2, A2, 2.0 / 3.0)
        assert_structure_equal(rp.cpu().numpy(), ci.cpu().numpy(), ref.rowptr, ref.colind)
        assert_values_within(va.cpu().numpy(), ref.vals, J.jacobi_abs(A2, A2, 2.0 / 3.0))


def test_small_path_bad_index():
    from paper_2103_11991_gb300 import spgemm as K
    A = I.laplacian_1d(20)
    cols = A.colind.copy()
    cols[7] = 25  # outside the 20 columns of A (= rows of B)
    Abad = I.ensure_csr(20, 20, A.rowptr, cols, A.vals)
    B = I.random_sparse(20, 10, 0.2, 3)
    dA, dB = K.DeviceCSR.from_host(Abad), K.DeviceCSR.from_host(B)
    with K.SpGEMM() as op:
        with pytest.raises(K.KKError) as e:
            op.symbolic(dA, dB)
        assert e.value.status == 8
