"""GPU: Jacobi-fused numeric phase C = (I - omega D^-1 A) B (paper Sec.
"Jacobi-Fused SpGEMM Kernel") through the C ABI against the CPU oracle
(oracle/jacobi.py): structure bit-exact, values within
1e-12 * (|s_i| sum |a_ij||b_jc| + |b_ic|)."""
import numpy as np
import pytest

from oracle import jacobi as J
from paper_2103_11991_gb300 import inputs as I
from tests._util import assert_structure_equal, assert_values_within

pytestmark = pytest.mark.gpu


def _run(A, B, omega, **opts):
    from paper_2103_11991_gb300 import spgemm as K
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM(**opts) as op:
        rp, nnz = op.symbolic(dA, dB)
        ci, va = op.jacobi_numeric(dA, dB, rp, nnz, omega)
        op.sync()
        st = op.stats()
        return rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy(), st


def _check(A, B, omega, rp, ci, va):
    ref = J.jacobi_spgemm(A, B, omega)
    assert_structure_equal(rp, ci, ref.rowptr, ref.colind)
    assert_values_within(va, ref.vals, J.jacobi_abs(A, B, omega))
    return ref


def _square(m, dens, seed, **kw):
    return I.with_diagonal(I.random_sparse(m, m, dens, seed, **kw), seed + 900,
                           split=kw.get("duplicates", False))


@pytest.mark.parametrize("arith", [1, 2])
@pytest.mark.parametrize("tier", [-1, 0, 1, 2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_jacobi_random(seed, tier, arith):
    u = I.uniform01(seed, "gj.dims", 2)
    m, k = 20 + int(u[0] * 180), 1 + int(u[1] * 250)
    A = _square(m, [0.02, 0.08, 0.2, 0.4][seed], seed, duplicates=seed % 2 == 0,
                unsorted=seed % 3 == 1)
    B = I.random_sparse(m, k, 0.1, seed + 40, duplicates=seed == 1, unsorted=seed == 2)
    omega = [2.0 / 3.0, 0.5, 1.25, -0.3][seed]
    rp, ci, va, _ = _run(A, B, omega, arith=arith, force_tier=tier)
    _check(A, B, omega, rp, ci, va)


@pytest.mark.parametrize("arith", [1, 2])
def test_jacobi_stencil_window_tier(arith):
    A = I.stencil_3d(20, 20, 20, 27, 26.0, -1.0)
    rp, ci, va, st = _run(A, A, 2.0 / 3.0, arith=arith)
    assert st["num_window_rows"] > 0 and st["kept_structure_rows"] > 0
    _check(A, A, 2.0 / 3.0, rp, ci, va)


def test_prolongator_smoothing_amg():
    # smoothed aggregation: (I - w D^-1 A) P on the 7-point Laplacian; interior
    # rows of the smoothed prolongator sum to 1 (A's interior rows sum to 0)
    g = 32
    A = I.stencil_3d(g, g, g, 7, 6.0, -1.0)
    P = I.aggregation_prolongator(g, g, g, 2)
    rp, ci, va, _ = _run(A, P, 2.0 / 3.0)
    _check(A, P, 2.0 / 3.0, rp, ci, va)
    sums = np.add.reduceat(va, rp[:-1].astype(np.int64))
    r = np.arange(g ** 3)
    x, y, z = r % g, (r // g) % g, r // (g * g)
    inner = (x > 0) & (x < g - 1) & (y > 0) & (y < g - 1) & (z > 0) & (z < g - 1)
    assert np.allclose(sums[inner], 1.0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("which", ["large_value", "rmat"])
def test_jacobi_wide_and_large_rows(which):
    if which == "large_value":
        # rows of 257..512 columns over a 30,000-wide matrix: large-value window bins
        A = I.with_diagonal(I.random_rows(30000, 30000, 14, 22, seed=41, purpose="jA"), 43)
        B = I.random_rows(30000, 30000, 14, 22, seed=42, purpose="jB")
    else:
        A = I.with_diagonal(I.rmat(12, 16, 0.57, 0.19, 0.19, seed=77), 78)
        B = A
    rp, ci, va, st = _run(A, B, 0.8)
    _check(A, B, 0.8, rp, ci, va)


def test_jacobi_reuse_and_plain_numeric_on_same_handle():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    from tests._gpu import check_against_oracle
    A = _square(300, 0.05, 5)
    B = I.random_sparse(300, 200, 0.05, 6)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dB)
        ci, va = op.jacobi_numeric(dA, dB, rp, nnz, 0.5)
        op.sync()
        _check(A, B, 0.5, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy())
        # new values of A, another omega: same structure
        dA.vals.mul_(1.5)
        A2 = I.CSR(A.m, A.n, A.rowptr, A.colind, A.vals * 1.5)
        op.jacobi_numeric(dA, dB, rp, nnz, 0.9, ci, va)
        op.sync()
        _check(A2, B, 0.9, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy())
        # the plain numeric phase on the same handle still gives A*B
        op.numeric(dA, dB, rp, nnz, ci, va)
        op.sync()
        check_against_oracle(A2, B, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy())


def test_jacobi_errors():
    from paper_2103_11991_gb300 import spgemm as K
    # non-square A: rejected on the host
    A = I.random_sparse(5, 7, 0.5, 1)
    B = I.random_sparse(7, 4, 0.5, 2)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dB)
        with pytest.raises(K.KKError) as e:
            op.jacobi_numeric(dA, dB, rp, nnz, 0.5)
        assert e.value.status == 1
    # a row without a stored diagonal: reported by the device at sync
    A = I.laplacian_1d(6)
    keep = np.ones(A.nnz, dtype=bool)
    keep[int(A.rowptr[3]) + 1] = False  # the (3,3) entry
    rows = np.repeat(np.arange(6), np.diff(A.rowptr))[keep]
    A2 = I.ensure_csr(6, 6, np.concatenate(([0], np.cumsum(np.bincount(rows, minlength=6)))),
                      A.colind[keep], A.vals[keep])
    Bi = I.identity(6)
    dA, dB = K.DeviceCSR.from_host(A2), K.DeviceCSR.from_host(Bi)
    # automatic tiers (the thread tier finds the row's diagonal itself) and each
    # forced tier (the row-scale kernel finds it)
    for tier in (-1, 0, 1, 2, 3):
        with K.SpGEMM(force_tier=tier) as op:
            rp, nnz = op.symbolic(dA, dB)
            with pytest.raises(K.KKError) as e:
                op.jacobi_numeric(dA, dB, rp, nnz, 0.5)
                op.sync()
            assert e.value.status == 1, tier
    # a diagonal that sums to zero (two stored entries cancel)
    rows = np.repeat(np.arange(6), np.diff(A.rowptr))
    cols = A.colind.copy()
    vals = A.vals.copy()
    d3 = int(np.nonzero((rows == 3) & (cols == 3))[0][0])
    rows = np.concatenate([rows, [3]])
    cols = np.concatenate([cols, [3]])
    vals = np.concatenate([vals, [-vals[d3]]])
    order = np.argsort(rows, kind="stable")
    A3 = I.ensure_csr(6, 6, np.concatenate(([0], np.cumsum(np.bincount(rows, minlength=6)))),
                      cols[order], vals[order])
    dA = K.DeviceCSR.from_host(A3)
    for tier in (-1, 0):
        with K.SpGEMM(force_tier=tier) as op:
            rp, nnz = op.symbolic(dA, dB)
            with pytest.raises(K.KKError) as e:
                op.jacobi_numeric(dA, dB, rp, nnz, 0.5)
                op.sync()
            assert e.value.status == 1, tier
