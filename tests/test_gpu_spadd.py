"""GPU: sparse matrix addition C = alpha A + beta B (paper Sec. "SpAdd") through
the C ABI against the CPU oracle (oracle/spadd.py): structure bit-exact, values
bit-exact when no column repeats within A or B, else within
1e-12 * (sum |alpha a| + sum |beta b|)."""
import numpy as np
import pytest

from oracle import spadd as S
from paper_2103_11991_gb300 import inputs as I
from tests._util import assert_structure_equal, assert_values_within

pytestmark = pytest.mark.gpu


def _run(A, B, alpha, beta, op=None):
    from paper_2103_11991_gb300 import spgemm as K
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    own = op is None
    if own:
        op = K.SpGEMM()
    try:
        rp, nnz = op.spadd_symbolic(dA, dB)
        ci, va = op.spadd_numeric(alpha, dA, beta, dB, rp, nnz)
        op.sync()
        return rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy()
    finally:
        if own:
            op.close()


def _check(A, B, alpha, beta, rp, ci, va, exact=False):
    ref = S.spadd(A, B, alpha, beta)
    assert_structure_equal(rp, ci, ref.rowptr, ref.colind)
    if exact:
        assert np.array_equal(va, ref.vals)
    else:
        assert_values_within(va, ref.vals, S.spadd_abs(A, B, alpha, beta) + 1e-300)


@pytest.mark.parametrize("seed", range(8))
def test_spadd_random(seed):
    u = I.uniform01(seed, "gsa.dims", 2)
    m, n = 50 + int(u[0] * 900), 1 + int(u[1] * 600)
    dens = [0.002, 0.01, 0.05, 0.2][seed % 4]
    dup, uns = seed % 3 == 0, seed % 2 == 1
    A = I.random_sparse(m, n, dens, seed, duplicates=dup, unsorted=uns, empty_rows=0.1)
    B = I.random_sparse(m, n, dens * 1.5, seed + 17, duplicates=seed % 4 == 1,
                        unsorted=seed % 3 == 2)
    al, be = [(1.0, 1.0), (2.0, -0.5), (-1.25, 3.0), (0.0, 1.0)][seed % 4]
    rp, ci, va = _run(A, B, al, be)
    exact = not dup and seed % 4 != 1
    _check(A, B, al, be, rp, ci, va, exact=exact)


@pytest.mark.parametrize("lens", [(120, 130), (300, 2000), (3000, 4000)])
def test_spadd_long_rows(lens):
    # rows of more than 256 combined entries take one CTA per row
    n = 20000
    A = I.random_rows(64, n, lens[0], lens[1], seed=lens[0], purpose="saA")
    B = I.random_rows(64, n, lens[0], lens[1], seed=lens[1], purpose="saB")
    rp, ci, va = _run(A, B, 1.0, -1.0)
    _check(A, B, 1.0, -1.0, rp, ci, va, exact=True)
    # unsorted long rows: the full bitonic sort
    Au = I.permute(A, None, I.permutation(n, 5))
    Bu = I.permute(B, None, I.permutation(n, 5))
    Au.colind = Au.colind.copy()
    rows = np.repeat(np.arange(Au.m), np.diff(Au.rowptr))
    key = I.uniform01(9, "shuffle", Au.nnz)
    o = np.lexsort((key, rows))
    Au = I.ensure_csr(Au.m, Au.n, Au.rowptr, Au.colind[o], Au.vals[o])
    rp, ci, va = _run(Au, Bu, 0.5, 2.0)
    _check(Au, Bu, 0.5, 2.0, rp, ci, va)


def test_spadd_reuse_mismatch_and_errors():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = I.random_sparse(300, 200, 0.05, 3)
    B = I.random_sparse(300, 200, 0.05, 4)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM() as op:
        with pytest.raises(K.KKError) as e:
            op.spadd_numeric(1.0, dA, 1.0, dB, torch.zeros(301, dtype=torch.int64, device="cuda"), 0)
        assert e.value.status == 7  # numeric before symbolic
        rp, nnz = op.spadd_symbolic(dA, dB)
        ci, va = op.spadd_numeric(1.0, dA, 1.0, dB, rp, nnz)
        # new values, other coefficients: numeric only
        dA.vals.mul_(3.0)
        op.spadd_numeric(-0.5, dA, 2.0, dB, rp, nnz, ci, va)
        op.sync()
        A3 = I.CSR(A.m, A.n, A.rowptr, A.colind, A.vals * 3.0)
        _check(A3, B, -0.5, 2.0, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy(), exact=True)
        # other index arrays than the symbolic call's
        dB2 = K.DeviceCSR.from_host(B)
        with pytest.raises(K.KKError) as e:
            op.spadd_numeric(1.0, dA, 1.0, dB2, rp, nnz, ci, va)
        assert e.value.status == 4
    # a row of more than 8192 combined entries
    big = I.random_rows(2, 50000, 4500, 4600, seed=1, purpose="big")
    with pytest.raises(K.KKError) as e:
        _run(big, big, 1.0, 1.0)
    assert e.value.status == 5
    # a column outside [0, n)
    dA = K.DeviceCSR.from_host(A)
    dA.colind[5] = A.n + 3
    with K.SpGEMM() as op:
        with pytest.raises(K.KKError) as e:
            op.spadd_symbolic(dA, K.DeviceCSR.from_host(B))
        assert e.value.status == 8
    # shapes differ
    with K.SpGEMM() as op:
        with pytest.raises(K.KKError) as e:
            op.spadd_symbolic(K.DeviceCSR.from_host(A),
                              K.DeviceCSR.from_host(I.random_sparse(300, 150, 0.05, 4)))
        assert e.value.status == 1


def test_spadd_edge_and_interleaved_spgemm():
    from paper_2103_11991_gb300 import spgemm as K
    from tests._gpu import check_against_oracle
    # empty matrices and empty rows
    for m, n in ((0, 5), (7, 0), (6, 9)):
        A = I.random_sparse(m, n, 0.0, 1)
        B = I.random_sparse(m, n, 0.3, 2)
        rp, ci, va = _run(A, B, 1.0, 1.0)
        _check(A, B, 1.0, 1.0, rp, ci[:int(rp[-1])], va[:int(rp[-1])], exact=True)
    # SpAdd between the SpGEMM phases of the same handle leaves the SpGEMM state
    # (kept window structure, fingerprints) intact
    A = I.stencil_3d(12, 12, 12, 27, 26.0, -1.0)
    dA = K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dA)
        rs, ci_s, va_s = _run(A, A, 1.0, 1.0, op=op)
        _check(A, A, 1.0, 1.0, rs, ci_s, va_s, exact=True)
        ci, va = op.numeric(dA, dA, rp, nnz)
        op.sync()
        check_against_oracle(A, A, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy())
