"""The allocation-free symbolic entry point (include/kk_noalloc.h).

It serves callers that cannot call cudaMalloc: applications that own all
device memory through their own pool and forbid allocations behind their back,
plug-ins running inside such a framework, and latency-critical loops where the
synchronisation an allocation may bring is not allowed.  Through the C ABI its
row pointers and nnz(C) must equal the CPU oracle's, on two calls in a row (its
fixed scratch is shared and keeps the previous call's contents), and a call
must not change the device's free memory.  Bad indices are reported, not read.
Collected last so a failure here does not stop the rest of the GPU suite."""
import numpy as np
import pytest

import oracle
from paper_2103_11991_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KK_ERR_CAPACITY = 5
KK_ERR_BAD_INDEX = 8


def _oracle_rowptr(A, B):
    cnt = oracle.symbolic(A, B)
    return np.concatenate([[0], np.cumsum(cnt, dtype=np.int64)])


def _device(m, n, rowptr, colind):
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    rp = torch.tensor(np.asarray(rowptr, dtype=np.int32), device="cuda")
    ci = torch.tensor(np.asarray(colind, dtype=np.int32), device="cuda")
    va = torch.ones(len(colind), dtype=torch.float64, device="cuda")
    return K.DeviceCSR(m, n, rp, ci, va)


def _problems():
    k = 1 << 24
    wide = I.CSR(2, 3, np.array([0, 2, 3]), np.array([0, 2, 1]), np.ones(3))
    wide_b = I.CSR(3, k, np.array([0, 2, 2, 3]), np.array([0, k - 1, 40000]), np.ones(3))
    return [
        (I.stencil_3d(20, 20, 20, 27, 26.0, -1.0), None),
        (I.random_rows(3000, 2500, 3, 40, seed=21), I.random_rows(2500, 70000, 5, 60, seed=22)),
        # columns 0, 40000 and 2^24 - 1 in one row: three non-empty windows of a
        # span of 512 windows
        (wide, wide_b),
    ]


def test_noalloc_symbolic_matches_oracle_twice():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    for A, B in _problems():
        B = A if B is None else B
        ref = _oracle_rowptr(A, B)
        dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
        for _ in range(2):
            rp = torch.full((A.m + 1,), -1, dtype=torch.int64, device="cuda")
            nnz = K.kk_spgemm_symbolic_noalloc(dA, dB, rp)
            torch.cuda.synchronize()
            assert nnz == int(ref[-1])
            assert np.array_equal(rp.cpu().numpy(), ref)


def test_noalloc_allocates_no_device_memory():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = I.random_rows(5000, 4000, 3, 40, seed=23)
    B = I.random_rows(4000, 9000, 3, 40, seed=24)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    rp = torch.empty(A.m + 1, dtype=torch.int64, device="cuda")
    K.kk_spgemm_symbolic_noalloc(dA, dB, rp)  # first call on the device: address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    nnz = K.kk_spgemm_symbolic_noalloc(dA, dB, rp)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == used0
    assert nnz == int(_oracle_rowptr(A, B)[-1])


def test_noalloc_empty_a():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = I.CSR(0, 5, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int64), np.zeros(0))
    B = I.random_rows(5, 7, 1, 3, seed=25)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    rp = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    assert K.kk_spgemm_symbolic_noalloc(dA, dB, rp) == 0
    assert rp.cpu().tolist() == [0]


def test_noalloc_reports_bad_indices():
    """Every bad index below stays inside the arrays' allocations; the kernel
    checks each row before it reads through its indices."""
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    good_b = ([0, 2, 3, 5], [0, 3, 1, 2, 4])       # 3 x 5
    cases = [
        # A column outside B's rows
        ((2, 3, [0, 2, 3], [0, 3, 1]), (3, 5) + good_b),
        # B row 1 with decreasing bounds (3 -> 2), all inside B's 5 entries
        ((2, 3, [0, 2, 3], [0, 1, 2]), (3, 5, [0, 3, 2, 5], [0, 3, 1, 2, 4])),
        # B column outside [0, B.n)
        ((2, 3, [0, 2, 3], [0, 1, 2]), (3, 5, [0, 2, 3, 5], [0, 3, 7, 2, 4])),
        # A.rowptr[0] != 0
        ((2, 3, [1, 2, 3], [0, 1, 2]), (3, 5) + good_b),
    ]
    for (am, an, arp, aci), (bm, bn, brp, bci) in cases:
        dA = _device(am, an, arp, aci)
        dB = _device(bm, bn, brp, bci)
        rp = torch.empty(am + 1, dtype=torch.int64, device="cuda")
        with pytest.raises(K.KKError) as e:
            K.kk_spgemm_symbolic_noalloc(dA, dB, rp)
        assert e.value.status == KK_ERR_BAD_INDEX
    # the shared scratch holds no stale error: a good call afterwards succeeds
    A = I.random_rows(50, 40, 1, 6, seed=26)
    B = I.random_rows(40, 60, 1, 6, seed=27)
    rp = torch.empty(A.m + 1, dtype=torch.int64, device="cuda")
    nnz = K.kk_spgemm_symbolic_noalloc(K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B), rp)
    assert np.array_equal(rp.cpu().numpy(), _oracle_rowptr(A, B))
    assert nnz == int(_oracle_rowptr(A, B)[-1])


def test_noalloc_rejects_too_many_rows():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    m = K.NOALLOC_MAX_ROWS + 1
    A = I.identity(m)
    dA = K.DeviceCSR.from_host(A)
    rp = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(K.KKError) as e:
        K.kk_spgemm_symbolic_noalloc(dA, dA, rp)
    assert e.value.status == KK_ERR_CAPACITY
