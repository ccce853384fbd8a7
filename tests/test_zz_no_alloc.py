"""The allocation-free symbolic entry point (include/kk_noalloc.h), for callers
that cannot call cudaMalloc (graph capture, restricted allocators, real-time
paths): through the C ABI it must give the same row pointers and nnz(C) as the
regular symbolic phase, on two calls in a row (its fixed scratch is shared and
reused between calls).  Collected last so a failure here does not stop the
rest of the GPU suite."""
import numpy as np
import pytest

from paper_2103_11991_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _regular(dA, dB):
    from paper_2103_11991_gb300 import spgemm as K
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dB)
        return rp.cpu().numpy(), nnz


def test_noalloc_symbolic_matches_regular_twice():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    problems = [
        (I.stencil_3d(20, 20, 20, 27, 26.0, -1.0), None),
        (I.random_rows(3000, 2500, 3, 40, seed=21), I.random_rows(2500, 70000, 5, 60, seed=22)),
    ]
    for A, B in problems:
        B = A if B is None else B
        dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
        ref_rp, ref_nnz = _regular(dA, dB)
        rp = torch.full((A.m + 1,), -1, dtype=torch.int64, device="cuda")
        nnz = K.kk_spgemm_symbolic_noalloc(dA, dB, rp)
        torch.cuda.synchronize()
        assert nnz == ref_nnz
        assert np.array_equal(rp.cpu().numpy(), ref_rp)


def test_noalloc_rejects_too_many_rows():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    m = K.NOALLOC_MAX_ROWS + 1
    A = I.identity(m)
    dA = K.DeviceCSR.from_host(A)
    rp = torch.empty(m + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(K.KKError) as e:
        K.kk_spgemm_symbolic_noalloc(dA, dA, rp)
    assert e.value.status == 5
