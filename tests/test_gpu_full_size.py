"""GPU parity at the full sizes of the five workloads, in the launch
configuration ``bench.py`` times (default options, one handle), against what
the oracle can compute in seconds: blocks of rows computed by the oracle, and
properties that hold at any size (closed forms of the stencil products, exact
Galerkin operator, row-count bounds, batch offsets)."""
import numpy as np
import pytest

import oracle
from paper_2103_11991_gb300 import inputs as I
from tests._util import assert_structure_equal, assert_values_within

pytestmark = pytest.mark.gpu


def _check_blocks(A, B, rp_dev, ci_dev, va_dev, blocks):
    """Rows [r0, r1) of C on the GPU against the oracle's rows [r0, r1)."""
    import torch
    for r0, r1 in blocks:
        rp = rp_dev[r0:r1 + 1].cpu().numpy()
        lo, hi = int(rp[0]), int(rp[-1])
        ci = ci_dev[lo:hi].cpu().numpy()
        va = va_dev[lo:hi].cpu().numpy()
        ref = oracle.spgemm(A, B, r0, r1)
        ab = oracle.spgemm_abs(A, B, r0, r1)
        assert_structure_equal(rp - lo, ci, ref.rowptr, ref.colind)
        assert_values_within(va, ref.vals, ab.vals)
        del ci, va
        torch.cuda.empty_cache()


def test_stencil3d27_100_full():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    d = I.config_inputs("stencil3d27_100")
    A = d["A"]
    dA = K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dA)
        ci, va = op.numeric(dA, dA, rp, nnz)
        op.sync()
        assert nnz == 494 ** 3
        # every row's count from the closed form: per dimension the 5 offsets
        # -2..2 clipped at the boundary
        n = 100
        node = np.arange(n ** 3)
        cnt = np.ones(n ** 3, dtype=np.int64)
        for c in (node % n, (node // n) % n, node // (n * n)):
            cnt *= np.minimum(c + 2, n - 1) - np.maximum(c - 2, 0) + 1
        assert np.array_equal(np.diff(rp.cpu().numpy()), cnt)
        _check_blocks(A, A, rp, ci, va, [(0, 1500), (494_000, 496_000), (n ** 3 - 1500, n ** 3)])


def test_amg_galerkin_128_full_exact():
    # R (A P) = 4 x (7-point Laplacian on 64^3 with 6 / -1), exactly
    from paper_2103_11991_gb300 import spgemm as K
    d = I.config_inputs("amg_galerkin_128")
    A, P, R = d["A"], d["P"], d["R"]
    dA, dP, dR = (K.DeviceCSR.from_host(X) for X in (A, P, R))
    import torch
    with K.SpGEMM() as op1, K.SpGEMM() as op2:
        rp1, n1 = op1.symbolic(dA, dP)
        c1, v1 = op1.numeric(dA, dP, rp1, n1)
        dAP = K.DeviceCSR(A.m, P.n, rp1.to(torch.int32), c1, v1)
        rp2, n2 = op2.symbolic(dR, dAP)
        c2, v2 = op2.numeric(dR, dAP, rp2, n2)
        op2.sync()
        assert n1 == 8_290_304 and n2 == 1_810_432
        L = I.stencil_3d(64, 64, 64, 7, 24.0, -4.0)
        assert_structure_equal(rp2.cpu().numpy(), c2.cpu().numpy(), L.rowptr, L.colind)
        assert np.array_equal(v2.cpu().numpy(), L.vals)
        # numeric refreshes on the kept structure, A's values rescaled by s:
        # R (sA P) = 4 s x the Laplacian, each entry within 1e-12 of its size
        base = dA.vals.clone()
        for s in I.uniform01(41, "galerkin.refresh", 3) * 1.5 + 0.5:
            dA.vals = base * float(s)
            op1.numeric(dA, dP, rp1, n1, c1, v1)
            op2.numeric(dR, dAP, rp2, n2, c2, v2)
            op2.sync()
            want = L.vals * float(s)
            assert np.all(np.abs(v2.cpu().numpy() - want) <= 1e-12 * np.abs(want))


def test_rmat20_full_sampled():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = I.config_inputs("rmat20")["A"]
    dA = K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dA)
        ci, va = op.numeric(dA, dA, rp, nnz)
        op.sync()
        cnt = np.diff(rp.cpu().numpy())
        flop = oracle.row_flops(A, A)
        assert cnt.sum() == nnz
        assert np.all(cnt <= np.minimum(flop, A.n))
        assert cnt.max() > 100_000  # the heavy rows are in the product
        # the heaviest rows (R-MAT's low ids), a middle block and the last rows
        _check_blocks(A, A, rp, ci, va, [(0, 48), (400_000, 402_000), (A.m - 2000, A.m)])
        del ci, va
    torch.cuda.empty_cache()


def test_rmat20_learned_full_sampled():
    """The learned form on its own workload (R-MAT scale 20) at full size, in
    the configuration the bench times (predictor trained on the training
    families, quantile 0.95): row pointers identical to the plain symbolic
    phase's, the same count bounds, and the heaviest rows, a middle block and
    the last rows against the oracle."""
    import torch
    from paper_2103_11991_gb300 import learned as L
    from paper_2103_11991_gb300 import spgemm as K
    X, y = L.make_training_set(L.training_pairs(small=True))
    params, _ = L.train_predictor(X, y, epochs=30)
    del X, y
    A = I.config_inputs("rmat20")["A"]
    dA = K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp_plain, nnz_plain = op.symbolic(dA, dA)
        rp_plain = rp_plain.cpu().numpy()
    with K.SpGEMM() as op:
        op.set_predictor(params, 0.95)
        rp, nnz = op.learned_symbolic(dA, dA)
        ci, va = op.learned_numeric(dA, dA, rp, nnz)
        op.sync()
        st = op.stats()
        assert nnz == nnz_plain
        assert np.array_equal(rp.cpu().numpy(), rp_plain)
        assert st["onepass_rows"] > 0
        cnt = np.diff(rp_plain)
        assert np.all(cnt <= np.minimum(oracle.row_flops(A, A), A.n))
        _check_blocks(A, A, rp, ci, va, [(0, 48), (400_000, 402_000), (A.m - 2000, A.m)])
        del ci, va
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def batch2000():
    return I.config_inputs("batch2000")["pairs"]


@pytest.mark.parametrize("mode", [2, 1])  # packed block-diagonal / persistent queue + graph
def test_batch2000_full_sampled(batch2000, mode):
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    pairs = batch2000
    dA = [K.DeviceCSR.from_host(A) for A, _ in pairs]
    dB = [K.DeviceCSR.from_host(B) for _, B in pairs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), K.BatchedSpGEMM(stream=stream, batched_mode=mode) as op:
        for _ in range(2):  # the second pass replays what the first captured
            rowptr, off, total = op.symbolic(dA, dB)
            colind, vals = op.numeric(dA, dB, rowptr, total)
            op.sync()
        assert off[0] == 0 and off[-1] == total and np.all(np.diff(off) >= 0)
        rows = np.concatenate(([0], np.cumsum([A.m for A, _ in pairs])))
        pick = [0, 1, 999, 1998, 1999] + list(I.permutation(2000, 77)[:10])
        for k in pick:
            A, B = pairs[k]
            r0 = int(rows[k])
            rp = rowptr[r0:r0 + A.m + 1].cpu().numpy()
            assert rp[0] == off[k] and rp[-1] == off[k + 1]
            ci = colind[rp[0]:rp[-1]].cpu().numpy()
            va = vals[rp[0]:rp[-1]].cpu().numpy()
            ref = oracle.spgemm(A, B)
            assert_structure_equal(rp - rp[0], ci, ref.rowptr, ref.colind)
            assert_values_within(va, ref.vals, oracle.spgemm_abs(A, B).vals)
        del colind, vals
    torch.cuda.empty_cache()
