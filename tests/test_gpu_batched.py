"""Batched form on the GPU: every product of a batch against the oracle
(structure exact, values within bound), with and without CUDA-graph replay."""
import numpy as np
import pytest

import oracle
from paper_2103_11991_gb300 import inputs as I
from tests._util import assert_structure_equal, assert_values_within

pytestmark = pytest.mark.gpu


def _check_batch(pairs, rowptr, off, colind, vals):
    rp = rowptr.cpu().numpy()
    ci = colind.cpu().numpy()
    va = vals.cpu().numpy()
    r0 = 0
    for k, (A, B) in enumerate(pairs):
        ref = oracle.spgemm(A, B)
        ab = oracle.spgemm_abs(A, B)
        local = rp[r0:r0 + A.m + 1]
        assert local[0] == off[k]
        assert_structure_equal(local - local[0], ci[local[0]:local[-1]], ref.rowptr, ref.colind)
        assert_values_within(va[local[0]:local[-1]], ref.vals, ab.vals)
        r0 += A.m


def _pairs(count, seed0, rows_hi=3000):
    pairs = I.batch_pairs(count, seed0=seed0, rows_lo=20, rows_hi=rows_hi)
    # edge cases: an empty A, a one-row product, an empty B row set
    pairs.append((I.random_sparse(0, 5, 0.5, 1), I.random_sparse(5, 7, 0.5, 2)))
    pairs.append((I.random_sparse(1, 4, 1.0, 3), I.random_sparse(4, 6, 0.5, 4)))
    pairs.append((I.random_sparse(9, 6, 0.3, 5), I.random_sparse(6, 8, 0.0, 6)))
    return pairs


@pytest.mark.parametrize("mode", [1, 2])  # persistent work queue / packed block-diagonal
@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("arith", [1, 2])
def test_batched_matches_oracle(graph, arith, mode):
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    pairs = _pairs(40, 7000)
    dA = [K.DeviceCSR.from_host(A) for A, _ in pairs]
    dB = [K.DeviceCSR.from_host(B) for _, B in pairs]
    stream = torch.cuda.Stream() if graph else None
    ctx = torch.cuda.stream(stream) if stream is not None else torch.cuda.stream(torch.cuda.current_stream())
    with ctx:
        with K.BatchedSpGEMM(stream=stream, batched_graph=graph, arith=arith, batched_mode=mode) as op:
            for rep in range(2):  # second round replays the captured graphs
                rowptr, off, total = op.symbolic(dA, dB)
                colind, vals = op.numeric(dA, dB, rowptr, total)
                op.sync()
                torch.cuda.synchronize()
                assert off[-1] == total
                _check_batch(pairs, rowptr, off, colind[:total], vals[:total])
            # new values, same patterns: numeric only
            for d in dA:
                d.vals.mul_(-2.0)
            colind2, vals2 = op.numeric(dA, dB, rowptr, total, colind, vals)
            op.sync()
            torch.cuda.synchronize()
            scaled = [(I.CSR(A.m, A.n, A.rowptr, A.colind, A.vals * -2.0), B) for A, B in pairs]
            _check_batch(scaled, rowptr, off, colind2[:total], vals2[:total])


def test_batched_empty_batch():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    with K.BatchedSpGEMM() as op:
        rowptr = torch.zeros(1, dtype=torch.int64, device="cuda")
        off, total = K.kk_spgemm_batched_symbolic(op.h, [], [], rowptr)
        assert total == 0 and list(off) == [0]


def test_batched_packed_moved_arrays():
    # numeric with the same patterns in other arrays: the packed batch is rebuilt
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    pairs = _pairs(12, 7100)
    dA = [K.DeviceCSR.from_host(A) for A, _ in pairs]
    dB = [K.DeviceCSR.from_host(B) for _, B in pairs]
    with K.BatchedSpGEMM(batched_mode=2) as op:
        rowptr, off, total = op.symbolic(dA, dB)
        dA2 = [K.DeviceCSR(d.m, d.n, d.rowptr.clone(), d.colind.clone(), d.vals.clone()) for d in dA]
        colind, vals = op.numeric(dA2, dB, rowptr, total)
        op.sync()
        torch.cuda.synchronize()
        _check_batch(pairs, rowptr, off, colind[:total], vals[:total])


@pytest.mark.parametrize("pred", ["none", "class2"])
def test_batched_learned_matches_oracle(pred):
    # the block-diagonal batch through the learned form: one speculative pass
    # (rows sized by the flop bound, or all predicted class 2 so that most rows
    # overflow and are re-run), then a numeric refresh with new values; the
    # structure cache off, so that window rows take the window one-pass too
    from paper_2103_11991_gb300 import spgemm as K
    pairs = _pairs(30, 7300)
    dA = [K.DeviceCSR.from_host(A) for A, _ in pairs]
    dB = [K.DeviceCSR.from_host(B) for _, B in pairs]
    with K.BatchedSpGEMM(batched_mode=2, batched_learned=1, structure_cache=0) as op:
        if pred == "class2":
            th = np.zeros(1872, dtype=np.float32)
            th[1872 - 16 + 2] = 10.0
            op.set_predictor(th, 0.95)
        rowptr, off, total = op.symbolic(dA, dB)
        st = op.stats()
        assert st["onepass_rows"] > 0
        if pred == "class2":
            assert st["overflow_rows"] > 0
        colind, vals = op.numeric(dA, dB, rowptr, total)
        op.sync()
        _check_batch(pairs, rowptr, off, colind[:total], vals[:total])
        for d in dA:
            d.vals.mul_(-2.0)
        colind2, vals2 = op.numeric(dA, dB, rowptr, total, colind, vals)
        op.sync()
        scaled = [(I.CSR(A.m, A.n, A.rowptr, A.colind, A.vals * -2.0), B) for A, B in pairs]
        _check_batch(scaled, rowptr, off, colind2[:total], vals2[:total])


@pytest.mark.parametrize("graph", [0, 1])
def test_persistent_batch_with_heavy_rows(graph):
    """A batch whose rows exceed the persistent kernels' accumulators (rows of
    about 26,000 products over 60,000 columns beside ordinary pairs): the persistent
    mode hands the batch to the block-diagonal form inside the same call; every
    product still matches the oracle, on repeated calls and a numeric refresh."""
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    pairs = _pairs(10, 7100)
    heavy_a = I.random_rows(30, 400, 180, 220, seed=91)
    heavy_b = I.random_rows(400, 60000, 120, 140, seed=92)
    pairs.insert(3, (heavy_a, heavy_b))
    dA = [K.DeviceCSR.from_host(A) for A, _ in pairs]
    dB = [K.DeviceCSR.from_host(B) for _, B in pairs]
    stream = torch.cuda.Stream() if graph else None
    ctx = torch.cuda.stream(stream) if stream is not None else torch.cuda.stream(torch.cuda.current_stream())
    with ctx:
        with K.BatchedSpGEMM(stream=stream, batched_graph=graph, batched_mode=1) as op:
            for _ in range(2):
                rowptr, off, total = op.symbolic(dA, dB)
                colind, vals = op.numeric(dA, dB, rowptr, total)
                op.sync()
                torch.cuda.synchronize()
                _check_batch(pairs, rowptr, off, colind[:total], vals[:total])
            for d in dA:
                d.vals.mul_(0.5)
            op.numeric(dA, dB, rowptr, total, colind, vals)
            op.sync()
            torch.cuda.synchronize()
    for A, _ in pairs:
        A.vals = A.vals * 0.5
    _check_batch(pairs, rowptr, off, colind[:total], vals[:total])
