"""GPU: compressed B (the paper's B_C) in the window tier, and the structure the
symbolic phase keeps for the numeric phase of the same A and B arrays.

The kept structure must give bit-identical C to the rebuild from B_C; it must
not be used for other index arrays; and a structure that changed behind the
same arrays is reported (KK_ERR_STRUCTURE_MISMATCH) instead of silently used."""
import numpy as np
import pytest

from paper_2103_11991_gb300 import inputs as I
from tests._gpu import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu


def _stencil_random(scale, seed):
    d = I.config_inputs("stencil3d27_100", scale=scale)
    A = d["A"].copy()
    A.vals = I.uniform01(seed, "ws", A.nnz) * 2 - 1
    return A


@pytest.mark.parametrize("arith", [1, 2])
def test_kept_structure_matches_rebuild(arith):
    A = _stencil_random(18, 1)
    S = I.stencil_2d(70, 50, 9, 8.0, -1.0)
    S.vals = I.uniform01(2, "ws2", S.nnz) * 2 - 1
    # uniform random rows: windows too full to keep (more than 64 words)
    B2 = I.random_rows(3000, 3000, 20, 40, seed=4)
    A2 = I.random_rows(700, 3000, 5, 30, seed=5)
    for X, Y, keeps in ((A, A, True), (S, S, True), (A2, B2, False)):
        kept = run_gpu(X, Y, arith=arith, force_tier=3, structure_cache=1)
        rebuilt = run_gpu(X, Y, arith=arith, force_tier=3, structure_cache=0)
        assert np.array_equal(kept[0], rebuilt[0]) and np.array_equal(kept[1], rebuilt[1])
        if keeps:  # every row in the window tier: same arithmetic in the same order
            assert np.array_equal(kept[2], rebuilt[2])
        check_against_oracle(X, Y, *kept[:3])
        check_against_oracle(X, Y, *rebuilt[:3])
        assert kept[4]["sym_window_rows"] > 0
        assert (kept[4]["kept_structure_rows"] > 0) == keeps
        assert rebuilt[4]["kept_structure_rows"] == 0
        assert 0 < kept[4]["compressed_b_pairs"] <= Y.nnz


def _distinct_words(B):
    # rows of at most 32 entries: one pair per distinct (row, column >> 5)
    assert np.diff(B.rowptr).max() <= 32
    w = B.colind.astype(np.int64) >> 5
    row = np.repeat(np.arange(B.m), np.diff(B.rowptr))
    first = np.ones(B.nnz, bool)
    first[1:] = (w[1:] != w[:-1]) | (row[1:] != row[:-1])
    return int(first.sum())


@pytest.mark.parametrize("scale", [20, 33])
def test_compressed_b_pairs_of_stencil(scale):
    A = I.config_inputs("stencil3d27_100", scale=scale)["A"]
    _, _, _, _, st = run_gpu(A, A)
    assert st["sym_window_rows"] == A.m
    assert st["compressed_b_pairs"] == _distinct_words(A)


def test_kept_structure_only_for_its_arrays():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = _stencil_random(12, 2)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dB)
        assert op.stats()["kept_structure_rows"] == A.m
        c1, v1 = op.numeric(dA, dB, rp, nnz)
        # same structure and values in other arrays: the structure is rebuilt
        dA2 = K.DeviceCSR(A.m, A.n, dA.rowptr.clone(), dA.colind.clone(), dA.vals.clone())
        c2, v2 = op.numeric(dA2, dB, rp, nnz)
        op.sync()
        assert torch.equal(c1, c2) and torch.equal(v1, v2)
        check_against_oracle(A, A, rp.cpu().numpy(), c1.cpu().numpy(), v1.cpu().numpy())


def test_kept_structure_with_new_values_in_place():
    # symbolic reuse: new values written into the same arrays keep the
    # fingerprint, so the kept structure is used and C follows the new values
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = _stencil_random(12, 31)
    dA = K.DeviceCSR.from_host(A)
    with K.SpGEMM() as op:
        rp, nnz = op.symbolic(dA, dA)
        assert op.stats()["kept_structure_rows"] > 0
        ci, va = op.numeric(dA, dA, rp, nnz)
        for seed in (32, 33):
            vals = I.uniform01(seed, "ws", A.nnz) * 2 - 1
            dA.vals.copy_(torch.from_numpy(vals).cuda())
            op.numeric(dA, dA, rp, nnz, ci, va)
            op.sync()
            A2 = I.CSR(A.m, A.n, A.rowptr, A.colind, vals)
            check_against_oracle(A2, A2, rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy())


@pytest.mark.parametrize("cache,debug", [(0, 0), (1, 0), (1, 1)])
def test_changed_structure_behind_same_arrays_is_reported(cache, debug):
    # cache 0: the rebuilt structure misses products of the new B; cache 1: the
    # index arrays' fingerprint differs from the symbolic call's (debug 0) or a
    # product falls outside the kept structure (debug 1, checked one by one)
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    A = I.config_inputs("stencil3d27_100", scale=10)["A"]
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(A)
    with K.SpGEMM(structure_cache=cache, debug_checks=debug) as op:
        rp, nnz = op.symbolic(dA, dB)
        st = op.stats()
        assert st["sym_window_rows"] == A.m and st["num_window_rows"] == A.m
        # B's rows swapped in pairs (same nnz, rows still sorted and in range),
        # written into the arrays the symbolic phase saw
        perm = np.arange(A.m)
        perm[0:A.m - 1:2] += 1
        perm[1:A.m:2] -= 1
        Bp = I.permute(A, perm, None)
        assert Bp.nnz == A.nnz
        # every read of the (stale) compressed rows stays inside its array
        assert np.all(Bp.rowptr[:-1].astype(np.int64) + np.diff(A.rowptr) <= A.nnz)
        dB.rowptr.copy_(torch.from_numpy(Bp.rowptr).cuda())
        dB.colind.copy_(torch.from_numpy(Bp.colind).cuda())
        dB.vals.copy_(torch.from_numpy(Bp.vals).cuda())
        with pytest.raises(K.KKError) as e:
            op.numeric(dA, dB, rp, nnz)
            op.sync()
        assert e.value.status == 4


def test_wide_kept_bits_match_rebuild():
    # rows with more columns than the wide kernel holds as values in shared
    # memory keep their bit vector from the symbolic phase; the result must be
    # the one of a rebuild (structure bit-exact, values within the bound)
    A = I.random_rows(60, 400, 250, 350, seed=31)
    B = I.random_rows(400, 200000, 100, 140, seed=32)
    kept = run_gpu(A, B, force_tier=2, structure_cache=1)
    rebuilt = run_gpu(A, B, force_tier=2, structure_cache=0)
    assert np.array_equal(kept[0], rebuilt[0]) and np.array_equal(kept[1], rebuilt[1])
    check_against_oracle(A, B, *kept[:3])
    check_against_oracle(A, B, *rebuilt[:3])
    assert kept[4]["num_dense_rows"] > 0
    assert np.diff(kept[0]).min() > 24000  # above the wide kernel's shared-memory value space


@pytest.mark.parametrize("n", [20000, 36000, 60000])
@pytest.mark.parametrize("lens", [(14, 22), (24, 34)])
@pytest.mark.parametrize("arith", [1, 2])
def test_large_value_window_bins(n, lens, arith):
    # rows of 257..1024 columns spread over the whole width of a matrix whose
    # width picks the 24576 / 40960 / 65536-bit window: random rows times random
    # rows give about lens^2 distinct columns per row of C, which lands in the
    # 512-slot (first lens) or 1024-slot (second lens) value array
    A = I.random_rows(600, n, lens[0], lens[1], seed=n + lens[0], purpose="lvA")
    B = I.random_rows(n, n, lens[0], lens[1], seed=n + lens[1], purpose="lvB")
    rp, ci, va, _, st = run_gpu(A, B, arith=arith)
    per_row = np.diff(rp)
    assert per_row.max() > 256 and st["num_window_rows"] > 0
    if lens[0] >= 24:
        assert (per_row > 512).any()
    check_against_oracle(A, B, rp, ci, va)


def test_automatic_arithmetic_runs_the_kept_pass_in_float64():
    """With options.arith = AUTO the kept-structure value pass runs in float64
    (on this part faster than DF32 there) while other tiers may take DF32: on a
    27-point stencil with random values, where every row keeps its structure,
    the result equals the oracle bit for bit (float64 in A-row storage order)."""
    A0 = I.stencil_3d(18, 18, 18, 27, 26.0, -1.0)
    A = I.ensure_csr(A0.m, A0.n, A0.rowptr, A0.colind, I.uniform01(7, "auto.vals", A0.nnz) * 2 - 1)
    rp, ci, va, _, st = run_gpu(A, A, arith=0)
    assert st["kept_structure_rows"] == A.m
    check_against_oracle(A, A, rp, ci, va, exact=True)
