"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element.  Structure bit-exact; values within 1e-12 * sum|a||b| (exact for
integer-valued inputs)."""
import numpy as np
import pytest

import oracle
from paper_2103_11991_gb300 import inputs as I
from tests._gpu import check_against_oracle, run_gpu
from tests._util import assert_structure_equal, assert_values_within

pytestmark = pytest.mark.gpu

ARITHS = [1, 2]  # KK_ARITH_FP64, KK_ARITH_DF32
TIERS = [-1, 0, 1, 2, 3]


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("tier", TIERS)
@pytest.mark.parametrize("seed", range(6))
def test_random_small(seed, tier, arith):
    u = I.uniform01(seed, "gpu.dims", 3)
    m, n, k = 1 + int(u[0] * 200), 1 + int(u[1] * 150), 1 + int(u[2] * 300)
    dens = [0.01, 0.05, 0.15, 0.4][seed % 4]
    A = I.random_sparse(m, n, dens, seed, duplicates=seed % 3 == 0, unsorted=seed % 2 == 1,
                        empty_rows=0.1)
    B = I.random_sparse(n, k, dens, seed + 50, duplicates=seed % 4 == 1, unsorted=seed % 3 == 2)
    rp, ci, va, _, _ = run_gpu(A, B, arith=arith, force_tier=tier)
    check_against_oracle(A, B, rp, ci, va)


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("tier", TIERS)
def test_integer_valued_exact(tier, arith):
    A = I.random_sparse(150, 120, 0.1, 3, integer=True)
    B = I.random_sparse(120, 170, 0.1, 4, integer=True)
    rp, ci, va, _, _ = run_gpu(A, B, arith=arith, force_tier=tier)
    check_against_oracle(A, B, rp, ci, va, exact=True)


@pytest.mark.parametrize("arith", ARITHS)
def test_stencil2d_64_exact(arith):
    d = I.config_inputs("stencil2d_64")
    rp, ci, va, _, st = run_gpu(d["A"], d["B"], arith=arith)
    ref = check_against_oracle(d["A"], d["B"], rp, ci, va, exact=True)
    assert ref.nnz == 51972


@pytest.mark.parametrize("window", [0, 1])
@pytest.mark.parametrize("arith", ARITHS)
def test_stencil3d27_small_exact(arith, window):
    d = I.config_inputs("stencil3d27_100", scale=22)
    rp, ci, va, _, st = run_gpu(d["A"], d["B"], arith=arith, use_window=window)
    check_against_oracle(d["A"], d["B"], rp, ci, va, exact=True)
    if window:
        assert st["sym_window_rows"] == d["A"].m and st["num_window_rows"] == d["A"].m


@pytest.mark.parametrize("arith", ARITHS)
def test_window_tier_random_values(arith):
    # stencil structure with random values, and random rows with a narrow span
    d = I.config_inputs("stencil3d27_100", scale=14)
    A = d["A"].copy()
    A.vals = I.uniform01(3, "w", A.nnz) * 2 - 1
    rp, ci, va, _, st = run_gpu(A, A, arith=arith, force_tier=3)
    check_against_oracle(A, A, rp, ci, va)
    assert st["num_window_rows"] > 0
    B = I.random_rows(3000, 3000, 20, 40, seed=4)
    A2 = I.random_rows(400, 3000, 5, 30, seed=5)
    rp, ci, va, _, st = run_gpu(A2, B, arith=arith, force_tier=3)
    check_against_oracle(A2, B, rp, ci, va)


@pytest.mark.parametrize("tier", TIERS)
def test_rmat_small(tier):
    A = I.rmat(11, 16, seed=3)
    rp, ci, va, _, _ = run_gpu(A, A, force_tier=tier)
    check_against_oracle(A, A, rp, ci, va)


def test_rmat_mixed_tiers_auto():
    # scale 13 has rows in every tier under the default thresholds
    A = I.rmat(13, 16, seed=5)
    rp, ci, va, _, st = run_gpu(A, A)
    check_against_oracle(A, A, rp, ci, va)
    assert st["sym_team_rows"] + st["sym_window_rows"] > 0
    assert st["num_team_rows"] + st["num_window_rows"] > 0
    assert st["num_cta_rows"] + st["num_dense_rows"] > 0


def test_dense_tier_multi_chunk():
    # k > one dense chunk (16384 columns): chunks swept with sorted B rows
    A = I.random_rows(60, 50, 20, 40, seed=1)
    B = I.random_rows(50, 70000, 200, 400, seed=2)
    rp, ci, va, _, st = run_gpu(A, B, force_tier=2)
    check_against_oracle(A, B, rp, ci, va)
    B2 = I.random_sparse(50, 40000, 0.01, 3, unsorted=True)
    rp, ci, va, _, st = run_gpu(A, B2, force_tier=2)
    check_against_oracle(A, B2, rp, ci, va)


def test_galerkin_with_symbolic_reuse():
    from paper_2103_11991_gb300 import spgemm as K
    import torch
    d = I.config_inputs("amg_galerkin_128", scale=16)
    A, P, R = d["A"], d["P"], d["R"]
    dA, dP, dR = (K.DeviceCSR.from_host(X) for X in (A, P, R))
    op1, op2 = K.SpGEMM(), K.SpGEMM()
    rp1, nnz1 = op1.symbolic(dA, dP)
    ci1, va1 = op1.numeric(dA, dP, rp1, nnz1)
    dAP = K.DeviceCSR(A.m, P.n, rp1.to(torch.int32), ci1, va1)
    rp2, nnz2 = op2.symbolic(dR, dAP)
    ci2, va2 = op2.numeric(dR, dAP, rp2, nnz2)
    L = I.stencil_3d(8, 8, 8, 7, 6.0, -1.0)
    scales = I.uniform01(11, "refresh", 3) * 1.5 + 0.5
    for it in range(4):
        s = 1.0 if it == 0 else float(scales[it - 1])
        if it > 0:
            dA.vals.copy_(torch.from_numpy(A.vals * s).cuda())
            op1.numeric(dA, dP, rp1, nnz1, ci1, va1)
            op2.numeric(dR, dAP, rp2, nnz2, ci2, va2)
        op1.sync()
        op2.sync()
        assert_structure_equal(rp2.cpu().numpy(), ci2.cpu().numpy(), L.rowptr, L.colind)
        As = I.CSR(A.m, A.n, A.rowptr, A.colind, A.vals * s)
        ref = oracle.spgemm(R, I.CSR(A.m, P.n, oracle.spgemm(As, P).rowptr.astype(np.int32),
                                     oracle.spgemm(As, P).colind, oracle.spgemm(As, P).vals))
        assert np.array_equal(ci2.cpu().numpy(), ref.colind)
        assert np.allclose(va2.cpu().numpy(), ref.vals, rtol=1e-13, atol=0)
        if it == 0:
            assert np.array_equal(va2.cpu().numpy(), 4.0 * L.vals)
    op1.close()
    op2.close()


def test_edge_cases():
    # empty rows everywhere, zero-size dims, single entries
    cases = [
        (I.random_sparse(10, 8, 0.0, 1), I.random_sparse(8, 9, 0.5, 2)),
        (I.random_sparse(10, 8, 0.5, 1), I.random_sparse(8, 9, 0.0, 2)),
        (I.random_sparse(1, 1, 1.0, 1), I.random_sparse(1, 1, 1.0, 2)),
        (I.random_sparse(0, 5, 0.5, 1), I.random_sparse(5, 4, 0.5, 2)),
        (I.random_sparse(6, 0, 0.5, 1), I.random_sparse(0, 4, 0.5, 2)),
        (I.random_sparse(6, 5, 0.5, 1), I.random_sparse(5, 0, 0.5, 2)),
    ]
    for A, B in cases:
        rp, ci, va, _, _ = run_gpu(A, B)
        check_against_oracle(A, B, rp, ci, va)


def test_cancellation_keeps_structural_zero():
    A = I.CSR(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    B = I.CSR(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, -1.0]))
    for arith in ARITHS:
        rp, ci, va, _, _ = run_gpu(A, B, arith=arith)
        assert list(rp) == [0, 1] and list(ci) == [0] and va[0] == 0.0


def test_df32_window_falls_back_to_fp64():
    A = I.random_sparse(40, 30, 0.2, 1)
    B = I.random_sparse(30, 20, 0.2, 2)
    B.vals[3] = 1e-30  # outside the DF32 window -> every row takes the float64 path
    rp, ci, va, arith, _ = run_gpu(A, B, arith=0)
    check_against_oracle(A, B, rp, ci, va)
    assert arith == 1
    A.vals[0] = 1e25  # a row of A outside the window
    B = I.random_sparse(30, 20, 0.2, 2)
    rp, ci, va, arith, _ = run_gpu(A, B, arith=0)
    check_against_oracle(A, B, rp, ci, va)


def test_determinism_vector_mode():
    d = I.config_inputs("stencil3d27_100", scale=16)
    A = d["A"].copy()
    A.vals = I.uniform01(1, "v", A.nnz) * 2 - 1
    r1 = run_gpu(A, A)
    r2 = run_gpu(A, A)
    assert np.array_equal(r1[2], r2[2])
    check_against_oracle(A, A, r1[0], r1[1], r1[2])


def test_errors_reported():
    from paper_2103_11991_gb300 import spgemm as K
    A = I.random_sparse(20, 10, 0.3, 1)
    B = I.random_sparse(10, 12, 0.3, 2)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    op = K.SpGEMM()
    import torch
    rp = torch.zeros(21, dtype=torch.int64, device="cuda")
    c = torch.zeros(4, dtype=torch.int32, device="cuda")
    v = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KKError) as e:
        K.kk_spgemm_numeric(op.h, dA, dB, rp, c, v)
    assert e.value.status == 7
    with pytest.raises(K.KKError) as e:
        K.kk_spgemm_symbolic(op.h, dB, dB, rp)  # 10x12 times 10x12: inner dims differ
    assert e.value.status == 1
    bad = A.copy()
    bad.colind[3] = 10  # column index out of range for B's rows
    with pytest.raises(K.KKError) as e:
        op.symbolic(K.DeviceCSR.from_host(bad), dB)
    assert e.value.status == 8
    rp, nnz = op.symbolic(dA, dB)
    A2 = I.random_sparse(20, 10, 0.5, 9)
    with pytest.raises(K.KKError) as e:
        op.numeric(K.DeviceCSR.from_host(A2), dB, rp, nnz)
    assert e.value.status == 4
    op.close()


@pytest.mark.parametrize("tier", [1, 2])
def test_very_wide_k_uses_hash_and_chunk_tiers(tier):
    # k beyond the wide tier's shared-memory bit vector: the CTA hash and the
    # chunked dense kernels take the CTA and dense bins
    k = 2_000_000
    A = I.random_rows(40, 300, 20, 60, seed=21)
    B = I.random_rows(300, k, 30, 90, seed=22)
    rp, ci, va, _, st = run_gpu(A, B, force_tier=tier)
    check_against_oracle(A, B, rp, ci, va)
    key = "num_cta_rows" if tier == 1 else "num_dense_rows"
    assert st[key] > 0


def test_copy_to_host_kernel():
    import torch
    from paper_2103_11991_gb300 import spgemm as K
    src = torch.arange(1_000_003, dtype=torch.float64, device="cuda") * 0.5
    dst = torch.empty(1_000_003, dtype=torch.float64).pin_memory()
    K.kk_copy_to_host(dst, src)  # 8,000,024 bytes: vectorised kernel
    torch.cuda.synchronize()
    assert torch.equal(dst, src.cpu())
    src32 = torch.arange(1001, dtype=torch.int32, device="cuda")
    dst32 = torch.zeros(1001, dtype=torch.int32).pin_memory()
    K.kk_copy_to_host(dst32, src32)  # 4,004 bytes: not a multiple of 16, copy engine
    torch.cuda.synchronize()
    assert torch.equal(dst32, src32.cpu())
    with pytest.raises(K.KKError) as e:  # pageable destination
        K.kk_copy_to_host(torch.empty(1001, dtype=torch.int32), src32)
    assert e.value.status == 1


def _long_short_rows(seed):
    """A with 48 rows of 200-300 entries and 48 rows of 10-60 entries; B rows
    (k = 256 columns, so every C row fits the window tier's value array) all
    hold columns 0..7, so those entries of a long row get more than 200
    contributions each."""
    long_a = I.random_rows(48, 2000, 200, 300, seed=seed)
    short_a = I.random_rows(48, 2000, 10, 60, seed=seed + 1)
    rp = np.concatenate([long_a.rowptr, long_a.rowptr[-1] + short_a.rowptr[1:]])
    ci = np.concatenate([long_a.colind, short_a.colind])
    A = I.CSR(96, 2000, rp.astype(np.int64), ci, I.uniform01(seed, "long.a", len(ci)) * 2 - 1)
    Br = I.random_rows(2000, 248, 10, 30, seed=seed + 2)
    rows, cols = [], []
    for j in range(2000):
        c = np.concatenate([np.arange(8), 8 + Br.colind[Br.rowptr[j]:Br.rowptr[j + 1]]])
        rows.append(np.full(len(c), j))
        cols.append(c)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    brp = np.zeros(2001, dtype=np.int64)
    np.add.at(brp, rows + 1, 1)
    B = I.CSR(2000, 256, np.cumsum(brp), cols, I.uniform01(seed, "long.b", len(cols)) * 2 - 1)
    return A, B


@pytest.mark.parametrize("seed", [0, 1])
def test_df32_rows_beyond_its_bound_run_in_float64(seed):
    """DF32's error bound (n + 2) * 2^-46 * sum|a||b| is under 1e-12 only up to
    68 contributions per entry: rows of more than 64 A entries must run in
    float64.  The window tier adds in A-row order, so a float64 row matches the
    oracle bit for bit, which a DF32 row of random values does not; the short
    rows still run in DF32 (the handle reports DF32) within the bound."""
    A, B = _long_short_rows(40 + seed)
    rp, ci, va, arith, st = run_gpu(A, B, arith=2, force_tier=3)
    assert arith == 2
    assert st["num_window_rows"] == A.m
    ref = check_against_oracle(A, B, rp, ci, va)
    long_end = int(ref.rowptr[48])
    assert np.array_equal(va[:long_end], ref.vals[:long_end]), "long rows did not run in float64"
    assert not np.array_equal(va[long_end:], ref.vals[long_end:]), "short rows did not run in DF32"
    # every tier keeps the bound on the same product
    for tier in (-1, 0, 1):
        rp, ci, va, _, _ = run_gpu(A, B, arith=2, force_tier=tier)
        check_against_oracle(A, B, rp, ci, va)


def test_df32_needs_strictly_ascending_b():
    """With a repeated column in a B row an entry can get more contributions
    than A(i,:) has entries, so the whole product runs in float64."""
    A = I.random_sparse(120, 90, 0.1, 11)
    B = I.random_sparse(90, 130, 0.1, 12, duplicates=True)
    rp, ci, va, arith, _ = run_gpu(A, B, arith=2)
    assert arith == 1
    check_against_oracle(A, B, rp, ci, va)


@pytest.mark.parametrize("stage", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_wide_rows_beyond_shared_values(seed, stage):
    """Wide-tier rows whose values do not fit shared memory (k = 2^20 columns,
    15,000 to 900,000 columns per row of C): the numeric phase reloads the bit
    vector the symbolic phase kept and adds every product into C's values.
    The B rows are long (600 to 2,600 entries), so both phases take the
    entry-piece walk; four rows have more A entries (1,100 to 1,300) than one
    segment of the walk.  With stage = 1 the symbolic phase copies the long
    B-row pieces into shared memory with bulk copies (options.stage_long_rows)."""
    k = 1 << 20
    n = 3000
    B = I.random_rows(n, k, 600, 2600, seed=60 + seed)
    A1 = I.random_rows(24, n, 10, 30, seed=70 + seed)
    A2 = I.random_rows(4, n, 1100, 1300, seed=80 + seed)
    rp = np.concatenate([A1.rowptr, A1.rowptr[-1] + A2.rowptr[1:]]).astype(np.int64)
    A = I.CSR(28, n, rp, np.concatenate([A1.colind, A2.colind]),
              I.uniform01(seed, "wide.a", int(rp[-1])) * 2 - 1)
    rp_, ci, va, _, st = run_gpu(A, B, stage_long_rows=stage)
    ref = check_against_oracle(A, B, rp_, ci, va)
    assert np.diff(ref.rowptr).max() > 20000
    assert st["num_dense_rows"] + st["num_cta_rows"] > 0
@pytest.mark.parametrize("kbits", [18, 19])
def test_wide_rows_beyond_shared_values_narrower_k(kbits):
    """The same wide-tier rows with k = 2^18 and 2^19 columns: 8 and 16
    bit-vector words per thread of the numeric kernel's rank tables (2^20 gives
    32), rows from 15,000 columns to more than half of k."""
    k = 1 << kbits
    n = 3000
    B = I.random_rows(n, k, 600, 2600, seed=160 + kbits)
    A1 = I.random_rows(24, n, 10, 30, seed=170 + kbits)
    A2 = I.random_rows(4, n, 1100, 1300, seed=180 + kbits)
    rp = np.concatenate([A1.rowptr, A1.rowptr[-1] + A2.rowptr[1:]]).astype(np.int64)
    A = I.CSR(28, n, rp, np.concatenate([A1.colind, A2.colind]),
              I.uniform01(kbits, "wide.a", int(rp[-1])) * 2 - 1)
    rp_, ci, va, _, st = run_gpu(A, B)
    ref = check_against_oracle(A, B, rp_, ci, va)
    assert np.diff(ref.rowptr).max() > k // 2
    assert st["num_dense_rows"] + st["num_cta_rows"] > 0


