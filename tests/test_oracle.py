"""Pins of the CPU oracle against facts that do not come from the oracle itself:
dense brute force, hand-worked and closed-form products, and invariants of the
product C = A*B (Kokkos Kernels paper, Sec. "Standard SpGEMM Kernel", Eq. 1)."""
import numpy as np
import pytest

import oracle as O
from paper_2103_11991_gb300 import inputs as I
from tests._util import (REL_TOL, assert_structure_equal, assert_values_within, csr_from_rows,
                         pattern_dense, read_golden_rows)


def _dense_check(A, B):
    C = O.spgemm(A, B)
    pat = (pattern_dense(A).astype(np.int64) @ pattern_dense(B).astype(np.int64)) > 0
    assert np.array_equal(pattern_dense(C), pat), "structure differs from the boolean product"
    # columns ascending and distinct within each row
    for i in range(C.m):
        cols = C.colind[C.rowptr[i]:C.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
    D = A.to_dense() @ B.to_dense()
    Dabs = np.abs(A.to_dense()) @ np.abs(B.to_dense())
    rows = np.repeat(np.arange(C.m), np.diff(C.rowptr))
    assert_values_within(C.vals, D[rows, C.colind], Dabs[rows, C.colind] + 1e-300)
    return C


@pytest.mark.parametrize("seed", range(12))
def test_dense_bruteforce_random(seed):
    u = I.uniform01(seed, "test.dims", 4)
    m, n, k = 1 + int(u[0] * 40), 1 + int(u[1] * 40), 1 + int(u[2] * 40)
    dens = [0.0, 0.05, 0.2, 0.6][seed % 4]
    A = I.random_sparse(m, n, dens, seed, duplicates=seed % 3 == 0, unsorted=seed % 2 == 0,
                        empty_rows=0.2)
    B = I.random_sparse(n, k, min(0.6, dens + 0.1), seed + 100, duplicates=seed % 5 == 0,
                        unsorted=seed % 3 == 1)
    _dense_check(A, B)


def test_dense_bruteforce_empty_dims():
    A = I.random_sparse(5, 0, 0.5, 1)
    B = I.random_sparse(0, 7, 0.5, 2)
    C = O.spgemm(A, B)
    assert C.nnz == 0 and np.all(C.rowptr == 0)
    A = I.random_sparse(0, 4, 0.5, 1)
    B = I.random_sparse(4, 3, 0.5, 2)
    C = O.spgemm(A, B)
    assert C.nnz == 0 and len(C.rowptr) == 1


def test_hand_worked_example():
    g = read_golden_rows("hand_worked_3x3.txt")
    A = csr_from_rows(g["A"], 3, 3)
    B = csr_from_rows(g["B"], 3, 2)
    C = O.spgemm(A, B)
    want = csr_from_rows(g["C"], 3, 2)
    assert_structure_equal(C.rowptr, C.colind, want.rowptr, want.colind)
    assert np.array_equal(C.vals, want.vals)
    A2 = csr_from_rows(g["A2"], 1, 2)
    B2 = csr_from_rows(g["B2"], 2, 1)
    C2 = O.spgemm(A2, B2)
    assert C2.nnz == 1 and C2.vals[0] == 0.0  # cancellation keeps the structural entry


def test_laplacian1d_squared_golden():
    g = read_golden_rows("laplacian1d_n8_squared.txt")["C"]
    A = I.laplacian_1d(8)
    C = O.spgemm(A, A)
    want = csr_from_rows(g, 8, 8)
    assert_structure_equal(C.rowptr, C.colind, want.rowptr, want.colind)
    assert np.array_equal(C.vals, want.vals)


def test_laplacian1d_squared_interior_large():
    n = 1000
    A = I.laplacian_1d(n)
    C = O.spgemm(A, A)
    for i in range(2, n - 2):
        s = slice(C.rowptr[i], C.rowptr[i + 1])
        assert list(C.colind[s]) == [i - 2, i - 1, i, i + 1, i + 2]
        assert list(C.vals[s]) == [1.0, -4.0, 6.0, -4.0, 1.0]


def _kernel_rows(C, g, dims):
    """Interior row of a stencil product as a dict offset-tuple -> value."""
    centre = tuple(d // 2 for d in dims)
    strides = np.cumprod([1] + list(dims[:-1]))
    i = int(sum(c * s for c, s in zip(centre, strides)))
    cols = C.colind[C.rowptr[i]:C.rowptr[i + 1]].astype(np.int64)
    vals = C.vals[C.rowptr[i]:C.rowptr[i + 1]]
    out = {}
    for c, v in zip(cols, vals):
        off = []
        r = c
        for s in strides[::-1]:
            off.append(r // s)
            r = r % s
        off = tuple(o - ce for o, ce in zip(off[::-1], centre))
        out[off] = v
    return out


def test_closed_form_2d_5pt():
    # A = 4I - (sum of the four unit shifts).  Interior row of A^2 by hand:
    # centre 16 + 4 = 20, unit neighbours 2*4*(-1) = -8, (+-2,0)/(0,+-2) -> 1,
    # diagonal (+-1,+-1) -> 2 (two paths).
    A = I.stencil_2d(11, 11, 5, 4.0, -1.0)
    C = O.spgemm(A, A)
    row = _kernel_rows(C, None, (11, 11))
    want = {}
    for dx in range(-2, 3):
        for dy in range(-2, 3):
            d = abs(dx) + abs(dy)
            if d == 0:
                want[(dx, dy)] = 20.0
            elif d == 1:
                want[(dx, dy)] = -8.0
            elif d == 2:
                want[(dx, dy)] = 2.0 if (dx and dy) else 1.0
    assert row == want


def test_nnz_2d_5pt_64_counts_manhattan_ball():
    # nnz(C) for the 64x64 5-point product = number of (node, node') pairs at
    # Manhattan distance <= 2 inside the grid, counted directly on the grid.
    g = 64
    A = I.stencil_2d(g, g, 5)
    cnt = O.symbolic(A, A)
    x, y = np.meshgrid(np.arange(g), np.arange(g), indexing="ij")
    total = 0
    per = np.zeros((g, g), dtype=np.int64)
    for dx in range(-2, 3):
        for dy in range(-2, 3):
            if abs(dx) + abs(dy) <= 2:
                ok = (x + dx >= 0) & (x + dx < g) & (y + dy >= 0) & (y + dy < g)
                per += ok
                total += int(ok.sum())
    assert total == 51972 and int(cnt.sum()) == total
    assert np.array_equal(cnt, per.T.reshape(-1))


def test_closed_form_3d_27pt():
    # A = 27 I - S with S = s(x)s(x)s, s = [1,1,1] (ones stencil incl. centre), so
    # A^2 = 729 I - 54 S + S^2 and S^2 = t(x)t(x)t with t = s*s = [1,2,3,2,1].
    g = 9
    A = I.stencil_3d(g, g, g, 27, 26.0, -1.0)
    C = O.spgemm(A, A)
    row = _kernel_rows(C, None, (g, g, g))
    t = np.convolve([1, 1, 1], [1, 1, 1])
    S2 = np.einsum("i,j,k->ijk", t, t, t).astype(float)
    S = np.zeros((5, 5, 5))
    S[1:4, 1:4, 1:4] = 1.0
    K = -54.0 * S + S2
    K[2, 2, 2] += 729.0
    want = {(dx, dy, dz): K[dx + 2, dy + 2, dz + 2]
            for dx in range(-2, 3) for dy in range(-2, 3) for dz in range(-2, 3)}
    assert row == want
    assert want[(0, 0, 0)] == 702 and want[(1, 0, 0)] == -36 and want[(1, 1, 1)] == -46


def test_nnz_3d_27pt_product_formula():
    # Each dimension contributes the count of in-range offsets in [-2, 2]; the
    # total factorises: nnz(C) = (sum_x #valid)^3.  For g = 100 that is 494^3.
    for g in (6, 10):
        A = I.stencil_3d(g, g, g, 27, 26.0, -1.0)
        per_dim = sum(sum(1 for d in range(-2, 3) if 0 <= x + d < g) for x in range(g))
        assert int(O.symbolic(A, A).sum()) == per_dim ** 3
    per_dim = sum(sum(1 for d in range(-2, 3) if 0 <= x + d < 100) for x in range(100))
    assert per_dim ** 3 == 120553784


def test_closed_form_galerkin_triple_product():
    # R (A P) with A the 7-point Laplacian (6/-1) and P the 2x2x2 aggregation:
    # inside one block 8 diagonals (48) minus 12 internal edges counted twice
    # (-24) give 24; two face-adjacent blocks share 4 edges (-4).  So the coarse
    # operator is exactly 4 x (7-point Laplacian 6/-1) on the coarse grid.
    g = 8
    d = I.config_inputs("amg_galerkin_128", scale=g)
    A, P, R = d["A"], d["P"], d["R"]
    AP = O.spgemm(A, P)
    APc = I.CSR(AP.m, AP.n, AP.rowptr.astype(np.int32), AP.colind, AP.vals)
    Ac = O.spgemm(R, APc)
    L = I.stencil_3d(g // 2, g // 2, g // 2, 7, 6.0, -1.0)
    assert_structure_equal(Ac.rowptr, Ac.colind, L.rowptr, L.colind)
    assert np.array_equal(Ac.vals, 4.0 * L.vals)
    # nnz of A*P: each fine node reaches the aggregates of itself and its 6 neighbours
    assert AP.nnz == int(sum(len({int(P.colind[j]) for j in A.colind[A.rowptr[i]:A.rowptr[i + 1]]})
                             for i in range(A.m)))


@pytest.mark.parametrize("seed", range(4))
def test_identity_invariant(seed):
    A = I.random_sparse(37, 23, 0.15, seed)
    CI = O.spgemm(A, I.identity(23))
    IC = O.spgemm(I.identity(37), A)
    for C in (CI, IC):
        assert_structure_equal(C.rowptr, C.colind, A.rowptr, A.colind)
        assert np.array_equal(C.vals, A.vals)


@pytest.mark.parametrize("seed", range(4))
def test_permutation_invariant(seed):
    A = I.random_sparse(31, 29, 0.2, seed)
    B = I.random_sparse(29, 31, 0.2, seed + 7)
    p = I.permutation(31, seed)
    q = I.permutation(29, seed + 1)
    C = O.spgemm(A, B)
    Cref = I.permute(I.CSR(C.m, C.n, C.rowptr.astype(np.int32), C.colind, C.vals), p, p)
    Cp = O.spgemm(I.permute(A, p, q), I.permute(B, q, p))
    assert_structure_equal(Cp.rowptr, Cp.colind, Cref.rowptr, Cref.colind)
    Ab = O.spgemm_abs(I.permute(A, p, q), I.permute(B, q, p))
    assert_values_within(Cp.vals, Cref.vals, Ab.vals)


@pytest.mark.parametrize("seed", range(4))
def test_structural_associativity(seed):
    A = I.random_sparse(19, 23, 0.15, seed)
    B = I.random_sparse(23, 17, 0.15, seed + 1)
    Cm = I.random_sparse(17, 21, 0.15, seed + 2)
    AB = O.spgemm(A, B)
    BC = O.spgemm(B, Cm)
    to = lambda X: I.CSR(X.m, X.n, X.rowptr.astype(np.int32), X.colind, X.vals)
    L = O.spgemm(to(AB), Cm)
    R = O.spgemm(A, to(BC))
    assert_structure_equal(L.rowptr, L.colind, R.rowptr, R.colind)
    Aa, Ba, Ca = (I.CSR(X.m, X.n, X.rowptr, X.colind, np.abs(X.vals)) for X in (A, B, Cm))
    bound = O.spgemm(to(O.spgemm(Aa, Ba)), Ca).vals
    assert np.all(np.abs(L.vals - R.vals) <= 2 * REL_TOL * bound + 1e-300)


@pytest.mark.parametrize("seed", range(3))
def test_row_sums_and_counts(seed):
    A = I.random_sparse(40, 30, 0.2, seed, duplicates=True)
    B = I.random_sparse(30, 50, 0.2, seed + 3)
    C = O.spgemm(A, B)
    ones = np.ones(B.n)
    lhs = np.add.reduceat(C.vals, C.rowptr[:-1]) * (np.diff(C.rowptr) > 0) if C.nnz else np.zeros(C.m)
    rhs = A.to_dense() @ (B.to_dense() @ ones)
    scale = np.abs(A.to_dense()) @ (np.abs(B.to_dense()) @ ones)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale + 1e-300)
    cnt = O.symbolic(A, B)
    flop = O.row_flops(A, B)
    assert int(cnt.sum()) == C.nnz
    assert np.all(cnt <= np.minimum(flop, B.n))
    # total flops = sum over inner index j of (#A entries in column j) * nnz(B(j,:))
    colcount = np.bincount(A.colind, minlength=A.n)
    assert int(flop.sum()) == int((colcount * B.row_lengths()).sum())


def test_row_blocks_agree_with_whole():
    A = I.rmat(9, 8, seed=3)
    C = O.spgemm(A, A)
    for r0, r1 in [(0, 100), (100, 101), (101, A.m)]:
        Cb = O.spgemm(A, A, r0, r1)
        base = C.rowptr[r0]
        assert np.array_equal(Cb.rowptr, C.rowptr[r0:r1 + 1] - base)
        assert np.array_equal(Cb.colind, C.colind[base:C.rowptr[r1]])
        assert np.array_equal(Cb.vals, C.vals[base:C.rowptr[r1]])


def test_planted_mistakes_are_caught():
    # The comparison helpers must reject a dropped term, a wrong sign and a
    # transposed operand produced by a deliberately broken copy of the oracle.
    A = I.random_sparse(12, 9, 0.3, 5)
    B = I.random_sparse(9, 11, 0.3, 6)
    C = O.spgemm(A, B)
    ab = O.spgemm_abs(A, B).vals
    with pytest.raises(AssertionError):
        v = C.vals.copy()
        v[0] = -v[0] if v[0] != 0 else 1.0
        assert_values_within(v, C.vals, ab)
    with pytest.raises(AssertionError):
        # drop the last contribution of row 0 (a dropped term)
        j = A.colind[A.rowptr[1] - 1]
        A2 = A.copy()
        A2.vals[A.rowptr[1] - 1] = 0.0
        assert_values_within(O.spgemm(A2, B).vals, C.vals, ab)
    with pytest.raises(AssertionError):
        Bt = I.transpose(I.random_sparse(11, 9, 0.3, 6))
        Ct = O.spgemm(A, Bt)
        assert_structure_equal(Ct.rowptr, Ct.colind, C.rowptr, C.colind)
