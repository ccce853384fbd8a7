"""Seeded synthetic CSR inputs shared by the tests, the oracle checks and the bench.

This module holds no SpGEMM arithmetic: it only builds input matrices (stencil
Laplacians, an aggregation prolongator and its transpose, R-MAT power-law graphs,
uniform random rows, batches of independent pairs) and reindexes them
(permutation).  Every random draw comes from one counter-based generator,
SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output t of stream (seed, purpose) is
``mix64(base + (t + 1) * GAMMA)`` with ``base = mix64(seed * GAMMA ^ purpose)``.

CSR convention (Kokkos Kernels paper, Sec. 2 "Sparse Linear Algebra": row
pointers, column indices, values): 0-based, int32 row pointers and column
indices, float64 values.  Generators emit rows with ascending, distinct columns.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "CSR", "splitmix_stream", "uniform01", "laplacian_1d", "stencil_2d", "stencil_3d",
    "aggregation_prolongator", "transpose", "rmat", "random_rows", "random_sparse",
    "identity", "permutation", "permute", "batch_pairs", "config_inputs",
    "ensure_csr",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclasses.dataclass
class CSR:
    """Host CSR matrix: ``m`` rows, ``n`` columns."""
    m: int
    n: int
    rowptr: np.ndarray  # int32[m+1] (int64 allowed for outputs)
    colind: np.ndarray  # int32[nnz]
    vals: np.ndarray    # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if self.m > 0 else 0

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), self.row_lengths())
        np.add.at(d, (rows, self.colind.astype(np.int64)), self.vals)
        return d

    def copy(self) -> "CSR":
        return CSR(self.m, self.n, self.rowptr.copy(), self.colind.copy(), self.vals.copy())


def ensure_csr(m, n, rowptr, colind, vals) -> CSR:
    return CSR(int(m), int(n), np.ascontiguousarray(rowptr, dtype=np.int32),
               np.ascontiguousarray(colind, dtype=np.int32),
               np.ascontiguousarray(vals, dtype=np.float64))


# ----------------------------------------------------------------------------
# SplitMix64 counter-based streams
# ----------------------------------------------------------------------------
def _mix64(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def _purpose_id(purpose: str) -> np.uint64:
    h = 1469598103934665603  # FNV-1a 64 over the purpose tag
    for ch in purpose.encode():
        h = ((h ^ ch) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(h)


def splitmix_stream(seed: int, purpose: str, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the stream (seed, purpose), uint64."""
    with np.errstate(over="ignore"):
        base = _mix64(np.array([np.uint64(seed) * _GAMMA ^ _purpose_id(purpose)], dtype=np.uint64))[0]
        t = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(base + t * _GAMMA)


def uniform01(seed: int, purpose: str, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    x = splitmix_stream(seed, purpose, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _uniform_int(seed: int, purpose: str, count: int, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by multiply-shift on 32 random bits."""
    span = hi - lo + 1
    x = splitmix_stream(seed, purpose, start, count) >> np.uint64(32)
    return (lo + ((x * np.uint64(span)) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


# ----------------------------------------------------------------------------
# CSR assembly helpers (pure reindexing)
# ----------------------------------------------------------------------------
def _from_sorted_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("input matrix too large for int32 row pointers")
    return CSR(m, n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def _coo_to_csr_merge(m: int, n: int, rows: np.ndarray, cols: np.ndarray) -> tuple:
    """Sort (row, col) pairs and drop duplicates; returns (rowptr, colind)."""
    key = rows.astype(np.int64) * np.int64(n) + cols.astype(np.int64)
    key = np.sort(key)
    if len(key):
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    r = (key // n).astype(np.int64)
    c = (key % n).astype(np.int32)
    counts = np.bincount(r, minlength=m).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr.astype(np.int32), c


# ----------------------------------------------------------------------------
# Stencil Laplacians (truncated at the boundary: no ghost nodes)
# ----------------------------------------------------------------------------
def laplacian_1d(n: int, diag: float = 2.0, off: float = -1.0) -> CSR:
    """Tridiagonal [off, diag, off] on n nodes."""
    return _stencil([n], [(-1,), (0,), (1,)], diag, off)


def _stencil(dims, offsets, diag, off) -> CSR:
    """Generic stencil on a lexicographic grid: node id = x + nx*y + nx*ny*z.
    ``offsets`` must be listed in ascending order of their linear offset so the
    generated rows come out sorted."""
    dims = list(dims)
    nd = len(dims)
    N = int(np.prod(dims))
    coords = np.indices(dims[::-1]).reshape(nd, -1)[::-1]  # coords[d] for d = x, y, z
    strides = [int(np.prod(dims[:d])) for d in range(nd)]
    node = np.arange(N, dtype=np.int64)
    cols = np.empty((N, len(offsets)), dtype=np.int64)
    valid = np.ones((N, len(offsets)), dtype=bool)
    vals = np.empty((N, len(offsets)), dtype=np.float64)
    for t, o in enumerate(offsets):
        lin = 0
        for d in range(nd):
            cd = coords[d] + o[d]
            valid[:, t] &= (cd >= 0) & (cd < dims[d])
            lin += o[d] * strides[d]
        cols[:, t] = node + lin
        vals[:, t] = diag if all(v == 0 for v in o) else off
    rows = np.repeat(node, len(offsets)).reshape(N, len(offsets))
    return _from_sorted_coo(N, N, rows[valid], cols[valid], vals[valid])


def stencil_2d(nx: int, ny: int, points: int = 5, diag: float = 4.0, off: float = -1.0) -> CSR:
    """2D 5-point or 9-point stencil on an nx-by-ny grid."""
    if points == 5:
        offs = [(0, -1), (-1, 0), (0, 0), (1, 0), (0, 1)]
    elif points == 9:
        offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError("points must be 5 or 9")
    return _stencil([nx, ny], offs, diag, off)


def stencil_3d(nx: int, ny: int, nz: int, points: int = 7, diag: float = 6.0, off: float = -1.0) -> CSR:
    """3D 7-point or 27-point stencil on an nx-by-ny-by-nz grid."""
    if points == 7:
        offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    elif points == 27:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError("points must be 7 or 27")
    return _stencil([nx, ny, nz], offs, diag, off)


# ----------------------------------------------------------------------------
# Aggregation prolongator and explicit transpose
# ----------------------------------------------------------------------------
def aggregation_prolongator(nx: int, ny: int, nz: int, block: int = 2) -> CSR:
    """Piecewise-constant prolongator: node (x,y,z) -> aggregate
    (x/b) + ax*(y/b) + ax*ay*(z/b), one 1.0 per row."""
    ax, ay, az = -(-nx // block), -(-ny // block), -(-nz // block)
    N = nx * ny * nz
    node = np.arange(N, dtype=np.int64)
    x = node % nx
    y = (node // nx) % ny
    z = node // (nx * ny)
    agg = (x // block) + ax * (y // block) + ax * ay * (z // block)
    return _from_sorted_coo(N, ax * ay * az, node, agg, np.ones(N))


def transpose(A: CSR) -> CSR:
    """Explicit CSR transpose (stable: within a row of A^T, columns ascend)."""
    rows = np.repeat(np.arange(A.m, dtype=np.int64), A.row_lengths())
    order = np.lexsort((rows, A.colind.astype(np.int64)))
    t_rows = A.colind.astype(np.int64)[order]
    return _from_sorted_coo(A.n, A.m, t_rows, rows[order], A.vals[order])


# ----------------------------------------------------------------------------
# R-MAT power-law graph
# ----------------------------------------------------------------------------
def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0) -> CSR:
    """R-MAT (Chakrabarti, Zhan, Faloutsos 2004) on 2^scale vertices with
    edge_factor * 2^scale directed edges.  For each edge and each bit level the
    quadrant is drawn with probabilities a, b, c, d = 1-a-b-c; b sets the column
    bit, c the row bit, d both.  No noise, no vertex permutation, self-loops
    kept, duplicate edges merged into one entry.  Values are drawn after merging,
    uniform in [-1, 1), in CSR order."""
    n = 1 << scale
    E = edge_factor * n
    rows = np.zeros(E, dtype=np.int64)
    cols = np.zeros(E, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for lvl in range(scale):
        u = uniform01(seed, "rmat.quadrant", E, start=lvl * E)
        bit = np.int64(1 << (scale - 1 - lvl))
        col_bit = ((u >= a) & (u < ab)) | (u >= abc)
        row_bit = (u >= ab)
        rows += row_bit.astype(np.int64) * bit
        cols += col_bit.astype(np.int64) * bit
    rowptr, colind = _coo_to_csr_merge(n, n, rows, cols)
    vals = uniform01(seed, "rmat.values", len(colind)) * 2.0 - 1.0
    return CSR(n, n, rowptr, colind, vals)


# ----------------------------------------------------------------------------
# Uniform random rows
# ----------------------------------------------------------------------------
def random_rows(m: int, n: int, nnz_lo: int, nnz_hi: int, seed: int, purpose: str = "rows") -> CSR:
    """m rows of n columns; row i has U{nnz_lo..nnz_hi} (capped at n) distinct
    columns drawn uniformly, sorted; values uniform in [-1, 1).  Each row draws
    2*cnt+8 candidate columns and keeps the first cnt distinct ones in draw
    order; a row left short (rare) is topped up with the next unused columns
    after a seeded offset."""
    cnt = np.minimum(_uniform_int(seed, purpose + ".cnt", m, nnz_lo, nnz_hi), n)
    k = 2 * cnt + 8
    r = np.repeat(np.arange(m, dtype=np.int64), k)
    draws = _uniform_int(seed, purpose + ".col", int(k.sum()), 0, n - 1)
    key = r * np.int64(n) + draws
    order = np.argsort(key, kind="stable")
    ks = key[order]
    first = order[np.concatenate(([True], ks[1:] != ks[:-1]))] if len(ks) else order
    first.sort()
    r1, c1 = r[first], draws[first]
    rowstart = np.searchsorted(r1, np.arange(m, dtype=np.int64))
    rank = np.arange(len(r1), dtype=np.int64) - rowstart[r1]
    keep = rank < cnt[r1]
    r1, c1 = r1[keep], c1[keep]
    got = np.bincount(r1, minlength=m)
    short = np.nonzero(got < cnt)[0]
    if len(short):
        extra_r, extra_c = [], []
        offs = _uniform_int(seed, purpose + ".topup", len(short), 0, n - 1)
        for t, i in enumerate(short):
            used = set(c1[r1 == i].tolist())
            c = int(offs[t])
            while len(used) < cnt[i]:
                if c not in used:
                    used.add(c)
                    extra_r.append(i)
                    extra_c.append(c)
                c = (c + 1) % n
        r1 = np.concatenate([r1, np.array(extra_r, np.int64)])
        c1 = np.concatenate([c1, np.array(extra_c, np.int64)])
    rowptr, colind = _coo_to_csr_merge(m, n, r1, c1)
    vals = uniform01(seed, purpose + ".vals", len(colind)) * 2.0 - 1.0
    return CSR(m, n, rowptr, colind, vals)


def random_sparse(m: int, n: int, density: float, seed: int, duplicates: bool = False,
                  unsorted: bool = False, empty_rows: float = 0.0, integer: bool = False) -> CSR:
    """Small random matrix for brute-force checks.  With ``duplicates`` some
    entries repeat a column within their row; with ``unsorted`` each row's
    entries are shuffled; ``empty_rows`` is the probability a row is empty;
    ``integer`` draws small integer values (exact products and sums)."""
    total = m * n
    u = uniform01(seed, "rs.mask", total).reshape(m, n)
    mask = u < density
    if empty_rows > 0:
        e = uniform01(seed, "rs.empty", m) < empty_rows
        mask[e, :] = False
    rows, cols = np.nonzero(mask)
    rows = rows.astype(np.int64)
    cols = cols.astype(np.int64)
    if duplicates and len(rows):
        d = uniform01(seed, "rs.dup", len(rows)) < 0.3
        rows = np.concatenate([rows, rows[d]])
        cols = np.concatenate([cols, cols[d]])
        o = np.lexsort((cols, rows))
        rows, cols = rows[o], cols[o]
    if unsorted and len(rows):
        pr = uniform01(seed, "rs.perm", len(rows))
        o = np.lexsort((pr, rows))
        rows, cols = rows[o], cols[o]
    if integer:
        vals = (_uniform_int(seed, "rs.ivals", len(rows), -4, 4)).astype(np.float64)
    else:
        vals = uniform01(seed, "rs.vals", len(rows)) * 2.0 - 1.0
    return _from_sorted_coo(m, n, rows, cols, vals)


def with_diagonal(A: CSR, seed: int, lo: float = 1.0, hi: float = 2.0, split: bool = False) -> CSR:
    """Square A with a stored diagonal entry in every row: rows that lack one get
    an entry appended at the end of the row (so unsorted rows stay unsorted),
    value uniform in [lo, hi) with a random sign.  ``split`` also stores the
    diagonal of every other row as two entries (a repeated column) whose values
    add up to the drawn one."""
    if A.m != A.n:
        raise ValueError("with_diagonal needs a square matrix")
    m = A.m
    rows = np.repeat(np.arange(m, dtype=np.int64), A.row_lengths())
    cols = A.colind.astype(np.int64)
    vals = A.vals.astype(np.float64)
    on = rows == cols
    has = np.zeros(m, dtype=bool)
    has[rows[on]] = True
    # existing diagonal entries are redrawn too, so that no row sums to zero
    u = uniform01(seed, "diag.vals", m)
    sg = np.where(uniform01(seed, "diag.sign", m) < 0.5, -1.0, 1.0)
    d = sg * (lo + (hi - lo) * u)
    keep_first = np.zeros(len(rows), dtype=bool)
    if on.any():
        first = np.nonzero(on)[0]
        _, idx = np.unique(rows[first], return_index=True)
        keep_first[first[idx]] = True
    vals = np.where(on, 0.0, vals)
    vals = np.where(keep_first, d[rows], vals)
    add_r = np.nonzero(~has)[0]
    pieces_r = [rows, add_r]
    pieces_c = [cols, add_r]
    pieces_v = [vals, d[add_r]]
    if split:
        sr = np.arange(0, m, 2, dtype=np.int64)
        half = 0.25 * d[sr]
        pieces_r.append(sr)
        pieces_c.append(sr)
        pieces_v.append(half)
        # the first stored diagonal entry of these rows keeps d - d/4
        first_of = np.full(m, -1, dtype=np.int64)
        allr = np.concatenate(pieces_r[:2])
        allc = np.concatenate(pieces_c[:2])
        alld = np.nonzero(allr == allc)[0]
        first_of[allr[alld[::-1]]] = alld[::-1]
        v01 = np.concatenate(pieces_v[:2])
        v01[first_of[sr]] -= half
        pieces_v[0], pieces_v[1] = v01[:len(rows)], v01[len(rows):]
    r = np.concatenate(pieces_r)
    c = np.concatenate(pieces_c)
    v = np.concatenate(pieces_v)
    o = np.argsort(r, kind="stable")  # entries keep their order within a row
    return _from_sorted_coo(m, m, r[o], c[o], v[o])


# ----------------------------------------------------------------------------
# Identity and permutations (for invariants)
# ----------------------------------------------------------------------------
def identity(n: int) -> CSR:
    idx = np.arange(n, dtype=np.int64)
    return _from_sorted_coo(n, n, idx, idx, np.ones(n))


def permutation(n: int, seed: int) -> np.ndarray:
    """A uniformly random permutation of 0..n-1 (argsort of seeded keys)."""
    return np.argsort(splitmix_stream(seed, "perm", 0, n), kind="stable").astype(np.int64)


def permute(A: CSR, row_perm: np.ndarray | None, col_perm: np.ndarray | None) -> CSR:
    """Return P_r A P_c^T: row i of the result is row row_perm[i] of A, and
    column col_perm[c] of A becomes column c; rows re-sorted by column."""
    m, n = A.m, A.n
    rp = np.arange(m) if row_perm is None else np.asarray(row_perm, dtype=np.int64)
    inv_c = np.arange(n) if col_perm is None else np.argsort(np.asarray(col_perm, dtype=np.int64))
    lens = A.row_lengths()
    src_rows = rp
    new_lens = lens[src_rows]
    starts = A.rowptr.astype(np.int64)[src_rows]
    idx = np.repeat(starts - np.concatenate([[0], np.cumsum(new_lens)[:-1]]), new_lens) + np.arange(new_lens.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), new_lens)
    cols = inv_c[A.colind.astype(np.int64)[idx]]
    vals = A.vals[idx]
    o = np.lexsort((cols, rows))
    return _from_sorted_coo(m, n, rows[o], cols[o], vals[o])


# ----------------------------------------------------------------------------
# Batches of independent pairs (uneven sizes)
# ----------------------------------------------------------------------------
def _batch_operand(seed: int, tag: str, nx: int, ny: int) -> CSR:
    n = nx * ny
    kind = int(splitmix_stream(seed, tag + ".kind", 0, 1)[0] >> np.uint64(63))
    if kind == 0:
        pts = 5 if (int(splitmix_stream(seed, tag + ".pts", 0, 1)[0] >> np.uint64(63)) == 0) else 9
        return stencil_2d(nx, ny, pts, 4.0 if pts == 5 else 8.0, -1.0)
    return random_rows(n, n, 3, 40, seed, purpose=tag)


def batch_pairs(count: int, seed0: int = 5000, rows_lo: int = 100, rows_hi: int = 50000) -> list:
    """``count`` independent pairs (A_k, B_k), pair k drawn from seed seed0 + k:
    row count r log-uniform in [rows_lo, rows_hi]; grid nx = round(sqrt(r)),
    ny = round(r / nx), n = nx*ny; A_k and B_k independently a 2D 5/9-point
    Laplacian (coin flips; values 4/-1 or 8/-1) or uniform random rows with
    U{3..40} nonzeros, values uniform in [-1, 1)."""
    out = []
    for t in range(count):
        s = seed0 + t
        u = float(uniform01(s, "batch.rows", 1)[0])
        r = math.exp(math.log(rows_lo) + u * (math.log(rows_hi) - math.log(rows_lo)))
        nx = max(1, int(round(math.sqrt(r))))
        ny = max(1, int(round(r / nx)))
        out.append((_batch_operand(s, "batch.A", nx, ny), _batch_operand(s, "batch.B", nx, ny)))
    return out


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------
def config_inputs(name: str, **kw):
    """Inputs of the named workload.  Returns a dict with the operands.

    - ``stencil2d_64``: 2D 5-point Laplacian on 64x64 (4 / -1), product A*A.
    - ``stencil3d27_100``: 3D 27-point stencil on 100^3 (26 / -1), product A*A.
    - ``amg_galerkin_128``: 3D 7-point Laplacian on 128^3 (6 / -1), aggregation
      prolongator P over 2x2x2 blocks, R = P^T; products A*P then R*(AP).
    - ``rmat20``: R-MAT scale 20, edge factor 16, (.57, .19, .19), seed 20; A*A.
    - ``batch2000``: 2000 pairs from seeds 5000..6999.
    Keyword ``scale`` shrinks a workload for tests (grid edge or R-MAT scale)."""
    if name == "stencil2d_64":
        g = kw.get("scale", 64)
        A = stencil_2d(g, g, 5, 4.0, -1.0)
        return {"A": A, "B": A}
    if name == "stencil3d27_100":
        g = kw.get("scale", 100)
        A = stencil_3d(g, g, g, 27, 26.0, -1.0)
        return {"A": A, "B": A}
    if name == "amg_galerkin_128":
        g = kw.get("scale", 128)
        A = stencil_3d(g, g, g, 7, 6.0, -1.0)
        P = aggregation_prolongator(g, g, g, 2)
        return {"A": A, "P": P, "R": transpose(P)}
    if name == "rmat20":
        s = kw.get("scale", 20)
        A = rmat(s, 16, 0.57, 0.19, 0.19, seed=kw.get("seed", 20))
        return {"A": A, "B": A}
    if name == "batch2000":
        return {"pairs": batch_pairs(kw.get("count", 2000), kw.get("seed0", 5000))}
    raise KeyError(name)
