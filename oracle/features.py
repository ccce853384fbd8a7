"""Row features and capacity labels of the learned row-capacity predictor,
written from their plain definitions (numpy, float64).  TEST INFRASTRUCTURE
ONLY (see oracle/__init__.py).

For row i of A (C = A*B) with referenced B rows R_i = {j : j in A(i,:)}:
  nnzA   = |A(i,:)| (entries, repeats counted)
  flop   = sum_{j in A(i,:)} nnz(B(j,:))           (the symbolic phase's bound)
  maxlen = max nnz(B(j,:)), minlen = min nnz(B(j,:)) over the entries (0 if none)
  mean   = flop / nnzA (0 if nnzA = 0)
  span   = max_j maxcol(B(j,:)) - min_j mincol(B(j,:)) + 1 over non-empty B rows
           (0 if there is none): every column of C(i,:) lies in that window
Features, in this order (F = 8), each log2(1 + value):
  nnzA, flop, maxlen, mean, maxlen - minlen, span, min(flop, span),
  min(flop, span, k)
Label: the capacity class of c = nnz(C(i,:)): class 0 holds c <= 16, class t
holds 16*2^(t-1) < c <= 16*2^t, capped at NUM_CLASSES - 1.  Capacity of class
t is 16*2^t entries.
"""
import numpy as np

NUM_FEATURES = 8
NUM_CLASSES = 16


def row_features(A, B) -> np.ndarray:
    arp = np.asarray(A.rowptr, dtype=np.int64)
    aci = np.asarray(A.colind, dtype=np.int64)
    brp = np.asarray(B.rowptr, dtype=np.int64)
    bci = np.asarray(B.colind, dtype=np.int64)
    blen = np.diff(brp)
    n = B.m
    bmin = np.full(n, np.iinfo(np.int64).max)
    bmax = np.full(n, -1, dtype=np.int64)
    rows_b = np.repeat(np.arange(n), blen)
    np.minimum.at(bmin, rows_b, bci)
    np.maximum.at(bmax, rows_b, bci)
    out = np.zeros((A.m, NUM_FEATURES), dtype=np.float64)
    for i in range(A.m):
        js = aci[arp[i]:arp[i + 1]]
        nnza = len(js)
        lens = blen[js]
        flop = int(lens.sum())
        mx = int(lens.max()) if nnza else 0
        mn = int(lens.min()) if nnza else 0
        mean = flop / nnza if nnza else 0.0
        ne = js[lens > 0]
        span = int(bmax[ne].max() - bmin[ne].min() + 1) if len(ne) else 0
        vals = [nnza, flop, mx, mean, mx - mn, span, min(flop, span), min(flop, span, B.n)]
        out[i] = np.log2(1.0 + np.asarray(vals, dtype=np.float64))
    return out


def capacity_class(counts) -> np.ndarray:
    c = np.asarray(counts, dtype=np.int64)
    cls = np.zeros(len(c), dtype=np.int64)
    big = c > 16
    cls[big] = np.ceil(np.log2(c[big] / 16.0)).astype(np.int64)
    # exact integer correction of the float log (c / 16 a power of two)
    cls[big & (16 * (1 << np.minimum(cls, 62)) < c)] += 1
    return np.minimum(cls, NUM_CLASSES - 1)


def class_capacity(cls) -> np.ndarray:
    return 16 * (1 << np.asarray(cls, dtype=np.int64))
