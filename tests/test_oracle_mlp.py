"""Pins of the learned-form oracle: MLP gradients against central finite
differences (float64), features against invariants of the product."""
import numpy as np

import oracle
from oracle import features as FE
from oracle import mlp as M
from paper_2103_11991_gb300 import inputs as I


def _theta(seed):
    u = I.uniform01(seed, "theta", M.NUM_PARAMS)
    return (u - 0.5) * 0.6


def test_param_count():
    assert M.NUM_PARAMS == 8 * 32 + 32 + 32 * 32 + 32 + 32 * 16 + 16


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(23, M.F))
    y = rng.integers(0, M.C, size=23)
    th = _theta(1)
    g = M.grad(th, X, y)
    h = 1e-6
    idx = np.linspace(0, M.NUM_PARAMS - 1, 120).astype(int)
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss(tp, X, y) - M.loss(tm, X, y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (k, fd, g[k])


def test_loss_of_uniform_logits_is_log_classes():
    th = np.zeros(M.NUM_PARAMS)
    X = np.ones((5, M.F))
    y = np.arange(5)
    assert abs(M.loss(th, X, y) - np.log(M.C)) < 1e-12


def test_capacity_class_boundaries():
    c = np.array([0, 1, 16, 17, 32, 33, 64, 65, 16 * 2 ** 14, 16 * 2 ** 14 + 1, 10 ** 9])
    cls = FE.capacity_class(c)
    assert list(cls) == [0, 0, 0, 1, 1, 2, 2, 3, 14, 15, 15]
    assert np.all(FE.class_capacity(cls[:-1]) >= c[:-1])


def test_features_against_product_invariants():
    for seed in range(3):
        A = I.random_sparse(40, 30, 0.15, seed, empty_rows=0.1)
        B = I.random_sparse(30, 50, 0.2, seed + 9, unsorted=True)
        X = FE.row_features(A, B)
        cnt = oracle.symbolic(A, B)
        flop = oracle.row_flops(A, B)
        assert np.allclose(2.0 ** X[:, 1] - 1.0, flop)
        span = np.rint(2.0 ** X[:, 5] - 1.0)
        assert np.all(span >= cnt)             # all of C(i,:) lies in the span window
        assert np.all(np.rint(2.0 ** X[:, 6] - 1.0) >= cnt)
        assert np.all(np.rint(2.0 ** X[:, 7] - 1.0) >= cnt)
        assert np.all(np.rint(2.0 ** X[:, 7] - 1.0) <= B.n)
        nnza = np.rint(2.0 ** X[:, 0] - 1.0)
        assert np.array_equal(nnza, np.diff(A.rowptr))


def _read_features_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "features_hand_worked.txt")
    k, brows, arows, feats = None, {}, {}, {}
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        tag, rest = line[0], line[1:]
        if tag == "K":
            k = int(rest[0])
        elif tag in ("A", "B"):
            (arows if tag == "A" else brows)[int(rest[0])] = [int(c) for c in rest[1:]]
        elif tag == "F":
            feats[int(rest[0])] = [float(v) for v in rest[1:]]

    def csr(rows, n):
        m = len(rows)
        rp = np.zeros(m + 1, dtype=np.int64)
        ci = []
        for r in range(m):
            ci += rows[r]
            rp[r + 1] = len(ci)
        return I.CSR(m, n, rp, np.array(ci, dtype=np.int64), np.ones(len(ci)))

    B = csr(brows, k)
    A = csr(arows, len(brows))
    return A, B, feats


def test_features_match_hand_worked_rows():
    """Every feature, including the max / mean / spread of the referenced B-row
    lengths, against rows worked by hand (tests/golden/features_hand_worked.txt):
    a max/min swap, a mean over distinct columns instead of entries, or a span
    that counts empty B rows fails here."""
    A, B, feats = _read_features_golden()
    X = FE.row_features(A, B)
    raw = 2.0 ** X - 1.0
    for i, want in feats.items():
        assert np.allclose(raw[i], want, rtol=1e-12, atol=1e-12), (i, raw[i], want)


def _theta_with_logits(logits):
    """Parameters whose network outputs the given logits for every input:
    all weights zero, the last bias = logits."""
    th = np.zeros(M.NUM_PARAMS)
    th[-M.C:] = logits
    return th


def test_predict_class_quantile_rule_hand_computed():
    """predict_class(quantile > 0) is the smallest class whose cumulative
    softmax probability reaches the quantile, classes taken in index order.
    Logits log(p) with p = (0.2, 0.3, 0.5) on classes 0..2 and -1000 on the
    others give the softmax p; cumulative 0.2, 0.5, 1.0."""
    logits = np.full(M.C, -1000.0)
    logits[:3] = np.log([0.2, 0.3, 0.5])
    th = _theta_with_logits(logits)
    X = np.zeros((1, M.F))
    assert M.predict_class(th, X, 0.0)[0] == 2          # argmax
    for q, want in [(0.1, 0), (0.19, 0), (0.21, 1), (0.49, 1), (0.51, 2), (0.95, 2), (0.999, 2)]:
        assert M.predict_class(th, X, q)[0] == want, q
    # mass on the last class: cumulative reaches any quantile below 1 only there
    logits = np.full(M.C, -1000.0)
    logits[M.C - 1] = 0.0
    assert M.predict_class(_theta_with_logits(logits), X, 0.95)[0] == M.C - 1
    # uniform over all classes: cumulative (t + 1) / C
    th = np.zeros(M.NUM_PARAMS)
    assert M.predict_class(th, X, 0.5)[0] == M.C // 2 - 1
    assert M.predict_class(th, X, 0.5 + 0.5 / M.C)[0] == M.C // 2
