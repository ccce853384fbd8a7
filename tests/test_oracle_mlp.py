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
