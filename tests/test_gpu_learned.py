"""Learned form on the GPU: MLP kernels against the float64 oracle, features
and labels against their plain definitions, and the speculative one-pass
SpGEMM against the Gustavson oracle (structure exact, values within bound),
including the overflow re-run path and the gain of the trained network."""
import numpy as np
import pytest

import oracle
from oracle import features as FE
from oracle import mlp as M
from paper_2103_11991_gb300 import inputs as I
from tests._gpu import check_against_oracle

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _theta(seed, scale=0.6):
    return ((I.uniform01(seed, "theta", M.NUM_PARAMS) - 0.5) * scale).astype(np.float32)


def test_mlp_gradient_matches_oracle():
    torch = _torch()
    from paper_2103_11991_gb300 import spgemm as K
    rng = np.random.default_rng(3)
    X = rng.normal(size=(1000, 8)).astype(np.float32)
    y = rng.integers(0, 16, size=1000).astype(np.int32)
    th = _theta(5)
    dX, dy, dth = (torch.from_numpy(a).cuda() for a in (X, y, th))
    g = torch.empty(M.NUM_PARAMS, dtype=torch.float32, device="cuda")
    l = torch.empty(1, dtype=torch.float32, device="cuda")
    K.kk_mlp_loss_grad(dX, dy, dth, g, l)
    torch.cuda.synchronize()
    ref_g = M.grad(th.astype(np.float64), X.astype(np.float64), y)
    ref_l = M.loss(th.astype(np.float64), X.astype(np.float64), y)
    assert abs(float(l.item()) - ref_l) <= 1e-4 * max(1.0, ref_l)
    np.testing.assert_allclose(g.cpu().numpy(), ref_g, rtol=1e-3, atol=1e-5)


def test_mlp_predict_matches_oracle():
    torch = _torch()
    from paper_2103_11991_gb300 import spgemm as K
    rng = np.random.default_rng(4)
    X = rng.normal(size=(4000, 8)).astype(np.float32) * 3
    th = _theta(9, 1.0)
    cls = torch.empty(4000, dtype=torch.int32, device="cuda")
    for q in (0.0, 0.9):
        K.kk_mlp_predict(torch.from_numpy(X).cuda(), torch.from_numpy(th).cuda(), cls, quantile=q)
        got = cls.cpu().numpy()
        ref = M.predict_class(th.astype(np.float64), X.astype(np.float64), quantile=q)
        assert np.mean(got == ref) > 0.995


def test_adam_step_matches_definition():
    torch = _torch()
    from paper_2103_11991_gb300 import spgemm as K
    th = _theta(2)
    g = _theta(3)
    p = torch.from_numpy(th.copy()).cuda()
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    K.kk_mlp_adam(torch.from_numpy(g).cuda(), p, m1, m2, 1, lr=0.01)
    # first Adam step (Kingma & Ba, Algorithm 1 with the step size folded into
    # lr_t = lr * sqrt(1 - b2^t) / (1 - b1^t)): m1 = (1-b1) g, m2 = (1-b2) g^2,
    # update lr_t * m1 / (sqrt(m2) + eps) = lr * g / (|g| + eps / sqrt(1 - b2))
    exp = th - 0.01 * g / (np.abs(g) + 1e-8 / np.sqrt(1 - 0.999))
    np.testing.assert_allclose(p.cpu().numpy(), exp, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("seed", range(3))
def test_features_and_classes_match_definitions(seed):
    torch = _torch()
    from paper_2103_11991_gb300 import spgemm as K
    A = I.random_sparse(300, 200, 0.05, seed, empty_rows=0.1)
    B = I.random_sparse(200, 250, 0.05, seed + 10, unsorted=seed == 1)
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM() as op:
        X = torch.empty((A.m, 8), dtype=torch.float32, device="cuda")
        K.kk_spgemm_row_features(op.h, dA, dB, X)
        rp, _ = op.symbolic(dA, dB)
        y = torch.empty(A.m, dtype=torch.int32, device="cuda")
        K.kk_capacity_classes(A.m, rp, y)
        torch.cuda.synchronize()
    np.testing.assert_allclose(X.cpu().numpy(), FE.row_features(A, B), rtol=2e-6, atol=2e-6)
    assert np.array_equal(y.cpu().numpy(), FE.capacity_class(oracle.symbolic(A, B)))


def _learned_run(A, B, params=None, quantile=0.95, refresh=False, **opts):
    torch = _torch()
    from paper_2103_11991_gb300 import spgemm as K
    dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
    with K.SpGEMM(**opts) as op:
        if params is not None:
            op.set_predictor(params, quantile)
        rp, nnz = op.learned_symbolic(dA, dB)
        ci, va = op.learned_numeric(dA, dB, rp, nnz)
        op.sync()
        st = op.stats()
        out = (rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy())
        if refresh:
            # same structure, new values: plain numeric reuses the learned symbolic result
            dA.vals.mul_(0.5)
            op.numeric(dA, dB, rp, nnz, ci, va)
            op.sync()
            out = out + (ci.cpu().numpy(), va.cpu().numpy())
    return out, st


def _always_class(c):
    th = np.zeros(M.NUM_PARAMS, dtype=np.float32)
    off_b3 = M.NUM_PARAMS - M.C
    th[off_b3 + c] = 10.0
    return th


@pytest.mark.parametrize("cache", [1, 0])
@pytest.mark.parametrize("which", ["stencil", "rmat", "random"])
@pytest.mark.parametrize("pred", ["none", "class0", "class4"])
def test_learned_parity(which, pred, cache):
    # cache = 0: the structure cache off, so that window rows take the window
    # one-pass (with it on they take the plain path)
    if which == "stencil":
        A = I.stencil_3d(14, 14, 14, 27, 26.0, -1.0)
        A.vals = I.uniform01(1, "lv", A.nnz) * 2 - 1
        B = A
    elif which == "rmat":
        A = I.rmat(11, 16, seed=9)
        B = A
    else:
        A = I.random_rows(2000, 1500, 3, 40, seed=2)
        B = I.random_rows(1500, 1800, 3, 40, seed=3)
    params = {"none": None, "class0": _always_class(0), "class4": _always_class(4)}[pred]
    (rp, ci, va, ci2, va2), st = _learned_run(A, B, params, quantile=0.0, refresh=True, structure_cache=cache)
    check_against_oracle(A, B, rp, ci, va)
    A2 = A.copy()
    A2.vals = A.vals * 0.5
    check_against_oracle(A2, B, rp, ci2, va2)
    if pred == "class0" and cache == 0:
        # every row with more than 16 outputs must have overflowed and been re-run
        cnt = np.diff(rp)
        assert st["overflow_rows"] >= int(((cnt > 16) & (cnt <= 256)).sum()) - st["heavy_rows"]
        assert st["overflow_rows"] > 0


def test_learned_edge_cases():
    for A, B in [(I.random_sparse(10, 8, 0.0, 1), I.random_sparse(8, 9, 0.5, 2)),
                 (I.random_sparse(1, 1, 1.0, 1), I.random_sparse(1, 1, 1.0, 2)),
                 (I.random_sparse(0, 5, 0.5, 1), I.random_sparse(5, 4, 0.5, 2))]:
        (rp, ci, va), _ = _learned_run(A, B)
        check_against_oracle(A, B, rp, ci, va)


def test_trained_predictor_gain():
    """Train on the reduced training families, then compare the learned form
    with the trained network against the same form without it (rows sized by
    the flop bound) on a held-out stencil: the network must send most rows
    through the one-pass with few overflows and a staging area close to
    nnz(C), where the flop bound sends them to the plain path."""
    torch = _torch()
    from paper_2103_11991_gb300 import learned as L
    from paper_2103_11991_gb300 import spgemm as K
    X, y = L.make_training_set(L.training_pairs(small=True))
    p0 = torch.empty(M.NUM_PARAMS, dtype=torch.float32, device="cuda")
    K.kk_mlp_init(p0, 7)
    g = torch.empty_like(p0)
    l0 = torch.empty(1, dtype=torch.float32, device="cuda")
    K.kk_mlp_loss_grad(X, y, p0, g, l0)
    params, loss = L.train_predictor(X, y, epochs=40)
    assert loss < 0.6 * float(l0.item())
    A = I.stencil_3d(20, 20, 20, 27, 26.0, -1.0)  # held out: grids 10, 16, 24 trained
    # the structure cache off: the stencil's window rows may take the one-pass
    (rp, ci, va), st = _learned_run(A, A, params, quantile=0.95, structure_cache=0)
    check_against_oracle(A, A, rp, ci, va, exact=True)
    (rp0, ci0, va0), st0 = _learned_run(A, A, None, structure_cache=0)
    nnz = int(rp[-1])
    assert st["onepass_rows"] >= 0.8 * A.m
    assert st["overflow_rows"] <= 0.05 * st["onepass_rows"]
    assert st["staging_entries"] <= 1.6 * nnz
    assert st0["onepass_rows"] < st["onepass_rows"]
