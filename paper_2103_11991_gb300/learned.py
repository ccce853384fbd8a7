"""Learned row-capacity predictor: training data, GPU training, and the
learned (speculative one-pass) SpGEMM form.

Training data come from the symbolic phase itself: for every row of a training
product the GPU computes the row features (``kk_spgemm_row_features``) and the
symbolic phase's count gives the capacity-class label
(``kk_capacity_classes``).  The training matrices are seeded synthetic
families disjoint from the evaluation inputs: R-MAT graphs at scales 14-18
(seeds 1000+), 2D 5/9-point and 3D 7/27-point stencils on grids other than the
evaluation grids, and uniform random rows.  The network is trained by the
library's own forward/backward/Adam kernels (``kk_mlp_train``).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import inputs as I
from . import spgemm as K

PKG = os.path.dirname(os.path.abspath(__file__))
TUNED = os.path.join(PKG, "tuned")


def training_pairs(small: bool = False):
    """(A, B) training products.  ``small`` keeps a reduced set for tests."""
    pairs = []
    rscales = [11, 12] if small else [14, 15, 16, 17, 18]
    for t, s in enumerate(rscales):
        A = I.rmat(s, 16, 0.57, 0.19, 0.19, seed=1000 + t)
        pairs.append((A, A))
    grids3 = [10, 16, 24] if small else [12, 18, 24, 32, 40, 48, 56]
    for g in grids3:
        A = I.stencil_3d(g, g, g, 27, 26.0, -1.0)
        pairs.append((A, A))
        A7 = I.stencil_3d(g, g, g, 7, 6.0, -1.0)
        pairs.append((A7, A7))
    grids2 = [40] if small else [48, 96, 160, 256]
    for g in grids2:
        for pts in (5, 9):
            A = I.stencil_2d(g, g, pts, 4.0 if pts == 5 else 8.0, -1.0)
            pairs.append((A, A))
    for t in range(1 if small else 4):
        n = 3000 if small else 20000
        A = I.random_rows(n, n, 3, 40, seed=1100 + t, purpose="train.A")
        B = I.random_rows(n, n, 3, 40, seed=1200 + t, purpose="train.B")
        pairs.append((A, B))
    return pairs


def make_training_set(pairs):
    """Device tensors X (float32[N, 8]) and y (int32[N]) from the given products."""
    import torch
    Xs, ys = [], []
    with K.SpGEMM() as op:
        for A, B in pairs:
            dA, dB = K.DeviceCSR.from_host(A), K.DeviceCSR.from_host(B)
            X = torch.empty((A.m, K.MLP_FEATURES), dtype=torch.float32, device="cuda")
            K.kk_spgemm_row_features(op.h, dA, dB, X)
            rp, _ = op.symbolic(dA, dB)
            y = torch.empty(A.m, dtype=torch.int32, device="cuda")
            K.kk_capacity_classes(A.m, rp, y)
            keep = (rp[1:] - rp[:-1]) > 0  # rows with products only
            Xs.append(X[keep])
            ys.append(y[keep])
    return torch.cat(Xs), torch.cat(ys)


def train_predictor(X, y, epochs: int = 30, batch: int = 1024, lr: float = 3e-3, seed: int = 7):
    """Train on the GPU; returns (params as numpy float32, final mean loss)."""
    import torch
    params = torch.empty(K.MLP_NUM_PARAMS, dtype=torch.float32, device="cuda")
    K.kk_mlp_init(params, seed)
    loss = K.kk_mlp_train(X, y, params, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return params.cpu().numpy(), loss


def save_predictor(params, path=None, meta=None):
    import torch
    os.makedirs(TUNED, exist_ok=True)
    if path is None:
        name = torch.cuda.get_device_name().replace(" ", "_")
        path = os.path.join(TUNED, f"predictor_{name}.json")
    with open(path, "w") as f:
        json.dump({"params": [float(v) for v in params], "meta": meta or {}}, f)
    return path


def load_predictor(path=None):
    import torch
    if path is None:
        name = torch.cuda.get_device_name().replace(" ", "_")
        path = os.path.join(TUNED, f"predictor_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return np.asarray(json.load(f)["params"], dtype=np.float32)


def get_predictor(small: bool = False, epochs: int = 30):
    """Stored predictor for this device, else train one (and store it)."""
    p = load_predictor()
    if p is not None:
        return p
    X, y = make_training_set(training_pairs(small))
    params, loss = train_predictor(X, y, epochs=epochs)
    save_predictor(params, meta={"samples": int(X.shape[0]), "final_loss": loss, "epochs": epochs})
    return params
