"""Float64 reference of the row-capacity MLP (features -> 32 -> 32 -> classes,
ReLU, softmax cross-entropy).  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Parameters are one flat vector in the order W1 (F x H1, row-major), b1 (H1),
W2 (H1 x H2), b2 (H2), W3 (H2 x C), b3 (C).  The loss is the mean over the
batch of -log softmax(z)[y].
"""
import numpy as np

F, H1, H2, C = 8, 32, 32, 16
SHAPES = [(F, H1), (H1,), (H1, H2), (H2,), (H2, C), (C,)]
NUM_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(theta[o:o + k].reshape(s))
        o += k
    return out


def forward(theta, X):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    a1 = X @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ W3 + b3
    return a1, h1, a2, h2, z


def loss(theta, X, y):
    *_, z = forward(theta, X)
    zm = z - z.max(axis=1, keepdims=True)
    logp = zm - np.log(np.exp(zm).sum(axis=1, keepdims=True))
    return float(-logp[np.arange(len(y)), y].mean())


def grad(theta, X, y):
    """Gradient of the mean loss with respect to the flat parameter vector."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    a1, h1, a2, h2, z = forward(theta, X)
    zm = z - z.max(axis=1, keepdims=True)
    p = np.exp(zm)
    p /= p.sum(axis=1, keepdims=True)
    N = len(y)
    dz = p.copy()
    dz[np.arange(N), y] -= 1.0
    dz /= N
    gW3 = h2.T @ dz
    gb3 = dz.sum(axis=0)
    dh2 = (dz @ W3.T) * (a2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    gW1 = X.T @ dh1
    gb1 = dh1.sum(axis=0)
    return np.concatenate([g.reshape(-1) for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def predict_class(theta, X, quantile: float = 0.0):
    """argmax class, or (quantile > 0) the smallest class whose cumulative
    softmax probability reaches the quantile."""
    *_, z = forward(theta, X)
    if quantile <= 0.0:
        return z.argmax(axis=1)
    zm = z - z.max(axis=1, keepdims=True)
    p = np.exp(zm)
    p /= p.sum(axis=1, keepdims=True)
    cum = np.cumsum(p, axis=1)
    return (cum < quantile).sum(axis=1).clip(max=C - 1)
