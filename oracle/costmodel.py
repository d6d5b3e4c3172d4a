"""FP64 reference of the schedule cost-model MLP (oracle; test infrastructure only).

Network: 16 inputs -> 64 (ReLU) -> 64 (ReLU) -> 1, parameters packed as
W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3.  Loss: mean over samples
of 0.5 * (f(x) - t)^2.  The backward pass is the chain rule written out layer
by layer; it is pinned in the tests by central finite differences.
"""
import numpy as np

IN, H = 16, 64
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(p, X):
    """Predictions and the intermediate values the backward pass needs."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ w["W1"].T + w["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w["W2"].T + w["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w["W3"] + w["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(p, X, t):
    y, _ = forward(p, X)
    r = y - np.asarray(t, dtype=np.float64)
    return 0.5 * float(np.mean(r * r))


def loss_grad(p, X, t):
    """(loss, gradient) of the mean squared error, by the chain rule."""
    w = unpack(p)
    y, (X, z1, h1, z2, h2) = forward(p, X)
    n = X.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    dy = r / n
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    d2 = np.outer(dy, w["W3"]) * (z2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ w["W2"]) * (z1 > 0)
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(axis=0)
    return 0.5 * float(np.mean(r * r)), pack(g)


def init(seed=0):
    """He-style random initial parameters (float32), seeded."""
    rng = np.random.default_rng(seed)
    d = {"W1": rng.normal(0, np.sqrt(2.0 / IN), (H, IN)), "b1": np.zeros(H),
         "W2": rng.normal(0, np.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
         "W3": rng.normal(0, np.sqrt(1.0 / H), H), "b3": np.zeros(1)}
    return pack(d).astype(np.float32)
