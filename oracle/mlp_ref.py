"""FP64 reference of the learned cost model — TEST INFRASTRUCTURE ONLY.

The paper's runtime picks a variant with performance models that it calls
machine-learning models, and expects better-trained models to pick better
(Sec. 3.2, results on matrix multiply; Sec. 5).  The cost model here is a
3-layer perceptron with ReLU:

    z1 = x W1^T + b1,  h1 = relu(z1)          (in -> H)
    z2 = h1 W2^T + b2, h2 = relu(z2)          (H -> H)
    y  = h2 W3^T + b3                          (H -> out)

trained on the masked mean squared error

    L = sum_{r,o} mask[r,o] * (y[r,o] - t[r,o])^2 / max(1, sum mask)

with Adam (Kingma & Ba 2015: first/second moment estimates with bias
correction).  Weight matrices are stored (out_features, in_features),
row-major.  This module is the plain statement of those formulas in float64,
with the chain rule written out layer by layer.
"""
import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_params(in_dim, hidden, out_dim, rng):
    """He-uniform weights, zero biases (float64)."""
    def lin(o, i):
        bound = np.sqrt(6.0 / i)
        return rng.uniform(-bound, bound, size=(o, i))
    return {"W1": lin(hidden, in_dim), "b1": np.zeros(hidden),
            "W2": lin(hidden, hidden), "b2": np.zeros(hidden),
            "W3": lin(out_dim, hidden), "b3": np.zeros(out_dim)}


def forward(p, x):
    """Returns (y, cache) for inputs x of shape (rows, in_dim)."""
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, z1, h1, z2, h2)


def loss(p, x, t, mask):
    y, _ = forward(p, x)
    den = max(1.0, float(np.sum(mask)))
    return float(np.sum(mask * (y - t) ** 2) / den)


def backward(p, x, t, mask):
    """Gradients of :func:`loss` with respect to every parameter."""
    y, (x, z1, h1, z2, h2) = forward(p, x)
    mask = np.asarray(mask, dtype=np.float64)
    den = max(1.0, float(np.sum(mask)))
    dy = 2.0 * mask * (y - t) / den
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place on p, m, v); ``step`` counts from 1."""
    for name in PARAM_NAMES:
        m[name] = beta1 * m[name] + (1.0 - beta1) * g[name]
        v[name] = beta2 * v[name] + (1.0 - beta2) * g[name] ** 2
        m_hat = m[name] / (1.0 - beta1 ** step)
        v_hat = v[name] / (1.0 - beta2 ** step)
        p[name] = p[name] - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p, m, v


def zeros_like(p):
    return {k: np.zeros_like(v) for k, v in p.items()}
