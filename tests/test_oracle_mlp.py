"""Pins for the FP64 MLP cost-model oracle (CPU only).

Gradients are checked against central finite differences of the loss; the
forward pass against a hand-set network with a closed-form output; Adam
against its known first-step behaviour.
"""
import numpy as np
import pytest

from oracle import mlp_ref as M


def _problem(seed=0, rows=9, in_dim=8, hidden=6, out_dim=4):
    g = np.random.default_rng(seed)
    p = M.init_params(in_dim, hidden, out_dim, g)
    for k in ("b1", "b2", "b3"):
        p[k] = g.normal(size=p[k].shape) * 0.1
    x = g.normal(size=(rows, in_dim))
    t = g.normal(size=(rows, out_dim))
    mask = (g.uniform(size=(rows, out_dim)) < 0.7).astype(np.float64)
    return p, x, t, mask


def test_gradients_match_finite_differences():
    p, x, t, mask = _problem()
    g = M.backward(p, x, t, mask)
    h = 1e-6
    for name in M.PARAM_NAMES:
        num = np.zeros_like(p[name])
        it = np.nditer(p[name], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[name][idx]
            p[name][idx] = old + h; lp = M.loss(p, x, t, mask)
            p[name][idx] = old - h; lm = M.loss(p, x, t, mask)
            p[name][idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g[name], num, rtol=1e-5, atol=1e-8), name


def test_hand_set_network_closed_form():
    # in=2, hidden=1, out=1: y = w3*relu(w2*relu(w1.x + b1) + b2) + b3
    p = {"W1": np.array([[2.0, -1.0]]), "b1": np.array([0.5]),
         "W2": np.array([[3.0]]), "b2": np.array([-1.0]),
         "W3": np.array([[-2.0]]), "b3": np.array([4.0])}
    x = np.array([[1.0, 1.0], [0.0, 3.0]])
    y, _ = M.forward(p, x)
    # row 0: z1 = 2-1+0.5 = 1.5 -> h1 1.5; z2 = 4.5-1 = 3.5; y = -7+4 = -3
    # row 1: z1 = -3+0.5 = -2.5 -> h1 0; z2 = -1 -> h2 0; y = 4
    assert np.array_equal(y, np.array([[-3.0], [4.0]]))


def test_masked_entries_do_not_contribute():
    p, x, t, mask = _problem(seed=3)
    t2 = t.copy(); t2[mask == 0] += 1e3
    assert M.loss(p, x, t, mask) == pytest.approx(M.loss(p, x, t2, mask), rel=0, abs=0)


def test_adam_first_step_is_lr_times_sign():
    p, x, t, mask = _problem(seed=4)
    g = M.backward(p, x, t, mask)
    p0 = {k: v.copy() for k, v in p.items()}
    lr = 1e-3
    M.adam_step(p, g, M.zeros_like(p), M.zeros_like(p), step=1, lr=lr, eps=1e-30)
    for k in M.PARAM_NAMES:
        nz = g[k] != 0
        assert np.allclose((p[k] - p0[k])[nz], -lr * np.sign(g[k][nz]), rtol=1e-12)
        assert np.array_equal(p[k][~nz], p0[k][~nz])


def test_training_reduces_loss():
    p, x, t, mask = _problem(seed=5, rows=64)
    m, v = M.zeros_like(p), M.zeros_like(p)
    l0 = M.loss(p, x, t, mask)
    for step in range(1, 301):
        M.adam_step(p, M.backward(p, x, t, mask), m, v, step, lr=1e-2)
    assert M.loss(p, x, t, mask) < 0.5 * l0
