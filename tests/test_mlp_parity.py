"""Parity of the learned cost model's CUDA kernels with the FP64 oracle
(oracle/mlp_ref.py), through the C ABI: forward pass, gradients of the
masked-MSE loss, Adam updates, a multi-step training trajectory, and the
hand-set closed-form network.

Tolerances: forward outputs and Adam parameters agree to 1e-5 relative (FP32
arithmetic, ~100-term dot products); gradients to 1e-4 relative to the
largest gradient of each tensor (sums over a 128-row batch)."""
import numpy as np
import pytest

import paper_2311_03543_b300 as cp
from oracle import mlp_ref as M

pytestmark = pytest.mark.gpu

IN, H, OUT = 8, 64, 2 * cp.NUM_VARIANTS


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_03543_b300 as cp
    c = cp.Context(0)
    yield c
    c.close()


def _flat(p):
    return np.concatenate([p[k].ravel() for k in M.PARAM_NAMES]).astype(np.float32)


def _unflat(v):
    shapes = {"W1": (H, IN), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (OUT, H), "b3": (OUT,)}
    out, o = {}, 0
    for k in M.PARAM_NAMES:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


def _problem(seed, rows=300):
    g = np.random.default_rng(seed)
    p = M.init_params(IN, H, OUT, g)
    for k in ("b1", "b2", "b3"):
        p[k] = g.normal(size=p[k].shape) * 0.1
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    X = g.normal(size=(rows, IN)).astype(np.float32)
    T = g.normal(size=(rows, OUT)).astype(np.float32)
    mask = (g.uniform(size=(rows, OUT)) < 0.3).astype(np.float32)
    return p, X, T, mask


def test_param_count():
    import paper_2311_03543_b300 as cp
    assert cp.compar_mlp_param_count() == IN * H + H + H * H + H + OUT * H + OUT


def test_forward_matches_oracle(ctx):
    p, X, _, _ = _problem(1)
    p2, _, _, _ = _problem(2)
    Y = ctx.mlp_forward(np.stack([_flat(p), _flat(p2)]), X)
    for member, pp in enumerate((p, p2)):
        ref, _ = M.forward(pp, X.astype(np.float64))
        assert np.max(np.abs(Y[member] - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


def test_forward_hand_set_closed_form(ctx):
    # weights that make the network y_o = 2*relu(3*relu(x0 - x1)) for output 0
    p = {k: np.zeros(s) for k, s in
         {"W1": (H, IN), "b1": (H,), "W2": (H, H), "b2": (H,), "W3": (OUT, H), "b3": (OUT,)}.items()}
    p["W1"][0, 0], p["W1"][0, 1] = 1.0, -1.0
    p["W2"][0, 0] = 3.0
    p["W3"][0, 0] = 2.0
    p["b3"][5] = 0.25
    X = np.zeros((3, IN), np.float32)
    X[0, :2] = (2.0, 0.5)      # 2*3*1.5 = 9
    X[1, :2] = (0.5, 2.0)      # relu cuts -> 0
    X[2, :2] = (1.0, 0.0)      # 6
    Y = ctx.mlp_forward(_flat(p)[None], X)[0]
    assert np.array_equal(Y[:, 0], np.array([9.0, 0.0, 6.0], np.float32))
    assert np.all(Y[:, 5] == 0.25)


@pytest.mark.parametrize("batch", [128, 37])
def test_gradients_match_oracle(ctx, batch):
    p, X, T, mask = _problem(3)
    idx = np.random.default_rng(4).choice(len(X), size=batch, replace=False)
    g_dev, loss = ctx.mlp_train_steps(_flat(p)[None], X, T, mask, idx[None, None, :],
                                      grads_only=True)
    g_ref = M.backward(p, X[idx].astype(np.float64), T[idx].astype(np.float64), mask[idx])
    got = _unflat(g_dev[0])
    for k in M.PARAM_NAMES:
        scale = max(np.max(np.abs(g_ref[k])), 1e-12)
        assert np.max(np.abs(got[k] - g_ref[k])) <= 1e-4 * scale, k
    ref_loss = M.loss(p, X[idx].astype(np.float64), T[idx].astype(np.float64), mask[idx])
    assert loss[0, 0] == pytest.approx(ref_loss, rel=1e-5)


def test_adam_steps_match_oracle(ctx):
    p, X, T, mask = _problem(5)
    rng = np.random.default_rng(6)
    steps, batch, lr = 25, 64, 2e-3
    idx = rng.integers(0, len(X), size=(1, steps, batch))
    new_p, m, v, loss = ctx.mlp_train_steps(_flat(p)[None], X, T, mask, idx, lr=lr)
    ref = {k: val.copy() for k, val in p.items()}
    rm, rv = M.zeros_like(ref), M.zeros_like(ref)
    ref_losses = []
    for s in range(steps):
        sel = idx[0, s]
        Xb, Tb, Mb = X[sel].astype(np.float64), T[sel].astype(np.float64), mask[sel]
        ref_losses.append(M.loss(ref, Xb, Tb, Mb))
        M.adam_step(ref, M.backward(ref, Xb, Tb, Mb), rm, rv, s + 1, lr)
    got = _unflat(new_p[0])
    diffs = np.concatenate([np.abs(got[k] - ref[k]).ravel() for k in M.PARAM_NAMES])
    # Each Adam step moves a parameter by about lr.  FP32 and FP64 runs agree
    # to a small fraction of one step, except where a gradient is so close to
    # zero that rounding decides its sign (Adam normalises it to +-lr).
    assert np.quantile(diffs, 0.99) <= 0.05 * lr
    assert diffs.max() <= 2 * lr * steps
    assert np.allclose(loss[0], ref_losses, rtol=1e-4)


def test_training_reduces_loss(ctx):
    p, X, T, mask = _problem(7, rows=512)
    T = (X @ np.random.default_rng(8).normal(size=(IN, OUT))).astype(np.float32)  # learnable
    idx = np.random.default_rng(9).integers(0, len(X), size=(2, 400, 128))
    params = np.stack([_flat(p), _flat(_problem(10)[0])])
    _, _, _, loss = ctx.mlp_train_steps(params, X, T, mask, idx, lr=3e-3)
    assert np.all(loss[:, -20:].mean(axis=1) < 0.2 * loss[:, :20].mean(axis=1))


def test_invalid_batch_index_is_refused(ctx):
    import ctypes
    import paper_2311_03543_b300 as cp
    p, X, T, mask = _problem(11, rows=10)
    params = _flat(p)[None].copy()
    with pytest.raises(ValueError):       # the binding checks before the call
        ctx.mlp_train_steps(params, X, T, mask, np.array([[[0, 10]]]), grads_only=True)
    # and the C ABI refuses the out-of-range row by itself
    f = lambda a: np.ascontiguousarray(a, np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    idx = np.array([[[0, 10]]], np.int32)
    g, loss = np.zeros_like(params), np.zeros((1, 1), np.float32)
    Xc, Tc, Mc = (np.ascontiguousarray(a, np.float32) for a in (X, T, mask))
    rc = cp.compar_mlp_train_steps(ctx.handle, f(params), None, None, 1, f(Xc), f(Tc), f(Mc), 10,
                                   idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1, 2,
                                   1e-3, 1, f(g), f(loss))
    assert rc == cp.ERR_INVALID
