"""Pins for the thermal-stencil oracle (CPU only): the array form against the
cell-by-cell form, and both against closed forms of the heat equation."""
import numpy as np
import pytest

import workloads as W
from oracle import stencil_ref as S

PRM = dict(c=0.2, gx=0.5, gy=0.5, gz=0.01, amb=80.0)


def test_array_step_equals_cell_by_cell_step():
    for rows, cols, seed in [(1, 1, 1), (1, 7, 2), (6, 1, 3), (5, 7, 4), (9, 4, 5)]:
        T, P = W.stencil_inputs(rows, cols, seed)
        assert np.allclose(S.step(T, P, **PRM), S.step_loops(T, P, **PRM), rtol=0, atol=1e-12)


def test_steady_at_ambient_without_power():
    T = np.full((13, 17), 80.0)
    P = np.zeros((13, 17))
    assert np.array_equal(S.run(T, P, 25, **PRM), T)


def test_insulated_grid_conserves_heat():
    # no leak to ambient, no power: the discrete Laplacian with insulated
    # edges sums to zero, so the total heat stays put while it spreads
    T, _ = W.stencil_inputs(20, 31, seed=6)
    P = np.zeros_like(T)
    prm = dict(PRM, gz=0.0)
    out = S.run(T, P, 50, **prm)
    assert abs(out.sum() - T.astype(np.float64).sum()) <= 1e-9 * abs(T.sum())
    assert out.std() < T.std()                      # and it evens out


def test_uniform_power_integrates_linearly():
    # uniform temperature and power, no leak: no gradient, T grows by c*p per step
    T = np.full((8, 9), 90.0)
    P = np.full((8, 9), 3.0)
    out = S.run(T, P, 7, **dict(PRM, gz=0.0))
    assert np.allclose(out, 90.0 + 7 * PRM["c"] * 3.0, rtol=0, atol=1e-12)


def test_leak_decays_geometrically_to_ambient():
    # uniform excess temperature, no power: excess *= (1 - c*gz) per step
    T = np.full((6, 6), 100.0)
    out = S.run(T, np.zeros((6, 6)), 10, **PRM)
    assert np.allclose(out, 80.0 + 20.0 * (1 - PRM["c"] * PRM["gz"]) ** 10, rtol=0, atol=1e-12)


def test_one_row_is_the_1d_heat_equation():
    # a single row sees no row neighbours (the edge replicates the cell)
    T, P = W.stencil_inputs(1, 12, seed=7)
    t = T[0].astype(np.float64).tolist()
    p = P[0].astype(np.float64).tolist()
    for _ in range(3):
        t = [t[j] + PRM["c"] * (p[j] + ((t[j - 1] if j else t[j]) + (t[j + 1] if j < 11 else t[j])
                                       - 2 * t[j]) * PRM["gx"] + (PRM["amb"] - t[j]) * PRM["gz"])
             for j in range(12)]
    assert np.allclose(S.run(T, P, 3, **PRM)[0], t, rtol=0, atol=1e-12)


def test_mirror_symmetry():
    T, P = W.stencil_inputs(10, 16, seed=8)
    T = np.concatenate([T, T[:, ::-1]], axis=1)
    P = np.concatenate([P, P[:, ::-1]], axis=1)
    out = S.run(T, P, 9, **PRM)
    assert np.allclose(out, out[:, ::-1], rtol=0, atol=1e-12)


def test_zero_iterations_and_stability_rule():
    T, P = W.stencil_inputs(4, 5, seed=9)
    assert np.array_equal(S.run(T, P, 0, **PRM), T.astype(np.float64))
    assert S.stable(PRM["c"], PRM["gx"], PRM["gy"], PRM["gz"])
    assert not S.stable(0.3, 1.0, 1.0, 0.0)


def test_workload_inputs_are_seeded_and_shaped():
    T, P = W.stencil_inputs(64, 80, seed=10)
    T2, P2 = W.stencil_inputs(64, 80, seed=10)
    assert T.shape == P.shape == (64, 80) and T.dtype == np.float32
    assert np.array_equal(T, T2) and np.array_equal(P, P2)
    assert 80.0 <= T.min() and T.max() <= 100.0 and P.max() > 5.0
    ctxs = W.stencil_contexts(50, seed=11)
    assert all(64 <= r <= 8192 and 64 <= c <= 8192 and 1 <= i <= 1000 for r, c, i in ctxs)
