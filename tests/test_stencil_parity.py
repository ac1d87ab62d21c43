"""Parity of the thermal-stencil variants with the FP64 oracle (GPU, through
the C ABI).

Tolerance: relative Frobenius error <= max(1e-6, 4 * iters * 2^-24): each
step rounds a handful of float32 operations on values of the size of T.
All variants evaluate the same rounded operations, so their grids must be
bit-identical, which is checked as well.  At the benchmark's full size
(8192 x 8192, 100 steps) sampled windows are checked against the oracle run
on the window plus a 100-cell margin (a cell depends only on cells within
`iters` of it, and windows touching the grid edge keep the true edge)."""
import numpy as np
import pytest

import workloads as W
from oracle import numerics as N
from oracle import stencil_ref as S

pytestmark = pytest.mark.gpu

PRM = W.STENCIL_PARAMS


def _tol(iters):
    return max(1e-6, 4 * iters * 2.0 ** -24)


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_03543_b300 as cp
    c = cp.Context(0)
    yield c
    c.close()


def _run(ctx, v, T0, P, iters):
    import torch
    import paper_2311_03543_b300 as cp
    dT, dP = torch.from_numpy(T0).cuda(), torch.from_numpy(P).cuda()
    out = torch.full_like(dT, float("nan"))
    ctx.stencil_force_variant(v)
    try:
        ctx.stencil(dT, dP, out, iters, cp.Context.stencil_params(**PRM))
        torch.cuda.synchronize()
    finally:
        ctx.stencil_force_variant(None)
    assert ctx.check_device_error() == cp.OK
    assert ctx.stencil_last_variant() == v
    # the inputs are not written
    assert np.array_equal(dT.cpu().numpy(), T0) and np.array_equal(dP.cpu().numpy(), P)
    return out.cpu().numpy()


SHAPES = [(1, 1, 3), (1, 36, 5), (50, 1, 5), (64, 64, 8), (65, 132, 9), (130, 200, 17),
          (257, 300, 20), (96, 64, 1), (80, 76, 0), (64, 112, 8), (65, 113, 9), (64, 224, 16),
          (130, 225, 17), (81, 240, 12), (200, 128, 7)]


@pytest.mark.parametrize("rows,cols,iters", SHAPES)
def test_variants_match_oracle_and_each_other(ctx, rows, cols, iters):
    import paper_2311_03543_b300 as cp
    T0, P = W.stencil_inputs(rows, cols, seed=rows + 7 * cols)
    ref = S.run(T0, P, iters, **PRM)
    outs = {}
    for v in range(cp.NUM_STENCIL_VARIANTS):
        if not ctx.stencil_supported(v, rows, cols):
            continue
        outs[v] = _run(ctx, v, T0, P, iters)
        assert N.rel_frobenius(outs[v], ref) <= _tol(iters), (v, N.rel_frobenius(outs[v], ref))
    assert cp.S_NAIVE in outs and cp.S_TILED in outs
    first = next(iter(outs.values()))
    for v, o in outs.items():
        assert np.array_equal(o, first), v


def test_selected_variant_and_insulated_conservation(ctx):
    # no power and no leak: the total heat of the grid stays (up to float32
    # rounding of the sum) while it spreads
    import torch
    import paper_2311_03543_b300 as cp
    rows, cols, iters = 300, 400, 40
    T0, _ = W.stencil_inputs(rows, cols, seed=3)
    prm = cp.Context.stencil_params(**dict(PRM, gz=0.0))
    dT = torch.from_numpy(T0).cuda()
    dP = torch.zeros_like(dT)
    out = torch.empty_like(dT)
    ctx.stencil(dT, dP, out, iters, prm)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    assert abs(got.sum() - T0.astype(np.float64).sum()) <= 1e-5 * T0.sum()
    ref = S.run(T0, np.zeros_like(T0), iters, **dict(PRM, gz=0.0))
    assert N.rel_frobenius(got, ref) <= _tol(iters)


def test_full_size_sampled_windows(ctx):
    import torch
    import paper_2311_03543_b300 as cp
    rows, cols, iters = W.STENCIL_HEADLINE
    T0, P = W.stencil_inputs(rows, cols, seed=21)
    dT, dP = torch.from_numpy(T0).cuda(), torch.from_numpy(P).cuda()
    outs = {}
    for v in (cp.S_TILED, cp.S_TMA, cp.S_NAIVE):
        out = torch.empty_like(dT)
        ctx.stencil_force_variant(v)
        try:
            ctx.stencil(dT, dP, out, iters, cp.Context.stencil_params(**PRM))
        finally:
            ctx.stencil_force_variant(None)
        torch.cuda.synchronize()
        outs[v] = out
    assert torch.equal(outs[cp.S_TILED], outs[cp.S_NAIVE])
    assert torch.equal(outs[cp.S_TMA], outs[cp.S_NAIVE])
    got = outs[cp.S_TILED].cpu().numpy()
    rng = np.random.default_rng(22)
    centres = [(0, 0), (rows - 1, cols - 1), (0, cols // 2)] + \
              [tuple(int(x) for x in rng.integers(0, [rows, cols])) for _ in range(3)]
    w = 8
    for (r, c) in centres:
        r0, r1 = max(0, r - w), min(rows, r + w + 1)
        c0, c1 = max(0, c - w), min(cols, c + w + 1)
        R0, R1 = max(0, r0 - iters), min(rows, r1 + iters)
        C0, C1 = max(0, c0 - iters), min(cols, c1 + iters)
        ref = S.run(T0[R0:R1, C0:C1], P[R0:R1, C0:C1], iters, **PRM)
        ref = ref[r0 - R0:r1 - R0, c0 - C0:c1 - C0]
        assert N.rel_frobenius(got[r0:r1, c0:c1], ref) <= _tol(iters), (r, c)


def test_bad_arguments_are_refused(ctx):
    import ctypes
    import torch
    import paper_2311_03543_b300 as cp
    g = torch.zeros((3, 8, 8), device="cuda")          # three 8 x 8 grids
    t_in, p_in, t_out = (g[i].data_ptr() for i in range(3))
    prm = cp.Context.stencil_params(**PRM)
    bad = cp.Context.stencil_params(float("nan"), 0.5, 0.5, 0.0, 80.0)
    assert cp.compar_stencil(ctx.handle, 8, 8, 1, ctypes.byref(bad), t_in, p_in, t_out,
                             None) == cp.ERR_INVALID
    # T_out overlapping T_in (shifted by one cell)
    assert cp.compar_stencil(ctx.handle, 8, 8, 1, ctypes.byref(prm), t_in, p_in, t_in + 4,
                             None) == cp.ERR_INVALID
    assert cp.compar_stencil(ctx.handle, 8, 8, -1, ctypes.byref(prm), t_in, p_in, t_out,
                             None) == cp.ERR_INVALID
    assert ctx.stencil_supported(cp.S_TMA, 8, 6) is False    # rows not 16-byte multiples
