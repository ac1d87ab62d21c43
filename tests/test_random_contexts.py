"""Seeded random calls against the FP64 oracle (GPU, through the C ABI).

Each context draws its shape log-uniformly in [1, 640] per dimension (up to
five 128-row tiles with a ragged tail), its input type (float32, bf16 or
E4M3), alpha and beta.  C is filled with NaN when beta == 0, because C is then
not read.  Every variant the library accepts for the context is forced in
turn and checked element by element:

    |C - C_ref| <= bound(v, k) * (|alpha| |A||B| + |beta| |C0|)

with the worst-case bounds of `gpu_util.elem_bound`.  C_ref is the oracle
evaluated on the values the variant multiplies: the inputs as given, or the
oracle's own bf16 rounding or E4M3 quantisation of float32 inputs.  The
selector's own pick at a random tolerance must stay within twice that
tolerance of the oracle on the given values.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu

CONTEXTS_PER_BLOCK = 10
BLOCKS = 8


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_03543_b300 as cp
    c = cp.Context(0)
    yield c
    c.close()


def _draw(i):
    """Context i: (dtype, m, n, k, alpha, beta, tol, seed)."""
    import paper_2311_03543_b300 as cp
    g = W.rng(7700 + i)
    r = g.random()
    dt = cp.F32 if r < 0.6 else (cp.BF16 if r < 0.85 else cp.F8E4M3)
    m, n, k = (int(round(np.exp(g.uniform(0.0, np.log(640.0))))) for _ in range(3))
    alpha = 1.0 if g.random() < 0.5 else float(np.float32(g.uniform(-2, 2)))
    beta = [0.0, 0.0, 1.0, float(np.float32(g.uniform(-2, 2)))][int(g.integers(0, 4))]
    tol = [1e-6, 1e-5, 1e-3, 1e-1][int(g.integers(0, 4))]
    return dt, m, n, k, alpha, beta, tol, 7700 + i


def _inputs(dt, m, n, k, seed):
    """(A, B) as passed to the library and their exact values in float64."""
    import paper_2311_03543_b300 as cp
    if dt == cp.F32:
        A, B = W.uniform(m, k, seed=seed), W.uniform(k, n, seed=seed + 50000)
        return A, B, A.astype(np.float64), B.astype(np.float64)
    if dt == cp.BF16:
        A, B = W.bf16_input(m, k, seed=seed), W.bf16_input(k, n, seed=seed + 50000)
        return A, B, N.bf16_to_f32(A).astype(np.float64), N.bf16_to_f32(B).astype(np.float64)
    A, B = W.fp8_input(m, k, seed=seed), W.fp8_input(k, n, seed=seed + 50000)
    return A, B, N.e4m3_to_f64(A), N.e4m3_to_f64(B)


def _call(ctx, v, A, B, C0, dt, alpha, beta, tol=0.0):
    from gpu_util import dev, empty_c, host
    import paper_2311_03543_b300 as cp
    m, n = A.shape[0], B.shape[1]
    C = empty_c(m, n) if beta == 0.0 else dev(C0)
    ctx.set_scalars(alpha, beta)
    ctx.force_variant(v)
    try:
        ctx.gemm(dev(A), dev(B), C, tol=tol, dtype=dt)
        out = host(C)
        used = ctx.last_variant()
    finally:
        ctx.force_variant(None)
        ctx.set_scalars(1.0, 0.0)
    assert ctx.check_device_error() == cp.OK
    return out, used


@pytest.mark.parametrize("block", range(BLOCKS))
def test_random_contexts_every_variant(ctx, block):
    import paper_2311_03543_b300 as cp
    from gpu_util import assert_elementwise, elem_bound
    checked = 0
    for i in range(block * CONTEXTS_PER_BLOCK, (block + 1) * CONTEXTS_PER_BLOCK):
        dt, m, n, k, alpha, beta, tol, seed = _draw(i)
        A, B, Ax, Bx = _inputs(dt, m, n, k, seed)
        C0 = W.uniform(m, n, seed=seed + 90000)
        exact = oracle.gemm(Ax, Bx)
        absp = oracle.gemm(np.abs(Ax), np.abs(Bx))
        for v in (0, 1, 2, 3, 4, 5, 7, 8, 9):
            if not ctx.supported(v, m, n, k, dt):
                continue
            got, _ = _call(ctx, v, A, B, C0, dt, alpha, beta)
            assert np.isfinite(got).all(), (i, v, "C read with beta == 0 or a bad value")
            prod, scale = exact, absp
            if dt == cp.F32 and v == 3:      # the kernel multiplies the bf16 roundings
                Ar, Br = N.bf16_round(A), N.bf16_round(B)
                prod, scale = oracle.gemm(Ar, Br), oracle.gemm(np.abs(Ar), np.abs(Br))
            elif dt == cp.F32 and v == 4:    # ... or the E4M3 codes with per-tensor scales
                qa, sa = N.fp8_quantize(A)
                qb, sb = N.fp8_quantize(B)
                Aq, Bq = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb)
                d = float(sa) * float(sb)
                prod, scale = oracle.gemm(Aq, Bq) / d, oracle.gemm(np.abs(Aq), np.abs(Bq)) / d
            ref = alpha * prod + beta * C0
            lim = abs(alpha) * scale + abs(beta) * np.abs(C0.astype(np.float64))
            try:
                assert_elementwise(got, ref, lim, elem_bound(v, k))
            except AssertionError as e:
                raise AssertionError(f"context {i} (dtype {dt}, {m}x{n}x{k}, alpha {alpha}, "
                                     f"beta {beta}) variant {v}: {e}") from None
            checked += 1
        # the selector's own pick, at the context's tolerance
        got, used = _call(ctx, None, A, B, C0, dt, alpha, beta, tol=tol)
        assert np.isfinite(got).all()
        err = N.rel_frobenius(got, alpha * exact + beta * C0)
        assert err <= 2 * tol, (i, used, tol, err)
    assert checked >= CONTEXTS_PER_BLOCK
