"""The library's FP64 residual check (the error labels of recorded runs)
against the relative Frobenius error computed by the FP64 oracle on the same
data (all rows, so both sides see the same sample)."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_03543_b300 as cp
    c = cp.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("variant", [1, 2, 3, 5])
def test_residual_matches_oracle_f32(ctx, variant):
    import torch
    m, n, k = 96, 130, 200
    A = W.uniform(m, k, seed=1); B = W.uniform(k, n, seed=2)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty((m, n), device="cuda")
    ctx.force_variant(variant)
    try:
        ctx.gemm(dA, dB, C)
    finally:
        ctx.force_variant(None)
    got = ctx.residual_check(dA, dB, C, nrows=m)
    want = N.rel_frobenius(C.cpu().numpy(), oracle.gemm(A, B))
    assert got == pytest.approx(want, rel=1e-6, abs=1e-12)


def test_residual_bf16_and_fp8_with_scales(ctx):
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev
    m, n, k = 64, 72, 48
    Ab, Bb = W.bf16_input(m, k, 3), W.bf16_input(k, n, 4)
    C = torch.from_numpy(W.uniform(m, n, seed=5)).cuda()
    got = ctx.residual_check(dev(Ab), dev(Bb), C, alpha=2.0, nrows=m, dtype=cp.BF16)
    ref = 2.0 * oracle.gemm(N.bf16_to_f32(Ab), N.bf16_to_f32(Bb))
    assert got == pytest.approx(N.rel_frobenius(C.cpu().numpy(), ref), rel=1e-6)
    Aq, Bq = W.fp8_input(m, k, 6), W.fp8_input(k, n, 7)
    ctx.set_fp8_scales(0.5, 4.0)
    try:
        got = ctx.residual_check(dev(Aq), dev(Bq), C, nrows=m, dtype=cp.F8E4M3)
    finally:
        ctx.set_fp8_scales(1.0, 1.0)
    ref = 2.0 * oracle.gemm(N.e4m3_to_f64(Aq), N.e4m3_to_f64(Bq))
    assert got == pytest.approx(N.rel_frobenius(C.cpu().numpy(), ref), rel=1e-6)


def test_residual_sampled_rows_bounded_by_full(ctx):
    import torch
    m, n, k = 512, 64, 64
    A = W.uniform(m, k, seed=8); B = W.uniform(k, n, seed=9)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.from_numpy((oracle.gemm(A, B) * (1 + 1e-3)).astype(np.float32)).cuda()
    # a uniform relative perturbation gives the same error on any row sample
    assert ctx.residual_check(dA, dB, C, nrows=16, seed=3) == pytest.approx(1e-3, rel=1e-3)
