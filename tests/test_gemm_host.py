"""GEMM on host matrices through the library (compar_gemm_host), against the
FP64 oracle: row panels, beta != 0, pageable and page-locked memory, bf16
inputs, several calls in flight on one stream (alternating device buffer
sets), and the degenerate sizes."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_03543_b300 as cp
    c = cp.Context(0)
    yield c
    c.close()


def _pinned(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
    t.numpy()[...] = a
    return t


def test_pinned_panels_with_beta(ctx):
    import torch
    m, n, k = 2600, 384, 300           # 2 row panels of 1300
    A = W.uniform(m, k, seed=31); B = W.uniform(k, n, seed=32)
    C0 = W.uniform(m, n, seed=33)
    hA, hB, hC = _pinned(A), _pinned(B), _pinned(C0)
    ctx.set_scalars(1.5, -0.5)
    try:
        ctx.gemm_host(hA, hB, hC, tol=TOL)
        torch.cuda.synchronize()
    finally:
        ctx.set_scalars(1.0, 0.0)
    rows = W.tile_rows(m, seed=34)
    ref = oracle.gemm_rows(A, B, rows, alpha=1.5, beta=-0.5, C0=C0)
    assert N.rel_frobenius(hC.numpy()[rows], ref) <= TOL


def test_pageable_numpy_and_bf16(ctx):
    import paper_2311_03543_b300 as cp
    import torch
    m, n, k = 70, 90, 110
    A = W.uniform(m, k, seed=35); B = W.uniform(k, n, seed=36)
    C = np.full((m, n), np.nan, np.float32)
    ctx.gemm_host(A, B, C, tol=TOL)
    torch.cuda.synchronize()
    assert N.rel_frobenius(C, oracle.gemm(A, B)) <= TOL
    Ab = W.bf16_input(m, k, seed=37); Bb = W.bf16_input(k, n, seed=38)
    C2 = np.full((m, n), np.nan, np.float32)
    ctx.gemm_host(Ab, Bb, C2, tol=1e-3)
    torch.cuda.synchronize()
    ref = oracle.gemm(N.bf16_to_f32(Ab), N.bf16_to_f32(Bb))
    assert N.rel_frobenius(C2, ref) <= TOL
    assert ctx.check_device_error() == cp.OK


def test_calls_in_flight_alternate_buffers(ctx):
    import torch
    shapes = [(1100, 200, 130), (64, 64, 64), (1500, 96, 257), (33, 17, 9)]
    ins = []
    for i, (m, n, k) in enumerate(shapes):
        A = W.uniform(m, k, seed=40 + i); B = W.uniform(k, n, seed=50 + i)
        hC = _pinned(np.full((m, n), np.nan, np.float32))
        ins.append((A, B, _pinned(A), _pinned(B), hC))
    for A, B, hA, hB, hC in ins:       # no synchronisation between the calls
        ctx.gemm_host(hA, hB, hC, tol=TOL)
    torch.cuda.synchronize()
    for A, B, hA, hB, hC in ins:
        assert N.rel_frobenius(hC.numpy(), oracle.gemm(A, B)) <= TOL


def test_degenerate_sizes(ctx):
    import torch
    C = np.full((4, 5), 2.0, np.float32)
    ctx.gemm_host(np.zeros((4, 0), np.float32), np.zeros((0, 5), np.float32), C)
    torch.cuda.synchronize()
    assert np.all(C == 0.0)            # k == 0, beta == 0: C = 0
    ctx.gemm_host(np.zeros((0, 3), np.float32), np.zeros((3, 5), np.float32),
                  np.zeros((0, 5), np.float32))
