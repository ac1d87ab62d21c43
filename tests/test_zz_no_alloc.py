"""The allocation-free SIMT entry point (compar_gemm_simt_noalloc).

It exists for callers that cannot allocate device memory where they need a
GEMM (a host framework that owns all device memory, a latency-critical path,
a plug-in without an allocator).  It must match the FP64 oracle
within the FP32 tolerance and give the same result as the regular entry
point running the same SIMT variant, call after call, although every call
reuses one fixed scratch array inside the library.  This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(A, B, C, alpha=1.0, beta=0.0):
    import paper_2311_03543_b300 as cp
    m, k = A.shape
    n = B.shape[1]
    return cp.compar_gemm_simt_noalloc(m, n, k, alpha, A.data_ptr(), B.data_ptr(), beta,
                                       C.data_ptr(), _stream())


def _regular(ctx, A, B, alpha=1.0, beta=0.0, C0=None):
    import torch
    import paper_2311_03543_b300 as cp
    C = C0.clone() if C0 is not None else torch.empty((A.shape[0], B.shape[1]), device="cuda")
    ctx.set_scalars(alpha, beta)
    ctx.force_variant(cp.V_SIMT)
    try:
        ctx.gemm(A, B, C)
    finally:
        ctx.force_variant(None)
        ctx.set_scalars(1.0, 0.0)
    return C


# (16, 4096, 4096) and (64, 512, 2048) take the split-K plan that uses the
# scratch array; (300, 200, 1000) does not.
@pytest.mark.parametrize("m,n,k", [(16, 4096, 4096), (64, 512, 2048), (300, 200, 1000)])
def test_noalloc_matches_regular_entry_point_twice(m, n, k):
    import torch
    import paper_2311_03543_b300 as cp
    with cp.Context(0) as ctx:
        for call in range(2):                       # two calls in a row, fresh data each
            A = torch.from_numpy(W.uniform(m, k, seed=10 * call + 1)).cuda()
            B = torch.from_numpy(W.uniform(k, n, seed=10 * call + 2)).cuda()
            C0 = torch.from_numpy(W.uniform(m, n, seed=10 * call + 3)).cuda()
            C = C0.clone()
            assert _noalloc(A, B, C, alpha=1.5, beta=-0.5) == cp.OK
            ref = _regular(ctx, A, B, alpha=1.5, beta=-0.5, C0=C0)
            torch.cuda.synchronize()
            got = C.cpu().numpy()
            assert N.rel_frobenius(got, ref.cpu().numpy()) <= TOL
            exact = oracle.gemm(A.cpu().numpy(), B.cpu().numpy(), alpha=1.5, beta=-0.5,
                                C0=C0.cpu().numpy())
            assert N.rel_frobenius(got, exact) <= TOL


def test_noalloc_refuses_a_plan_beyond_its_scratch_limit():
    import torch
    import paper_2311_03543_b300 as cp
    # 128 x 4096 x 4096: 32 tiles split 10 ways -> 10*128*4096*4 bytes > 16 MiB
    A = torch.zeros((128, 4096), device="cuda")
    B = torch.zeros((4096, 4096), device="cuda")
    C = torch.zeros((128, 4096), device="cuda")
    assert _noalloc(A, B, C) == cp.ERR_INVALID
    assert b"16 MiB" in cp.compar_last_error()


@pytest.mark.parametrize("m,n,k", [(16, 4096, 4096), (64, 15360, 2048), (8, 227328, 1000)])
def test_skinny_in_kernel_slab_sum_equals_reduce_pass_bitwise(m, n, k):
    """The skinny-M plan adds up to 8 cluster sums in the kernel (the last
    cluster to arrive); the allocation-free entry point adds the same slabs
    with the reduce pass.  Both add them in cluster order and apply alpha and
    beta the same way, so the results agree bit for bit."""
    import torch
    import paper_2311_03543_b300 as cp
    plan = cp.Context.simt_plan(m, n, k)
    assert plan["skinny"] == 1 and 1 < plan["splits"] <= 8
    with cp.Context(0) as ctx:
        A = torch.from_numpy(W.uniform(m, k, seed=91)).cuda()
        B = torch.from_numpy(W.uniform(k, n, seed=92)).cuda()
        C0 = torch.from_numpy(W.uniform(m, n, seed=93)).cuda()
        C = C0.clone()
        assert _noalloc(A, B, C, alpha=1.5, beta=-0.5) == cp.OK
        ref = _regular(ctx, A, B, alpha=1.5, beta=-0.5, C0=C0)
        torch.cuda.synchronize()
        assert torch.equal(C, ref)
