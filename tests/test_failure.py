"""Failure detection without faulting the GPU.

* Device side: a kernel whose bounded wait can never complete (an mbarrier
  nothing arrives on) gives up after the wait budget, records
  COMPAR_ERR_TIMEOUT in the context's error word and returns; the context
  stays usable.
* Host side: COMPAR_TEST_FAIL_VARIANT makes the dispatcher treat one variant's
  launch as failed; the runtime quarantines it and re-dispatches the call to
  the next choice, which still computes the right product.
* A call refused for the caller's reasons (its workspace would have to grow
  inside a stream capture) returns its status and quarantines nothing.
* Bad arguments are refused synchronously."""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    import paper_2311_03543_b300 as cp
    with cp.Context(0) as ctx:
        ctx.set_wait_budget(2_000_000)           # 2 ms
        ctx.selftest_timeout()
        assert ctx.check_device_error() == cp.ERR_TIMEOUT
        assert ctx.check_device_error() == cp.OK  # read-and-clear
        A = torch.from_numpy(W.uniform(64, 64, 1)).cuda()
        B = torch.from_numpy(W.uniform(64, 64, 2)).cuda()
        C = torch.empty((64, 64), device="cuda")
        ctx.gemm(A, B, C)
        torch.cuda.synchronize()
        assert N.rel_frobenius(C.cpu().numpy(), oracle.gemm(A.cpu().numpy(),
                                                            B.cpu().numpy())) <= 1e-5
        assert ctx.check_device_error() == cp.OK


def test_injected_variant_failure_is_quarantined(monkeypatch):
    import torch
    import paper_2311_03543_b300 as cp
    m = n = k = 2048
    A = torch.from_numpy(W.uniform(m, k, 3)).cuda()
    B = torch.from_numpy(W.uniform(k, n, 4)).cuda()
    with cp.Context(0) as probe:
        first = probe.select(m, n, k, cp.F32, 1e-5)
    monkeypatch.setenv("COMPAR_TEST_FAIL_VARIANT", str(first))
    with cp.Context(0) as ctx:
        C = torch.empty((m, n), device="cuda")
        ctx.gemm(A, B, C, tol=1e-5)
        used = ctx.last_variant()
        assert used != first and used >= 0
        torch.cuda.synchronize()
        rows = W.sample_rows(m, 16, 5)
        ref = oracle.gemm_rows(A.cpu().numpy(), B.cpu().numpy(), rows)
        assert N.rel_frobenius(C.cpu().numpy()[rows], ref) <= 1e-5
        # the quarantined variant stays out of later calls of this context
        ctx.clear_decisions()
        assert ctx.select(m, n, k, cp.F32, 1e-5) != first


# the refused call enqueues nothing, so the capture ends with an empty graph
@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_capture_refusal_quarantines_nothing():
    """With the decision cached but the workspace still empty, the call inside
    a stream capture is refused (COMPAR_ERR_UNSUPPORTED); the refused variant
    is still the selection afterwards, and the same call outside the capture
    runs it and matches the oracle."""
    import torch
    import paper_2311_03543_b300 as cp
    m = n = k = 2048
    A = torch.from_numpy(W.uniform(m, k, 13)).cuda()
    B = torch.from_numpy(W.uniform(k, n, 14)).cuda()
    C = torch.empty((m, n), device="cuda")
    with cp.Context(0) as ctx:
        v = ctx.select(m, n, k, cp.F32, 1e-5)     # cached; nothing has run yet
        assert v == cp.V_SPLIT3, cp.VARIANT_NAMES[v]  # its pre-pass needs the workspace
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        status = None
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            try:
                ctx.gemm(A, B, C, tol=1e-5, stream=s)
            except cp.ComparError as e:
                status = e.status
        del g                                     # never replayed
        assert status == cp.ERR_UNSUPPORTED
        ctx.clear_decisions()
        assert ctx.select(m, n, k, cp.F32, 1e-5) == v
        ctx.gemm(A, B, C, tol=1e-5)
        assert ctx.last_variant() == v
        torch.cuda.synchronize()
        rows = W.sample_rows(m, 16, 15)
        ref = oracle.gemm_rows(A.cpu().numpy(), B.cpu().numpy(), rows)
        assert N.rel_frobenius(C.cpu().numpy()[rows], ref) <= 1e-5
        assert ctx.check_device_error() == cp.OK


def test_error_left_pending_by_the_caller_fails_no_launch():
    """A CUDA error the caller left pending (an ignored failing runtime call)
    is not read as the library's launch failing: the selected variant runs,
    stays the selection, and matches the oracle."""
    import ctypes
    import torch
    import paper_2311_03543_b300 as cp
    rt = ctypes.CDLL("libcudart.so.13")      # the runtime the library runs on
    m = n = k = 1024
    A = torch.from_numpy(W.uniform(m, k, 16)).cuda()
    B = torch.from_numpy(W.uniform(k, n, 17)).cuda()
    C = torch.empty((m, n), device="cuda")
    with cp.Context(0) as ctx:
        v = ctx.select(m, n, k, cp.F32, 1e-5)
        torch.cuda.synchronize()
        assert rt.cudaSetDevice(ctypes.c_int(1 << 20)) != 0   # leaves an error pending
        ctx.gemm(A, B, C, tol=1e-5)
        assert ctx.last_variant() == v
        ctx.clear_decisions()
        assert ctx.select(m, n, k, cp.F32, 1e-5) == v
        torch.cuda.synchronize()
        rows = W.sample_rows(m, 16, 18)
        ref = oracle.gemm_rows(A.cpu().numpy(), B.cpu().numpy(), rows)
        assert N.rel_frobenius(C.cpu().numpy()[rows], ref) <= 1e-5


# the refused calls enqueue nothing, so the capture ends with an empty graph
@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_uncapturable_calls_refuse_a_capturing_stream():
    """The batched call (it runs a graph of its own), the autotuner, the
    variant timer and the residual check (they synchronise) and the
    host-buffer call (its copy streams are its own) return
    COMPAR_ERR_UNSUPPORTED on a stream being captured and enqueue nothing;
    the context then runs the same calls normally."""
    import torch
    import paper_2311_03543_b300 as cp
    m, n, k = 96, 80, 64
    A = torch.from_numpy(W.uniform(m, k, 19)).cuda()
    B = torch.from_numpy(W.uniform(k, n, 20)).cuda()
    C = torch.empty((m, n), device="cuda")
    probs = [dict(m=m, n=n, k=k, lda=k, ldb=n, ldc=n, dtype=cp.F32, A=A.data_ptr(),
                  B=B.data_ptr(), C=C.data_ptr())]
    hA, hB = A.cpu().numpy(), B.cpu().numpy()
    hC = np.zeros((m, n), np.float32)
    with cp.Context(0) as ctx:
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        codes = []
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for call in (lambda: ctx.gemm_batched(probs, tol=1e-5, stream=s),
                         lambda: ctx.autotune_batched(probs, tol=1e-5, stream=s),
                         lambda: ctx.gemm_host(hA, hB, hC, stream=s),
                         lambda: ctx.measure(cp.V_SIMT, A, B, C, stream=s),
                         lambda: ctx.residual_check(A, B, C, stream=s)):
                try:
                    call()
                    codes.append(cp.OK)
                except cp.ComparError as e:
                    codes.append(e.status)
        del g
        assert codes == [cp.ERR_UNSUPPORTED] * 5
        ref = oracle.gemm(hA, hB)
        ctx.gemm_batched(probs, tol=1e-5)
        torch.cuda.synchronize()
        assert N.rel_frobenius(C.cpu().numpy(), ref) <= 1e-5
        ctx.gemm_host(hA, hB, hC)
        torch.cuda.synchronize()
        assert N.rel_frobenius(hC, ref) <= 1e-5


def test_bad_arguments_are_refused():
    import torch
    import paper_2311_03543_b300 as cp
    with cp.Context(0) as ctx:
        h = ctx.handle
        assert cp.compar_gemm(h, -1, 4, 4, cp.F32, 0.0, 16, 16, 16, None) == cp.ERR_INVALID
        assert cp.compar_gemm(h, 4, 4, 4, cp.F32, 0.0, None, 16, 16, None) == cp.ERR_INVALID
        assert cp.compar_gemm(h, 4, 4, 4, 7, 0.0, 16, 16, 16, None) == cp.ERR_INVALID
        assert cp.compar_gemm(h, 4, 4, 4, cp.F32, float("nan"), 16, 16, 16, None) == cp.ERR_INVALID
        assert cp.compar_set_fp8_scales(h, 0.0, 1.0) == cp.ERR_INVALID
        assert cp.compar_set_scalars(h, float("inf"), 0.0) == cp.ERR_INVALID
        assert cp.compar_gemm(h, 4, 4, 4, cp.F32, 1e-30, 16, 4096, 8192, None) == cp.ERR_NO_VARIANT
        # C sharing bytes with A or B (a 4 x 4 float32 operand spans 64 bytes)
        assert cp.compar_gemm(h, 4, 4, 4, cp.F32, 0.0, 4096, 8192, 4096 + 48, None) == cp.ERR_INVALID
        assert cp.compar_gemm(h, 4, 4, 4, cp.F32, 0.0, 4096, 8192, 8192 - 48, None) == cp.ERR_INVALID
