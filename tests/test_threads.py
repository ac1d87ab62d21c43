"""Several host threads, one context each (the documented threading model),
on one GPU at once (GPU).

The library's process-wide state (per-device kernel set-up, launch
counters, the thread-local error text) is shared by the threads, and each
context's workspace is its own.  ctypes releases the GIL while a library call
runs, so the calls overlap on the host; each thread uses its own stream, so
their kernels may overlap on the GPU too.  Every thread checks its results
against the oracle."""
import threading

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu

# (m, n, k, forced variant or None): a pair-kernel 3xBF16 call, the fused
# variant, the SIMT skinny plan (its cluster-sum arrival counters live in
# the context's workspace), a TF32 call and the selector's own pick
CALLS = [(1536, 1024, 768, 5), (512, 384, 256, 9), (16, 2048, 2048, 1), (300, 200, 1000, 2),
         (257, 129, 65, None)]


def _worker(tid, errors):
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev
    try:
        s = torch.cuda.Stream()
        with cp.Context(0) as ctx:
            for rep in range(3):
                for j, (m, n, k, v) in enumerate(CALLS):
                    seed = 1000 * tid + 10 * j + rep
                    A = W.uniform(m, k, seed=seed)
                    B = W.uniform(k, n, seed=seed + 5)
                    with torch.cuda.stream(s):
                        dA, dB = dev(A), dev(B)
                        C = torch.full((m, n), float("nan"), device="cuda")
                    s.synchronize()
                    ctx.force_variant(v)
                    try:
                        ctx.gemm(dA, dB, C, tol=1e-5 if v != 2 else 0.0, stream=s)
                    finally:
                        ctx.force_variant(None)
                    s.synchronize()
                    rows = W.tile_rows(m, seed=seed)
                    ref = oracle.gemm_rows(A, B, rows)
                    err = N.rel_frobenius(C.cpu().numpy()[rows], ref)
                    lim = 2e-3 if v == 2 else 1e-5
                    if not err <= lim:
                        errors.append((tid, rep, (m, n, k, v), err))
            if ctx.check_device_error(s) != cp.OK:
                errors.append((tid, "device error"))
    except Exception as e:  # reported by the main thread
        errors.append((tid, repr(e)))


def test_contexts_on_several_threads_at_once():
    errors = []
    threads = [threading.Thread(target=_worker, args=(t, errors)) for t in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads), "a worker did not finish"
    assert not errors, errors
