"""Online selection on the GPU: exploration picks run and are recorded, the
MLP is fine-tuned from its weights after enough new records, and every call
still computes the right product."""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu

SELECTOR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2311_03543_b300", "selector_default.bin")


def test_exploration_records_and_finetunes():
    import torch
    import paper_2311_03543_b300 as cp
    with cp.Context(0) as ctx:
        ctx.selector_load(SELECTOR)
        before = ctx.predict(300, 200, 100, cp.F32, 1e-3)[0]
        n0 = len(ctx.records())
        ctx.set_online(epsilon=0.5, retrain_every=40, finetune_steps=200)
        g = np.random.default_rng(3)
        for i in range(90):
            m, n, k = (int(x) for x in g.integers(16, 400, size=3))
            A = torch.from_numpy(W.uniform(m, k, seed=i)).cuda()
            B = torch.from_numpy(W.uniform(k, n, seed=1000 + i)).cuda()
            C = torch.empty((m, n), device="cuda")
            ctx.gemm(A, B, C, tol=1e-5)
            if i % 30 == 0:
                torch.cuda.synchronize()
                ref = oracle.gemm(A.cpu().numpy(), B.cpu().numpy())
                assert N.rel_frobenius(C.cpu().numpy(), ref) <= 1e-5
        explored, retrains = ctx.online_stats()
        assert explored > 10
        assert retrains >= 2
        assert len(ctx.records()) >= n0 + 90
        after = ctx.predict(300, 200, 100, cp.F32, 1e-3)[0]
        assert after != before          # the model moved
        ctx.set_online(0.0, 0, 0)
