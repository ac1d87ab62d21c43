"""Selection for the thermal-stencil component on held-out contexts (GPU).

The selector file shipped with the package carries a stencil history table
(timings of every stencil variant on 150 seeded training contexts).  For 60
held-out contexts (grids 64 - 8192 per side, 1 - 1000 steps, a seed disjoint
from training) the selector's pick is compared with exhaustive measurement on
a separate judge context; every stencil variant computes the same grid, so
all are feasible and regret is by time alone (oracle/selector_ref)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import selector_ref as S

pytestmark = pytest.mark.gpu

SELECTOR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2311_03543_b300", "selector_default.bin")


def test_stencil_selection_regret():
    import torch
    import paper_2311_03543_b300 as cp
    sel = cp.Context(0)
    sel.selector_load(SELECTOR)
    judge = cp.Context(0)
    prm = cp.Context.stencil_params(**W.STENCIL_PARAMS)
    regrets = []
    try:
        for i, (rows, cols, iters) in enumerate(W.stencil_contexts(60, seed=12345)):
            pick = sel.stencil_select(rows, cols, iters)
            g = torch.Generator(device="cuda")
            g.manual_seed(9000 + i)
            T = torch.rand((rows, cols), generator=g, device="cuda") * 20 + 80
            P = torch.rand((rows, cols), generator=g, device="cuda")
            out = torch.empty_like(T)
            times = {v: judge.stencil_measure(v, T, P, out, iters, prm, warmup=1, reps=3)
                     for v in range(cp.NUM_STENCIL_VARIANTS)
                     if judge.stencil_supported(v, rows, cols)}
            assert pick in times
            errs = {v: 0.0 for v in times}
            regrets.append(S.regret(pick, times, errs, 1.0))
    finally:
        sel.close()
        judge.close()
    r = np.array(regrets)
    print(f"\nstencil held-out contexts: {len(r)}; mean regret {100 * r.mean():.2f} %")
    assert r.mean() <= 0.10
