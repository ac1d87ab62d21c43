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
        explored, retrains, rejected = ctx.online_stats()
        assert explored > 10
        assert retrains >= 2
        assert len(ctx.records()) >= n0 + 90
        after = ctx.predict(300, 200, 100, cp.F32, 1e-3)[0]
        # a kept fine-tune moves the model; a discarded one leaves it as it was
        assert (after != before) == (rejected < retrains)
        ctx.set_online(0.0, 0, 0)


def _square_selector(path, steps=6000):
    """A selector that has seen square shapes only: every variant timed (and
    its error labelled) on n x n x n for 18 sizes from 16 to 4096 and every
    dtype, through the library's own recording, then the MLP ensemble trained
    by the library's kernels and the file written (its rehearsal sample is
    these square records)."""
    import torch
    import paper_2311_03543_b300 as cp
    from paper_2311_03543_b300 import train_selector as TS
    sizes = sorted({int(round(16 * 2 ** (8 * i / 17))) for i in range(18)})
    contexts = [(n, n, n, dt) for dt in (W.F32, W.BF16, W.F8E4M3) for n in sizes]
    with cp.Context(0, selector=None) as ctx:
        ctx.record_enable(True)
        TS.collect(ctx, cp, torch, contexts, 4, torch.device("cuda", 0), log=lambda *a: None)
        ctx.selector_train(steps=steps, batch=128, lr=1e-3, seed=1)
        ctx.selector_save(path)


def _judge_contexts(contexts, seed0):
    """Every eligible variant timed once per context by a context of its own
    (so no timing reaches the selector under test), and its error against
    the FP64 oracle on the first and last row of every 128-row tile."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev
    from test_selector_regret import _exact, _inputs
    judge = cp.Context(0)
    out = []
    for i, (m, n, k, dt, tol) in enumerate(contexts):
        A, B = _inputs(m, n, k, dt, seed0 + 2 * i)
        dA, dB = dev(A), dev(B)
        C = torch.empty((m, n), device="cuda")
        rows = W.tile_rows(m, seed=i, inner=0)
        ref = oracle.gemm_rows(_exact(A, dt), _exact(B, dt), rows)
        times, errs = {}, {}
        for v in range(cp.NUM_VARIANTS):
            if not judge.supported(v, m, n, k, dt):
                continue
            times[v] = judge.measure(v, dA, dB, C, tol=tol, warmup=1, reps=3, dtype=dt)
            got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
            errs[v] = N.rel_frobenius(got, ref)
        out.append((m, n, k, dt, tol, times, errs))
    judge.close()
    return out


def _mean_regret(sel, judged, worst=None):
    from oracle import selector_ref as S
    rs, viol = [], 0
    for m, n, k, dt, tol, times, errs in judged:
        if S.exhaustive_pick(times, errs, tol) is None:
            continue
        sel.clear_decisions()
        pick = sel.select(m, n, k, dt, tol)
        viol += pick not in S.feasible(errs, tol)
        rs.append(S.regret(pick, times, errs, tol))
        if worst is not None:
            worst.append((rs[-1], (m, n, k, dt, tol), pick, S.exhaustive_pick(times, errs, tol)))
    return float(np.mean(rs)), viol, len(rs)


def test_online_selection_lowers_regret_from_a_squares_only_selector(tmp_path):
    """The paper's runtime mis-selects where its performance models are
    under-trained and names better model training as future work (Sec. 3.2,
    Sec. 5).  A selector trained only on square shapes serves a program whose
    120 rectangular contexts (the first held-out contexts, never seen in
    training) it calls again and again: eight passes in shuffled order with
    exploration (probability 0.25, on every call) and a 300-step warm-start
    fine-tune every 100 new timing records.  Afterwards its mean regret on
    those contexts against the exhaustive judge must have fallen, with no
    tolerance violated; on the next 120 held-out contexts, which the program
    never called, it must not have risen (by more than a point; it fell in
    every run measured: the fine-tuned model generalises).  Measured: 7.8 - 8.9 % -> 3.3 - 5.5 % on the program in
    most runs; in one run most fine-tunes were discarded by the held-out
    guard (the timings it learns from are measured, so they vary) and it fell
    only from 7.8 % to 7.2 %.  So the bound asserted is a 5 % drop.  On the
    contexts never called: 6.9 - 7.8 % -> 4.2 - 5.2 %."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev
    from test_selector_regret import _inputs
    path = str(tmp_path / "squares.bin")
    _square_selector(path)
    program, unseen_set = W.heldout_contexts()[:120], W.heldout_contexts()[120:240]
    judged = _judge_contexts(program, 60000)
    unseen = _judge_contexts(unseen_set, 62000)
    order = np.random.default_rng(8).permutation(np.tile(np.arange(len(program)), 8))
    inputs = {}
    with cp.Context(0) as sel:
        sel.selector_load(path)
        wb, wa = [], []
        before, v_before, n_ctx = _mean_regret(sel, judged, wb)
        unseen_before, _, _ = _mean_regret(sel, unseen)
        sel.set_online(epsilon=0.25, retrain_every=100, finetune_steps=300)
        for i in order:
            m, n, k, dt, tol = program[i]
            if i not in inputs:
                A, B = _inputs(m, n, k, dt, 80000 + 2 * int(i))
                inputs[i] = (dev(A), dev(B), torch.empty((m, n), device="cuda"))
            A, B, C = inputs[i]
            sel.gemm(A, B, C, tol=tol, dtype=dt)
        torch.cuda.synchronize()
        explored, tunes, rejected = sel.online_stats()
        sel.set_online(0.0, 0, 0)
        after, v_after, _ = _mean_regret(sel, judged, wa)
        unseen_after, v_unseen, _ = _mean_regret(sel, unseen)
        assert sel.check_device_error() == cp.OK
    print(f"\nonline selection from a squares-only selector, {n_ctx} program contexts: "
          f"regret {100 * before:.2f} % (violations {v_before}) -> {100 * after:.2f} % "
          f"(violations {v_after}); {explored} explored calls, {tunes} fine-tunes "
          f"({rejected} discarded); {len(unseen_set)} contexts never called: {100 * unseen_before:.2f} % -> "
          f"{100 * unseen_after:.2f} % (violations {v_unseen})")
    for name, w in (("before", wb), ("after", wa)):
        print(name, "worst contexts (regret, context, pick, best):",
              [(round(r, 3), c, p, b) for r, c, p, b in sorted(w, reverse=True)[:6]])
    assert tunes >= 6 and explored >= 100
    assert v_after == 0 and v_unseen == 0
    assert after <= 0.95 * before
    # where the fine-tunes are mostly discarded the model barely moves: the
    # contexts never called may then shift by a fraction of a point
    assert unseen_after <= unseen_before + 0.01
