"""Record timings and errors through the library, train the learned selector
on the GPU, and write a selector file.

    python -m paper_2311_03543_b300.train_selector --out selector.bin

Training contexts are the shapes of the three GEMM workloads: the 256^3
product, the FP32-accuracy size sweep (square n = 64..8192 step 64 plus
4096x4096x64 and 16x4096x4096) and the 4096^3 precision study, each with
float32, bf16 and E4M3 inputs, plus 3000 seeded random contexts (rectangular
shapes; the seed is disjoint from every evaluation set).  The MLP's time
head learns a correction to the roofline prior, log2(measured / prior), so
far from its data it falls back towards the prior.  For every context and
every variant that can
run it, ``compar_measure`` times the variant (one record per timed run) and
``compar_residual_check`` labels its relative error (one more record).  The
MLP ensemble is then trained by the library's own CUDA kernels
(``compar_selector_train``); the history table is filled by the same
measurements.  The thermal-stencil component's history table is filled by
timing its variants on 150 seeded stencil contexts (grids 64 - 8192, 1 - 1000
steps).  Everything runs through the C ABI; nothing here computes.
"""
import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def training_contexts(random_count=3000):
    """The three workloads' shapes for every dtype, plus seeded random
    contexts (M, N, K log-uniform in [16, 8192], seed disjoint from any
    evaluation set) so that rectangular shapes are seen too."""
    import workloads as W
    shapes = [W.PARITY_256] + W.sweep_shapes() + [(4096, 4096, 4096)]
    out = []
    for dt in (W.F32, W.BF16, W.F8E4M3):
        for s in shapes:
            out.append(s + (dt,))
    for (m, n, k, dt, _tol) in W.training_contexts(random_count):
        out.append((m, n, k, dt))
    return out


def make_inputs(torch, m, n, k, dt, seed, dev):
    """Seeded device inputs of the given element type."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    A = torch.rand((m, k), generator=g, device=dev) * 2 - 1
    B = torch.rand((k, n), generator=g, device=dev) * 2 - 1
    if dt == 1:     # bf16 values
        A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
    elif dt == 2:   # E4M3 values (as raw bytes)
        A = (A * 8).to(torch.float8_e4m3fn).view(torch.uint8)
        B = (B * 8).to(torch.float8_e4m3fn).view(torch.uint8)
    return A.contiguous(), B.contiguous()


def collect(ctx, cp, torch, contexts, reps, dev, log=print, budget_s=None):
    t0 = time.time()
    n_rec = 0
    for i, (m, n, k, dt) in enumerate(contexts):
        A, B = make_inputs(torch, m, n, k, dt, 1000 + i, dev)
        C = torch.empty((m, n), device=dev)
        for v in range(cp.NUM_VARIANTS):
            if not ctx.supported(v, m, n, k, dt):
                continue
            r = reps if m * n * k <= 2 ** 33 else max(3, reps // 3)
            ctx.measure(v, A, B, C, tol=1.0, warmup=1, reps=r, dtype=dt)
            err = ctx.residual_check(A, B, C, nrows=8, seed=i, dtype=dt)
            rec = cp.compar_record_t()
            rec.m, rec.n, rec.k, rec.dtype, rec.variant, rec.batch = m, n, k, dt, v, 1
            rec.tol, rec.time_ms, rec.rel_err = 1.0, -1.0, max(err, 1e-12)
            ctx.record_add([rec])
            n_rec += r + 1
        if i % 50 == 0:
            log(f"[train_selector] {i}/{len(contexts)} contexts, {n_rec} records, "
                f"{time.time() - t0:.0f} s")
        if budget_s and time.time() - t0 > budget_s:
            log("[train_selector] time budget reached")
            break
    return n_rec


def collect_stencil(ctx, cp, torch, contexts, reps, dev, log=print):
    """Time every stencil variant on each (rows, cols, iters) context; the
    measurements feed the context's stencil history table."""
    import workloads as W
    prm = cp.Context.stencil_params(**W.STENCIL_PARAMS)
    t0 = time.time()
    for i, (rows, cols, iters) in enumerate(contexts):
        g = torch.Generator(device=dev)
        g.manual_seed(3000 + i)
        T = torch.rand((rows, cols), generator=g, device=dev) * 20 + 80
        P = torch.rand((rows, cols), generator=g, device=dev)
        out = torch.empty_like(T)
        for v in range(cp.NUM_STENCIL_VARIANTS):
            if ctx.stencil_supported(v, rows, cols):
                ctx.stencil_measure(v, T, P, out, iters, prm, warmup=1, reps=reps)
        if i % 20 == 0:
            log(f"[train_selector] stencil {i}/{len(contexts)} contexts, {time.time() - t0:.0f} s")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2311_03543_b300",
                                                  "selector_default.bin"))
    ap.add_argument("--reps", type=int, default=16)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--budget-s", type=float, default=None)
    ap.add_argument("--random-count", type=int, default=3000,
                    help="seeded random training contexts added to the workloads' shapes")
    ap.add_argument("--stencil-count", type=int, default=150,
                    help="seeded stencil training contexts (grids 64-8192, 1-1000 steps)")
    args = ap.parse_args(argv)
    import torch
    import paper_2311_03543_b300 as cp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    with cp.Context(0, selector=None) as ctx:   # trained from its own records only
        ctx.record_enable(True)
        n = collect(ctx, cp, torch, training_contexts(args.random_count), args.reps, dev,
                    budget_s=args.budget_s)
        import workloads as W
        collect_stencil(ctx, cp, torch, W.stencil_contexts(args.stencil_count, seed=777), 3, dev)
        t0 = time.time()
        vl = ctx.selector_train(steps=args.steps, batch=128, lr=args.lr, seed=args.seed)
        print(f"[train_selector] {n} records; trained {args.steps} steps in "
              f"{time.time() - t0:.1f} s; held-out loss {vl:.4f}")
        ctx.selector_save(args.out)
        print(f"[train_selector] wrote {args.out}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
