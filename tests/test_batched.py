"""Batched calls (GPU): the persistent grouped kernel in its CUDA graph and
the per-GEMM loop, against the FP64 oracle problem by problem.

Modes: float32 problems at tol 1e-5 run as 3xBF16 (<= 1e-5 vs the oracle);
at a loose tolerance as TF32 (<= 2e-3); bf16 problems exactly on their bf16
values (<= 1e-5); E4M3 problems, and float32 problems at a tolerance below
3xBF16's error level, leave the grouped launch and run one by one."""
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


def _make_batch(specs, seed):
    """specs: (m, n, k, dtype, lda_pad, ldb_pad, ldc_pad, alpha, beta)."""
    import torch
    from gpu_util import dev
    probs, host = [], []
    for i, (m, n, k, dt, pa, pb, pc, alpha, beta) in enumerate(specs):
        lda, ldb, ldc = k + pa, n + pb, n + pc
        if dt == W.F32:
            A = W.uniform(m, lda, seed + 3 * i)
            B = W.uniform(k, ldb, seed + 3 * i + 1)
        elif dt == W.BF16:
            A = W.bf16_input(m, lda, seed + 3 * i)
            B = W.bf16_input(k, ldb, seed + 3 * i + 1)
        else:
            A = W.fp8_input(m, lda, seed + 3 * i, 7)
            B = W.fp8_input(k, ldb, seed + 3 * i + 1, 7)
        C0 = W.uniform(m, ldc, seed + 3 * i + 2)
        dA, dB, dC = dev(A), dev(B), dev(C0)
        probs.append(dict(m=m, n=n, k=k, lda=lda, ldb=ldb, ldc=ldc, dtype=dt,
                          A=dA.data_ptr(), B=dB.data_ptr(), C=dC.data_ptr(),
                          alpha=alpha, beta=beta))
        host.append((A, B, C0, dA, dB, dC))
    return probs, host


def _exact(X, dt):
    if dt == W.F32:
        return X.astype(np.float64)
    if dt == W.BF16:
        return N.bf16_to_f32(X).astype(np.float64)
    return N.e4m3_to_f64(X)


def _check(specs, host, tol_f32):
    import torch
    torch.cuda.synchronize()
    worst = 0.0
    for (m, n, k, dt, pa, pb, pc, alpha, beta), (A, B, C0, dA, dB, dC) in zip(specs, host):
        if m == 0 or n == 0:
            continue
        got = dC.cpu().numpy()[:, :n]
        ref = oracle.gemm(_exact(A[:, :k], dt), _exact(B[:, :n], dt), alpha=alpha, beta=beta,
                          C0=C0[:, :n].astype(np.float64))
        err = N.rel_frobenius(got, ref)
        lim = tol_f32 if dt == W.F32 else 1e-5
        assert err <= lim, (m, n, k, dt, err)
        worst = max(worst, err)
        # padding columns of C are never written
        assert np.array_equal(dC.cpu().numpy()[:, n:], C0[:, n:])
    return worst


def _random_specs(count, seed, lo=1, hi=300, dtypes=(W.F32, W.BF16)):
    g = np.random.default_rng(seed)
    specs = []
    for _ in range(count):
        m, n, k = (int(x) for x in g.integers(lo, hi, size=3))
        dt = dtypes[int(g.integers(0, len(dtypes)))]
        pads = [int(x) for x in g.integers(0, 3, size=3)]
        specs.append((m, n, k, dt, pads[0], pads[1], pads[2], float(g.choice([1.0, 0.5, -2.0])),
                      float(g.choice([0.0, 1.0, -0.5]))))
    return specs


def test_grouped_fp32_accurate_and_bf16(ctx):
    import paper_2311_03543_b300 as cp
    specs = _random_specs(40, seed=1)
    probs, host = _make_batch(specs, 100)
    ctx.force_variant(cp.V_GROUPED)
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.force_variant(None)
    assert ctx.check_device_error() == cp.OK
    _check(specs, host, 1e-5)


@pytest.mark.parametrize("config", [1, 2, 3, 4])
def test_every_grouped_configuration(ctx, config):
    """Tiles of 128 or 256 columns, problems in given order or largest
    first: same products."""
    import paper_2311_03543_b300 as cp
    specs = _random_specs(30, seed=11, hi=600)
    probs, host = _make_batch(specs, 900)
    ctx.set_batched_config(config)
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.set_batched_config(None)
    assert ctx.check_device_error() == cp.OK
    assert ctx.last_variant() == cp.V_GROUPED
    _check(specs, host, 1e-5)


def test_batched_config_is_validated(ctx):
    import paper_2311_03543_b300 as cp
    assert cp.compar_set_batched_config(ctx.handle, 5) == cp.ERR_INVALID
    assert cp.compar_set_batched_config(ctx.handle, -2) == cp.ERR_INVALID


def test_grouped_bf16_operands_read_in_place(ctx):
    """bf16 problems whose rows are 16-byte aligned (ld a multiple of 8) are
    read by TMA as stored: A row-major M x K, B row-major K x N (MN-major),
    no pre-pass.  Shapes straddle the 128-row, 64/128-column and 64-deep K
    tiles."""
    import paper_2311_03543_b300 as cp
    shapes = [(1, 8, 1), (17, 64, 63), (128, 128, 64), (129, 136, 65), (200, 320, 129),
              (64, 8, 300), (300, 72, 40)]
    specs = [(m, n, k, W.BF16, (-k) % 8, 0, 0, 1.0, 0.0) for (m, n, k) in shapes]
    probs, host = _make_batch(specs, 700)
    ctx.force_variant(cp.V_GROUPED)
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.force_variant(None)
    assert ctx.check_device_error() == cp.OK
    _check(specs, host, 1e-5)


def test_grouped_tf32_mode(ctx):
    import paper_2311_03543_b300 as cp
    specs = _random_specs(24, seed=2, dtypes=(W.F32,))
    probs, host = _make_batch(specs, 200)
    ctx.force_variant(cp.V_GROUPED)
    try:
        ctx.gemm_batched(probs, tol=1e-2)
    finally:
        ctx.force_variant(None)
    _check(specs, host, 2e-3)


def test_tolerance_below_3xbf16_runs_those_problems_singly(ctx):
    """At tol 2e-6 the grouped kernel's float32 mode (3xBF16, ~4e-6) does not
    qualify: float32 problems are selected one by one (6-product split or
    FP32 SIMT) and still meet the tolerance; bf16 problems stay grouped."""
    import paper_2311_03543_b300 as cp
    specs = _random_specs(16, seed=6)
    probs, host = _make_batch(specs, 600)
    ctx.force_variant(cp.V_GROUPED)
    try:
        ctx.gemm_batched(probs, tol=2e-6)
    finally:
        ctx.force_variant(None)
    assert ctx.check_device_error() == cp.OK
    _check(specs, host, 2e-6)


def test_fp8_and_empty_problems_in_a_batch(ctx):
    import paper_2311_03543_b300 as cp
    specs = [(64, 80, 96, W.F8E4M3, 0, 0, 0, 1.0, 0.0), (33, 17, 0, W.F32, 0, 0, 0, 1.0, 2.0),
             (0, 5, 7, W.F32, 0, 0, 0, 1.0, 0.0), (100, 120, 140, W.F32, 1, 0, 0, 1.0, 0.0),
             (50, 60, 70, W.BF16, 8, 0, 4, 1.0, 0.5)]
    probs, host = _make_batch(specs, 300)
    ctx.force_variant(cp.V_GROUPED)
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.force_variant(None)
    _check(specs, host, 1e-5)


def test_graph_replay_with_new_data(ctx):
    import paper_2311_03543_b300 as cp
    specs = _random_specs(16, seed=3)
    for rnd in range(3):                       # same shapes: the graph is reused
        probs, host = _make_batch(specs, 400 + 50 * rnd)
        ctx.force_variant(cp.V_GROUPED)
        try:
            ctx.gemm_batched(probs, tol=1e-5)
        finally:
            ctx.force_variant(None)
        _check(specs, host, 1e-5)


def test_graph_cache_separates_3xbf16_and_tf32_batches(ctx):
    """The same float32 shapes at a 3xBF16 tolerance and at a TF32 one.  With
    A's rows not 16-byte aligned, A is copied in both modes, so the two
    batches have the same counts of problems, tiles, pre-pass jobs and
    pre-pass tiles.  Only the TF32 batch's pre-pass transposes B, though, and
    each batch must replay a graph captured for its own mode.  K > N
    throughout; fresh data every round."""
    import paper_2311_03543_b300 as cp
    specs = [(50, 20, 300, W.F32, 1, 0, 0, 1.0, 0.0), (130, 40, 257, W.F32, 1, 0, 0, 0.5, 1.0),
             (70, 64, 190, W.F32, 3, 0, 0, 1.0, 0.0)]
    assert all((k + pa) % 4 != 0 and k > n for (m, n, k, dt, pa, *_rest) in specs)
    for rnd, (tol, lim) in enumerate([(1e-5, 1e-5), (1e-2, 2e-3), (1e-5, 1e-5), (1e-2, 2e-3)]):
        probs, host = _make_batch(specs, 700 + 50 * rnd)
        ctx.force_variant(cp.V_GROUPED)
        try:
            ctx.gemm_batched(probs, tol=tol)
        finally:
            ctx.force_variant(None)
        assert ctx.check_device_error() == cp.OK
        _check(specs, host, lim)


def _check_elementwise(specs, host):
    """Every problem element by element within its mode's worst-case bound
    relative to |alpha| |A||B| + |beta| |C0| (3xBF16 for float32, exact-input
    accumulation for bf16).  For tiny random problems this is the right test:
    a short dot product can cancel, and then the relative Frobenius error of a
    two-element output says little about the arithmetic."""
    import torch
    from gpu_util import assert_elementwise, elem_bound
    torch.cuda.synchronize()
    for (m, n, k, dt, pa, pb, pc, alpha, beta), (A, B, C0, dA, dB, dC) in zip(specs, host):
        if m == 0 or n == 0:
            continue
        out = dC.cpu().numpy()
        Ax, Bx = _exact(A[:, :k], dt), _exact(B[:, :n], dt)
        c0 = C0[:, :n].astype(np.float64)
        ref = oracle.gemm(Ax, Bx, alpha=alpha, beta=beta, C0=c0)
        scale = abs(alpha) * oracle.gemm(np.abs(Ax), np.abs(Bx)) + abs(beta) * np.abs(c0)
        assert_elementwise(out[:, :n], ref, scale, elem_bound(5 if dt == W.F32 else 3, k))
        assert np.array_equal(out[:, n:], C0[:, n:])


def test_staging_growth_drops_and_recaptures_graphs(ctx):
    """A small batch, then one far larger (the descriptor staging buffers
    grow, which frees the old ones and drops every graph that copies from
    them), then the small batch again, captured anew: all against the
    oracle, element by element."""
    import paper_2311_03543_b300 as cp
    small = _random_specs(12, seed=21, hi=120)
    big = _random_specs(1500, seed=22, lo=1, hi=40)
    for rnd, specs in enumerate([small, big, small]):
        probs, host = _make_batch(specs, 800 + 100 * rnd)
        ctx.force_variant(cp.V_GROUPED)
        try:
            ctx.gemm_batched(probs, tol=1e-5)
        finally:
            ctx.force_variant(None)
        assert ctx.check_device_error() == cp.OK
        _check_elementwise(specs, host)


@pytest.mark.parametrize("v", [2, 3, 4, 5, 7, 8, 9])
def test_problems_run_singly_leave_c_padding_alone(ctx, v):
    """Problems run one by one (a forced tensor-core variant) with ldc > n
    and beta == 0: the padding columns of every row of C keep their
    contents, also when n is not a multiple of 4 (a bulk-tensor store
    clipped at the row's end writes up to the next 16-byte boundary, so those
    calls store C with plain stores)."""
    import paper_2311_03543_b300 as cp
    specs = [(52, 77, 796, W.F32, 5, 2, 3, 1.0, 0.0), (13, 1011, 1201, W.F32, 1, 8, 5, 0.5, 0.0),
             (130, 66, 300, W.F32, 0, 2, 6, 1.0, 0.0), (40, 64, 128, W.F32, 0, 0, 4, 1.0, 0.0)]
    if v == 4:
        specs += [(52, 77, 796, W.F8E4M3, 5, 2, 3, 1.0, 0.0)]
    if v == 9:   # the fused split reads float32 A and B in place: 16-byte rows
        specs = [(m, n, k, dt, (-k) % 4, (-n) % 4, pc, al, be)
                 for (m, n, k, dt, pa, pb, pc, al, be) in specs]
    else:        # (the support query assumes contiguous operands: padded ones run too)
        specs = [sp for sp in specs if ctx.supported(v, sp[0], sp[1], sp[2], sp[3])]
    assert specs
    probs, host = _make_batch(specs, 1200 + v)
    ctx.force_variant(v)
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.force_variant(None)
    assert ctx.check_device_error() == cp.OK
    _check(specs, host, {2: 2e-3, 3: 1e-2, 4: 1e-1}.get(v, 1e-5))


def test_random_batches_every_mode(ctx):
    """Ten seeded random batches on one context (float32 / bf16 / E4M3
    problems, shapes 1-400, padded leading dimensions, alpha and beta, C
    NaN-filled where beta == 0), at tolerances that select each float32 mode
    (3xBF16 at 1e-5, TF32 at 1e-2, one-by-one selection at 2e-6); every third
    batch repeats an earlier one, so its graph is replayed.  Element by
    element against the oracle, padding untouched."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import assert_elementwise, elem_bound
    g = np.random.default_rng(2024)
    made = []
    for b in range(10):
        if b % 3 == 2:
            specs, tol = made[int(g.integers(0, len(made)))]
        else:
            specs = []
            for _ in range(int(g.integers(1, 60))):
                m, n, k = (int(x) for x in np.exp(g.uniform(0, np.log(400), size=3)).round())
                dt = [W.F32, W.F32, W.BF16, W.F8E4M3][int(g.integers(0, 4))]
                pads = [int(x) for x in g.integers(0, 9, size=3)]
                specs.append((m, n, k, dt, pads[0], pads[1], pads[2],
                              float(g.choice([1.0, -1.5])), float(g.choice([0.0, 0.0, 0.5]))))
            tol = float(g.choice([1e-5, 1e-2, 2e-6]))
            made.append((specs, tol))
        probs, host = _make_batch(specs, 3000 + 100 * b)
        for (m, n, k, dt, pa, pb, pc, al, be), (A, B, C0, dA, dB, dC) in zip(specs, host):
            if be == 0.0:
                dC[:, :n] = float("nan")   # C is not read when beta == 0
        ctx.gemm_batched(probs, tol=tol)
        assert ctx.check_device_error() == cp.OK
        torch.cuda.synchronize()
        for (m, n, k, dt, pa, pb, pc, al, be), (A, B, C0, dA, dB, dC) in zip(specs, host):
            out = dC.cpu().numpy()
            Ax, Bx = _exact(A[:, :k], dt), _exact(B[:, :n], dt)
            c0 = C0[:, :n].astype(np.float64)
            ref = oracle.gemm(Ax, Bx, alpha=al, beta=be, C0=c0)
            scale = abs(al) * oracle.gemm(np.abs(Ax), np.abs(Bx)) + abs(be) * np.abs(c0)
            # the loosest mode a problem of this type can take at this tol
            v = (2 if tol >= 2e-3 else 5) if dt == W.F32 else 3
            assert_elementwise(out[:, :n], ref, scale, elem_bound(v, k))
            assert np.array_equal(out[:, n:], C0[:, n:]), (b, m, n, k, dt)


def test_loop_and_grouped_agree(ctx):
    import paper_2311_03543_b300 as cp
    specs = [s[:6] + (0, 1.0, 0.0) for s in _random_specs(12, seed=4, lo=16, hi=200)]
    probs, host = _make_batch(specs, 500)
    ctx.force_variant(cp.V_SIMT)               # loop mode, SIMT per problem
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.force_variant(None)
    _check(specs, host, 1e-5)


def test_autotune_then_run(ctx):
    specs = [s[:6] + (0, 1.0, 0.0) for s in _random_specs(30, seed=5, lo=32, hi=600)]
    probs, host = _make_batch(specs, 600)
    best, times = ctx.autotune_batched(probs, tol=1e-5)
    assert 0 <= best <= 4
    assert all(t > 0 for t in times)
    assert times[best] == min(times)
    ctx.gemm_batched(probs, tol=1e-5)          # uses the tuned configuration
    _check(specs, host, 1e-5)


def test_config4_batch_sampled(ctx):
    """512 problems, M, N, K log-uniform in [32, 2048] (seed 5), f32/bf16 mixed;
    12 problems checked on 16 oracle rows each."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev
    plist = W.batched_problems()
    rng = np.random.default_rng(6)
    probs, keep = [], {}
    check = set(int(i) for i in rng.choice(len(plist), size=12, replace=False))
    for i, (m, n, k, dt) in enumerate(plist):
        g = torch.Generator(device="cuda")
        g.manual_seed(i)
        A = torch.rand((m, k), generator=g, device="cuda") * 2 - 1
        B = torch.rand((k, n), generator=g, device="cuda") * 2 - 1
        if dt == W.BF16:
            A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
        C = torch.empty((m, n), device="cuda")
        probs.append(dict(m=m, n=n, k=k, lda=k, ldb=n, ldc=n, dtype=dt, A=A.data_ptr(),
                          B=B.data_ptr(), C=C.data_ptr()))
        keep[i] = (A, B, C)
    ctx.force_variant(cp.V_GROUPED)
    try:
        ctx.gemm_batched(probs, tol=1e-5)
    finally:
        ctx.force_variant(None)
    torch.cuda.synchronize()
    for i in check:
        m, n, k, dt = plist[i]
        A, B, C = keep[i]
        A64 = A.float().cpu().numpy().astype(np.float64)
        B64 = B.float().cpu().numpy().astype(np.float64)
        rows = W.tile_rows(m, seed=i)
        ref = oracle.gemm_rows(A64, B64, rows)
        assert N.rel_frobenius(C.cpu().numpy()[rows], ref) <= 1e-5, (m, n, k, dt)
