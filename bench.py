#!/usr/bin/env python
"""Benchmark of the variant-selecting GEMM on one B300 (or N replicas).

Metric: selected-variant GEMM TFLOP/s at <= 1e-5 relative Frobenius error,
over the FP32-accuracy size sweep: square n = 64, 128, ..., 8192 plus
4096x4096x64 and 16x4096x4096, float32 inputs uniform in [-1, 1) (seeded),
tol = 1e-5.  One step = one compar_gemm call per sweep shape (selection,
operand pre-passes, variant kernel, epilogue).  Throughput = sum of 2MNK over
the sweep / step time.  Every shape has its own A, B, C buffers (about 35 GB
in total), so each step streams far more than the 126 MB L2.

Printed JSON line keys follow the benchmark contract: value (device-resident
inputs), e2e (every shape through compar_gemm_host on page-locked host
buffers: the library's own H2D/D2H inside the timed region), roofline of
the dominant kernel (CUDA-event kernel time inside the timed region), the
CPU oracle baseline, clocks sampled during the timed region, kernel launch
count, and the selector's regret on 200 held-out contexts.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm):
each step is a bounded sample of the same sweep (squares 64..1024).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "selected-variant GEMM TFLOP/s at <=1e-5 rel err vs FP32 SIMT; selector regret %"
WORKLOAD = ("fp32-accuracy size sweep: square n=64..8192 step 64 + 4096x4096x64 + "
            "16x4096x4096, f32 uniform[-1,1] seeded, tol 1e-5, selected variant per call")
TOL = 1e-5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweep", default="full", choices=["full", "pow2"])
    ap.add_argument("--shapes", default=None,
                    help="comma-separated sizes replacing the sweep (profiling runs): "
                         "n for n x n x n, or MxNxK")
    ap.add_argument("--no-regret", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-stencil", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the 512-GEMM batched measurement (profiling runs)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the roofline denominators and exit")
    ap.add_argument("--variants", action="store_true",
                    help="time every variant on the headline shapes and exit")
    ap.add_argument("--selector", default=os.path.join(ROOT, "paper_2311_03543_b300",
                                                        "selector_default.bin"))
    ap.add_argument("--detail", default=None, help="write per-shape detail JSON here")
    ap.add_argument("--online-study", default=None, metavar="SELECTOR_FILE",
                    help="online-selection study: regret of the selector in SELECTOR_FILE on "
                         "held-out contexts before and after a stream of exploring calls")
    ap.add_argument("--cpu-table", action="store_true",
                    help="CPU oracle beside the selected GPU variant on 256^3 .. 8192^3")
    return ap.parse_args()


def flops_of(shapes):
    return sum(2.0 * m * n * k for m, n, k in shapes)


def reduce_max(value, dist, device):
    """The maximum of `value` over all ranks (the slowest replica sets the time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(world, flops_per_rank_step, ms_per_step):
    """Whole-job throughput: every rank's work of one step over the max step time."""
    return world * flops_per_rank_step / (ms_per_step / 1e3) / 1e12


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(budget_s=15.0, shapes=None):
    """Time the FP64 oracle on squares 64, 128, ... until ~budget_s of work."""
    import numpy as np
    import oracle
    import workloads as W
    shapes = shapes or [(n, n, n) for n in range(64, 8193, 64)]
    done, t_total, fl = [], 0.0, 0.0
    for (m, n, k) in shapes:
        A = W.uniform(m, k, seed=2); B = W.uniform(k, n, seed=3)
        t0 = time.perf_counter()
        oracle.gemm(A, B)
        dt = time.perf_counter() - t0
        t_total += dt
        fl += 2.0 * m * n * k
        done.append(m)
        if t_total > budget_s:
            break
    return {"value": fl / t_total / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 triple-loop oracle on squares n={done[0]}..{done[-1]} step 64 "
                      f"({len(done)} GEMMs, {t_total:.1f} s)"}


def cpu_table():
    """FP64 oracle (all host cores) beside the library's selected variant at
    tol 1e-5 on 256^3, 1024^3, 4096^3 (median of 3 CPU runs) and 8192^3 (one
    CPU run); GPU: median of 20 calls, CUDA events, inputs resident."""
    import numpy as np
    import torch
    import oracle
    import paper_2311_03543_b300 as cp
    import workloads as W
    torch.cuda.set_device(0)
    rows = []
    with cp.Context(0) as ctx:
        for n in (256, 1024, 4096, 8192):
            A = W.uniform(n, n, seed=2); B = W.uniform(n, n, seed=3)
            reps = 1 if n == 8192 else 3
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                oracle.gemm(A, B)
                ts.append(time.perf_counter() - t0)
            t_cpu = sorted(ts)[len(ts) // 2]
            dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            C = torch.empty((n, n), device="cuda")
            ctx.gemm(dA, dB, C, tol=TOL)
            v = ctx.last_variant()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(40)]
            for i in range(20):
                ev[2 * i].record()
                ctx.gemm(dA, dB, C, tol=TOL)
                ev[2 * i + 1].record()
            torch.cuda.synchronize()
            t_gpu = sorted(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(20))[10] / 1e3
            fl = 2.0 * n ** 3
            rows.append({"n": n, "cpu_s": t_cpu, "cpu_tflops": fl / t_cpu / 1e12,
                         "cpu_cores": oracle.num_threads(), "gpu_variant": cp.VARIANT_NAMES[v],
                         "gpu_s": t_gpu, "gpu_tflops": fl / t_gpu / 1e12, "speedup": t_cpu / t_gpu})
            print(json.dumps(rows[-1]), flush=True)
    return rows


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        # torchrun gives every rank one OpenMP thread; rank 0 runs alone here,
        # on all of the host's cores (set before the oracle's runtime starts)
        os.environ["OMP_NUM_THREADS"] = str(len(os.sched_getaffinity(0)))
    shapes = [(n, n, n) for n in range(64, 1025, 64)]
    import oracle
    import workloads as W
    mats = [(W.uniform(m, k, seed=2), W.uniform(k, n, seed=3)) for m, n, k in shapes]

    def step():
        for A, B in mats:
            oracle.gemm(A, B)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    fl = flops_of(shapes)
    val = fl / dt / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "squares n=64..1024 step 64 per step"},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "FP64 triple-loop oracle, squares n=64..1024 step 64"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- peaks / variants
def measure_peaks(ctx, torch, dev):
    """Roofline denominators on this GPU: the FP32 FMA pipe (the library's own
    microkernel), dense GEMM peaks of the tensor formats through PyTorch's
    library matmuls (bf16, TF32, FP8 E4M3 via _scaled_mm; 8192^3, best of 10),
    and copy bandwidth (1 GiB, read + write bytes)."""
    out = {"ffma_tflops": ctx.peak_ffma()}
    n = 8192
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def best_of(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = ev(), ev()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)
    x = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
    y = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
    out["bf16_tflops"] = 2 * n ** 3 / (best_of(lambda: x @ y) / 1e3) / 1e12
    xf, yf = x.float(), y.float()
    torch.backends.cuda.matmul.allow_tf32 = True
    out["tf32_tflops"] = 2 * n ** 3 / (best_of(lambda: xf @ yf) / 1e3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        x8 = x.to(torch.float8_e4m3fn)
        y8 = y.to(torch.float8_e4m3fn).t().contiguous().t()
        one = torch.ones((), device=dev)
        out["fp8_tflops"] = 2 * n ** 3 / (best_of(
            lambda: torch._scaled_mm(x8, y8, scale_a=one, scale_b=one,
                                     out_dtype=torch.bfloat16)) / 1e3) / 1e12
    except Exception as e:  # a library without an fp8 path
        out["fp8_tflops"] = None
        out["fp8_note"] = str(e)[:120]
    src = torch.empty(1 << 28, device=dev)
    dst = torch.empty_like(src)
    out["copy_gbs"] = 2 * src.numel() * 4 / (best_of(lambda: dst.copy_(src)) / 1e3) / 1e9
    return out


def measure_variants(ctx, cp, torch, dev, peaks):
    """Every variant forced on the headline shapes: whole-call time (operand
    pre-passes included) and kernel-only time (the library's CUDA-event
    profiler), TFLOP/s, and the fraction of the variant's own roofline:
    min(pipe peak, arithmetic intensity x copy bandwidth)."""
    shapes = [(1024,) * 3, (4096,) * 3, (8192,) * 3, (4096, 4096, 64), (16, 4096, 4096)]
    pipe = {cp.V_NAIVE: peaks["ffma_tflops"], cp.V_SIMT: peaks["ffma_tflops"],
            cp.V_TC_TF32: peaks["tf32_tflops"], cp.V_TC_BF16: peaks["bf16_tflops"],
            cp.V_TC_FP8: peaks.get("fp8_tflops") or 2 * peaks["bf16_tflops"],
            cp.V_SPLIT3: peaks["bf16_tflops"] / 3, cp.V_SPLIT6: peaks["bf16_tflops"] / 6,
            cp.V_SPLIT3_TF32: peaks["tf32_tflops"] / 3,
            cp.V_SPLIT3_FUSED: peaks["bf16_tflops"] / 3}
    rows = []
    for (m, n, k) in shapes:
        g = torch.Generator(device=dev)
        g.manual_seed(m + n + k)
        A = torch.rand((m, k), generator=g, device=dev) * 2 - 1
        B = torch.rand((k, n), generator=g, device=dev) * 2 - 1
        C = torch.empty((m, n), device=dev)
        flops = 2.0 * m * n * k
        for v in range(cp.NUM_VARIANTS):
            if not ctx.supported(v, m, n, k, cp.F32):
                continue
            reps = 3 if (v == cp.V_NAIVE and m * n * k > 2 ** 33) else 10
            ctx.profile_reset()
            ctx.profile_enable(True)
            t_call = ctx.measure(v, A, B, C, tol=1.0, warmup=2, reps=reps)
            ctx.profile_enable(False)
            kms, kn = ctx.profile_read(v)
            t_kern = kms / max(kn, 1)
            byts = 4.0 * (m * k + k * n + m * n)
            roof = min(pipe[v], flops / byts * peaks["copy_gbs"] / 1e3)
            rows.append({"shape": [m, n, k], "variant": cp.VARIANT_NAMES[v],
                         "call_ms": t_call, "kernel_ms": t_kern,
                         "call_tflops": flops / t_call / 1e9,
                         "kernel_tflops": flops / t_kern / 1e9,
                         "roofline_tflops": roof,
                         "kernel_frac_of_roofline": flops / t_kern / 1e9 / roof,
                         "call_gbs": byts / t_call / 1e6})
    return rows


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched_only:
        import torch
        import workloads as W
        import paper_2311_03543_b300 as cp
        torch.cuda.set_device(0)
        with cp.Context(0) as ctx:
            print(json.dumps({"batched_512": measure_batched(ctx, cp, W, torch,
                                                             torch.device("cuda", 0))}),
                  flush=True)
        return 0
    if args.cpu_table:
        print(json.dumps({"cpu_vs_gpu": cpu_table()}), flush=True)
        return 0
    if args.online_study:
        import torch
        import workloads as W
        import paper_2311_03543_b300 as cp
        torch.cuda.set_device(0)
        with cp.Context(0) as ctx:
            print(json.dumps({"online_study": online_study(ctx, cp, W, torch,
                                                           torch.device("cuda", 0),
                                                           args.online_study)}), flush=True)
        return 0
    if args.peaks or args.variants:
        import torch
        import paper_2311_03543_b300 as cp
        torch.cuda.set_device(0)
        dev = torch.device("cuda", 0)
        with cp.Context(0) as ctx:
            peaks = measure_peaks(ctx, torch, dev)
            out = {"peaks": peaks}
            if args.variants:
                out["variants"] = measure_variants(ctx, cp, torch, dev, peaks)
        print(json.dumps(out), flush=True)
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump(out, f, indent=1)
        return 0
    import torch
    import workloads as W
    import paper_2311_03543_b300 as cp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    shapes = W.sweep_shapes() if args.sweep == "full" else W.pow2_sweep_shapes()
    if args.shapes:   # "4096" (square) or "4096x4096x64" (M x N x K)
        shapes = [tuple(int(x) for x in s.split("x")) if "x" in s else (int(s),) * 3
                  for s in args.shapes.split(",")]
    ctx = cp.Context(dev.index)
    if os.path.exists(args.selector):
        ctx.selector_load(args.selector)
    stream = torch.cuda.current_stream()
    ctypes_stream = __import__("ctypes").c_void_p(stream.cuda_stream)

    # inputs: one seeded buffer set per shape, created on the device
    gen = torch.Generator(device=dev)
    bufs = []
    for i, (m, n, k) in enumerate(shapes):
        gen.manual_seed(1000 * (rank + 1) + i)
        A = torch.rand((m, k), generator=gen, device=dev) * 2 - 1
        B = torch.rand((k, n), generator=gen, device=dev) * 2 - 1
        C = torch.empty((m, n), device=dev)
        bufs.append((A, B, C))

    def step():
        for (m, n, k), (A, B, C) in zip(shapes, bufs):
            rc = cp.compar_gemm(ctx.handle, m, n, k, cp.F32, TOL, A.data_ptr(), B.data_ptr(),
                                C.data_ptr(), ctypes_stream)
            if rc != 0:
                raise cp.ComparError(rc, f"compar_gemm {m}x{n}x{k}")

    # warm-up (first step fills the decision cache and grows the workspace)
    picks = []
    for (m, n, k), (A, B, C) in zip(shapes, bufs):
        ctx.gemm(A, B, C, tol=TOL)
        picks.append(ctx.last_variant())
    for _ in range(max(args.warmup - 1, 0)):
        step()
    torch.cuda.synchronize()

    # timed region
    ctx.profile_reset()
    ctx.profile_enable(True)
    sampler = ClockSampler(dev.index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = cp.compar_launch_count()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = cp.compar_launch_count() - launches0
    if dist:
        dist.barrier()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, dist, dev)
    ctx.profile_enable(False)
    fl_step = flops_of(shapes)
    value = whole_job_tflops(world, fl_step, ms)

    # dominant kernel and its roofline
    prof = {v: ctx.profile_read(v) for v in range(cp.NUM_VARIANTS)}
    dom = max(prof, key=lambda v: prof[v][0])
    dom_ms, dom_n = prof[dom]
    pieces = {cp.V_SPLIT3: 3, cp.V_SPLIT6: 6, cp.V_SPLIT3_FUSED: 3,
              cp.V_SPLIT3_TF32: 3}.get(dom, 1)
    dom_flops = args.steps * sum(2.0 * m * n * k * pieces
                                 for (m, n, k), v in zip(shapes, picks) if v == dom)
    achieved = dom_flops / (dom_ms / 1e3) / 1e12 if dom_ms > 0 else 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    if dom in (cp.V_NAIVE, cp.V_SIMT):
        peak, bound, src = ctx.peak_ffma(), "alu", "measured FFMA loop (compar_peak_ffma)"
    else:
        scale = {cp.V_TC_TF32: 0.5, cp.V_SPLIT3_TF32: 0.5, cp.V_TC_FP8: 2.0}.get(dom, 1.0)
        base = peaks.get("bf16_tflops_sustained")
        src = "measured bf16 sustained (MEASURED_PEAKS.json)"
        if base is None:
            base, src = 1400.0, "fallback bf16 sustained"
        peak, bound = base * scale, "tensor"
        if scale != 1.0:
            src += f" x nominal ratio {scale}"
    traffic, traffic_note = measured_traffic(cp.VARIANT_NAMES[dom], dom_flops / max(dom_n, 1))
    roofline = {"bound": bound, "kernel": cp.VARIANT_NAMES[dom], "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                "traffic": traffic, "traffic_note": traffic_note,
                "peak_source": src + (" (of fallback)" if src.startswith("fallback")
                                      else " (of measured)"), "launches": dom_n,
                "kernel_ms_per_step": dom_ms / args.steps,
                "share_of_step": (dom_ms / args.steps) / ms if ms else None}

    # end-to-end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        mx = max(max(m * k, k * n, m * n) for m, n, k in shapes)
        hA = torch.empty(mx, dtype=torch.float32, pin_memory=True).uniform_(-1, 1)
        hB = torch.empty(mx, dtype=torch.float32, pin_memory=True).uniform_(-1, 1)
        hC = torch.empty(mx, dtype=torch.float32, pin_memory=True)
        h2d = sum((m * k + k * n) * 4 for m, n, k in shapes)
        d2h = sum(m * n * 4 for m, n, k in shapes)

        # Every shape through the library's host-buffer call: it uploads A
        # and B, runs the selected variant per row panel and downloads C,
        # overlapping the transfers with the products (and consecutive calls
        # with each other through its two device buffer sets).
        def e2e_step():
            for (m, n, k) in shapes:
                rc = cp.compar_gemm_host(ctx.handle, m, n, k, cp.F32, TOL, hA.data_ptr(),
                                         hB.data_ptr(), hC.data_ptr(), ctypes_stream)
                if rc != 0:
                    raise cp.ComparError(rc, "compar_gemm_host (e2e)")
        e2e_step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        ems = reduce_max(f0.elapsed_time(f1) / args.steps, dist, dev)
        e2e = {"value": whole_job_tflops(world, fl_step, ems), "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ems}

    # selector regret against exhaustive measurement (held-out contexts)
    regret = None
    if not args.no_regret and rank == 0:
        r_pct, r_viol, r_n, r_worst = measure_regret(ctx, cp, W, torch, dev)
        t_pct, t_viol, t_n, t_worst = measure_regret(ctx, cp, W, torch, dev, count=50,
                                                     contexts=W.heldout_tight_contexts())
        regret = {"mean_pct": r_pct, "violations": r_viol, "contexts": r_n, "worst": r_worst,
                  "set": "held-out contexts 0..199 (M,N,K log-uniform [16,4096], f32/bf16/fp8, "
                         "tol 1e-5/1e-3/1e-1)", "feasibility": "library FP64 residual check, 8 rows",
                  "tight": {"mean_pct": t_pct, "violations": t_viol, "contexts": t_n,
                            "worst": t_worst,
                            "set": "f32 contexts 0..49 at tol 1e-6 (same shape law)"}}

    batched = None
    if not args.no_batched and rank == 0:
        batched = measure_batched(ctx, cp, W, torch, dev)

    stencil = None
    if not args.no_stencil and rank == 0:
        stencil = measure_stencil(ctx, cp, W, torch, dev)

    accuracy = None
    if not args.no_accuracy and rank == 0:
        accuracy = measure_accuracy(ctx, cp, W, torch, dev)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_sample()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "shapes": len(shapes),
                           "gflop_per_step": fl_step / 1e9, "tol": TOL,
                           "l2": "inputs larger than L2 (distinct buffers per shape, "
                                 f"{sum((m*k+k*n+m*n)*4 for m,n,k in shapes)/1e9:.1f} GB per step)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "selected": {cp.VARIANT_NAMES[v]: picks.count(v)
                                        for v in sorted(set(picks))}},
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e,
                "gpu_launches": launches, "regret_pct": regret, "batched_512": batched,
                "stencil": stencil, "accuracy": accuracy}
        print(json.dumps(line), flush=True)
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump({"shapes": shapes, "picks": picks, "line": line}, f)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def measured_traffic(kernel, flops_per_launch):
    """DRAM bytes per launch from the committed ncu capture, scaled to the
    average launch by work (GEMM traffic grows with 2MNK at fixed tiles); None
    when there is no capture or the kernel source changed since it was taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except (OSError, ValueError, KeyError):
        return None, "no ncu capture for this kernel"
    h = hashlib.sha1()
    for f in ("gemm_tc.cu", "ptx.cuh", "epilogue.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2311_03543_b300", "csrc", f), "rb").read())
    if h.hexdigest() != rec["src_sha1"]:
        return None, "kernel changed since the ncu capture"
    m, n, k = rec["shape"]
    products = {"split-3xbf16": 3, "split-6xbf16": 6, "split-3xtf32": 3,
                "split-3xbf16-fused": 3}.get(kernel, 1)
    scale = flops_per_launch / (2.0 * m * n * k * products)
    return (rec["dram_bytes_per_launch"] * scale,
            f"ncu dram read+write of one {m}x{n}x{k} launch ({rec['source']}) scaled by work "
            f"to the average launch (x{scale:.3f})")


def measure_batched(ctx, cp, W, torch, dev, reps=5):
    """The uneven batched workload: 512 GEMMs, M, N, K log-uniform in [32, 2048]
    (seed 5), f32 (tol 1e-5 -> 3xBF16) or bf16 with probability 1/2, every
    leading dimension rounded up to 16 bytes.  The autotuner times the
    per-GEMM loop and the grouped kernel's configurations; then the chosen one
    and the loop are each timed over `reps` calls."""
    import ctypes
    plist = W.batched_problems()
    keep, probs = [], []
    for i, (m, n, k, dt) in enumerate(plist):
        g = torch.Generator(device=dev)
        g.manual_seed(5000 + i)
        per16 = 8 if dt == cp.BF16 else 4            # elements per 16 bytes
        lda, ldb, ldc = -(-k // per16) * per16, -(-n // per16) * per16, -(-n // 4) * 4
        A = torch.rand((m, lda), generator=g, device=dev) * 2 - 1
        B = torch.rand((k, ldb), generator=g, device=dev) * 2 - 1
        if dt == cp.BF16:
            A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
        C = torch.empty((m, ldc), device=dev)
        keep.append((A, B, C))
        probs.append(dict(m=m, n=n, k=k, lda=lda, ldb=ldb, ldc=ldc, dtype=dt, A=A.data_ptr(),
                          B=B.data_ptr(), C=C.data_ptr()))
    arr = cp.Context.problem_array(probs)
    best, tuned_ms = ctx.autotune_batched(arr, tol=TOL)
    stream = torch.cuda.current_stream()

    def timed(force):
        ctx.force_variant(force)
        try:
            ctx.gemm_batched(arr, tol=TOL)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ctx.gemm_batched(arr, tol=TOL)
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            ctx.force_variant(None)
        return e0.elapsed_time(e1) / reps

    ms_best = timed(None)                      # the autotuned choice
    ms_loop = tuned_ms[0]                      # per-GEMM launches (autotuner's median)
    flops = sum(2.0 * m * n * k for m, n, k, _ in plist)
    # tensor-pipe work: a float32 problem at tol 1e-5 runs as 3xBF16 (three
    # bf16 products per useful product), a bf16 problem as one
    bf16_work = sum(2.0 * m * n * k * (3 if dt == cp.F32 else 1) for m, n, k, dt in plist)
    del keep
    names = ["per-GEMM launches", "grouped BN=128", "grouped BN=256",
             "grouped BN=128 largest-first", "grouped BN=256 largest-first"]
    roof = {"bound": "tensor", "unit": "TFLOP/s",
            "achieved": bf16_work / (ms_best / 1e3) / 1e12,
            "work": "bf16 MMA work: 2MNK per bf16 problem, 3 x 2MNK per float32 (3xBF16) problem"}
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        roof["peak"] = pk["bf16_tflops_sustained"]
        roof["peak_source"] = "measured bf16 sustained (MEASURED_PEAKS.json) (of measured)"
        roof["frac_of_burst"] = roof["achieved"] / pk["bf16_tflops"]
    except (OSError, ValueError, KeyError):
        roof["peak"], roof["peak_source"] = 1400.0, "fallback 1.4 PFLOP/s sustained (of fallback)"
    roof["frac"] = roof["achieved"] / roof["peak"]
    return {"problems": len(plist), "gflop": flops / 1e9, "ld": "rounded up to 16 bytes",
            "chosen": names[best],
            "ms_chosen": ms_best, "tflops_chosen": flops / (ms_best / 1e3) / 1e12,
            "ms_per_gemm_launches": ms_loop,
            "tflops_per_gemm_launches": flops / (ms_loop / 1e3) / 1e12,
            "autotune_ms": dict(zip(names, tuned_ms)), "roofline": roof}


def measure_accuracy(ctx, cp, W, torch, dev, nrows=32):
    """The metric's error, both ways, outside the timed region: for a few sweep
    shapes (f32 uniform[-1,1], seeded), the variant selected at the metric's
    tolerance is checked (a) against FP64 products of `nrows` sampled rows by
    the library's residual check, the gate, and (b) against the forced FP32
    SIMT variant's output on the same inputs (relative Frobenius difference
    over all of C), the metric's wording."""
    out = []
    for i, (m, n, k) in enumerate([(256, 256, 256), (1024, 1024, 1024), (4096, 4096, 4096),
                                   (4096, 4096, 64), (16, 4096, 4096)]):
        g = torch.Generator(device=dev)
        g.manual_seed(900 + i)
        A = torch.rand((m, k), generator=g, device=dev) * 2 - 1
        B = torch.rand((k, n), generator=g, device=dev) * 2 - 1
        C = torch.empty((m, n), device=dev)
        ctx.gemm(A, B, C, tol=TOL)
        v = ctx.last_variant()
        fp64 = ctx.residual_check(A, B, C, nrows=nrows, seed=7 + i)
        S = torch.empty_like(C)
        ctx.force_variant(cp.V_SIMT)
        try:
            ctx.gemm(A, B, S, tol=TOL)
        finally:
            ctx.force_variant(None)
        vs_simt = float((C.double() - S.double()).norm() / S.double().norm())
        out.append({"shape": f"{m}x{n}x{k}", "variant": cp.VARIANT_NAMES[v],
                    "rel_err_vs_fp64_rows": fp64, "rel_err_vs_fp32_simt": vs_simt})
    return {"tol": TOL, "fp64_rows": nrows, "shapes": out}


def measure_stencil(ctx, cp, W, torch, dev, reps=5):
    """The thermal-stencil component on its headline workload (8192 x 8192
    grid, 100 steps, seeded chip on the device): the selected variant timed
    over `reps` calls after two warm-ups (CUDA events; three grids of 268 MB,
    larger than L2), every variant timed for context, and the roofline of the
    selected one: HBM for the naive variant (12 bytes per cell and step); for
    temporal blocking the FP32 pipe, which bounds it once a warp's row moves
    through shared memory in 16-byte pieces (the instruction issue is the
    limit: 10 FP32 operations per cell and step, counted once per cell of the
    grid, against the FP32 lane-operation rate of the library's measured FFMA
    loop, near the 148 SMs x 128 lanes x 2032 MHz = 38.5 T operations/s of the
    data sheet; the kernel also recomputes the 128 x 80 region of every
    112 x 64 tile, x1.43)."""
    rows, cols, iters = W.STENCIL_HEADLINE
    prm = cp.Context.stencil_params(**W.STENCIL_PARAMS)
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    T = torch.rand((rows, cols), generator=g, device=dev) * 20 + 80
    P = torch.rand((rows, cols), generator=g, device=dev)
    out = torch.empty_like(T)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ctx.stencil(T, P, out, iters, prm)
    chosen = ctx.stencil_last_variant()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.stencil(T, P, out, iters, prm)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    per_variant = {cp.STENCIL_NAMES[v]: ctx.stencil_measure(v, T, P, out, iters, prm, warmup=1,
                                                            reps=3)
                   for v in range(cp.NUM_STENCIL_VARIANTS) if ctx.stencil_supported(v, rows, cols)}
    cell_steps = float(rows) * cols * iters
    if chosen == cp.S_NAIVE:
        roof = {"bound": "hbm", "unit": "GB/s", "achieved": cell_steps * 12 / (ms / 1e3) / 1e9}
        try:
            roof["peak"] = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
            roof["peak_source"] = "measured copy bandwidth (MEASURED_PEAKS.json)"
        except (OSError, ValueError, KeyError):
            roof["peak"], roof["peak_source"] = 6400.0, "fallback 6.4 TB/s"
    else:
        # FP32 lane operations per second of the measured FFMA loop (an FMA
        # counts once here, as in the 10 operations per cell and step)
        region = (128.0 * 80.0) / (112.0 * 64.0)
        roof = {"bound": "alu", "unit": "Tops/s",
                "achieved": cell_steps * 10 / (ms / 1e3) / 1e12, "peak": ctx.peak_ffma() / 2,
                "peak_source": "measured FFMA loop (compar_peak_ffma, FMA instructions x 32 "
                               "lanes per second) (of measured)",
                "derived_peak": 38.5, "derived_source": "148 SMs x 128 FP32 lanes x 2032 MHz",
                "with_halo": cell_steps * 10 * region / (ms / 1e3) / 1e12}
    roof["frac"] = roof["achieved"] / roof["peak"]
    return {"workload": f"thermal stencil {rows}x{cols}, {iters} steps, seeded chip",
            "chosen": cp.STENCIL_NAMES[chosen], "ms": ms,
            "gcells_per_s": cell_steps / (ms / 1e3) / 1e9, "variants_ms": per_variant,
            "roofline": roof}


def measure_regret(ctx, cp, W, torch, dev, count=200, contexts=None):
    """Mean regret (%) of the selector on held-out contexts vs exhaustive timing.

    The first `count` held-out contexts (M, N, K log-uniform in [16, 4096],
    dtype f32/bf16/fp8, tol 1e-5/1e-3/1e-1; never used in training).  Every
    eligible variant is timed with compar_measure; its error is the library's
    FP64 residual check on 8 rows.  best = fastest feasible variant (ties
    within 2 % go to the lower id); regret = t(pick)/t(best) - 1, and an
    infeasible pick costs a rerun.  A context whose regret exceeds 10 % has
    its pick and its best variant timed once more (each keeps its faster
    time).  Returns (regret %, violations, contexts, worst context).
    """
    import numpy as np
    tie = 0.02
    rs, viol, worst = [], 0, None
    judge = cp.Context(dev.index)   # measures; the selector's history never sees it
    contexts = W.heldout_contexts() if contexts is None else contexts
    for i, (m, n, k, dt, tol) in enumerate(contexts[:count]):
        g = torch.Generator(device=dev)
        g.manual_seed(90000 + i)
        A = torch.rand((m, k), generator=g, device=dev) * 2 - 1
        B = torch.rand((k, n), generator=g, device=dev) * 2 - 1
        if dt == cp.BF16:
            A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
        elif dt == cp.F8E4M3:
            A = A.to(torch.float8_e4m3fn).view(torch.uint8)
            B = B.to(torch.float8_e4m3fn).view(torch.uint8)
        C = torch.empty((m, n), device=dev)
        ctx.clear_decisions()
        pick = ctx.select(m, n, k, dt, tol)
        times, feas = {}, set()
        for v in range(cp.NUM_VARIANTS):
            if not judge.supported(v, m, n, k, dt):
                continue
            times[v] = judge.measure(v, A, B, C, tol=tol, warmup=1, reps=3, dtype=dt)
            if judge.residual_check(A, B, C, nrows=8, seed=i, dtype=dt) <= tol:
                feas.add(v)
        if not feas:
            continue

        def regret():
            t_best = min(times[v] for v in feas)
            if pick not in feas:
                return (times[pick] + t_best) / t_best - 1.0
            return 0.0 if times[pick] <= t_best * (1 + tie) else times[pick] / t_best - 1.0

        r = regret()
        if r > 0.1:
            # a large gap: time the pick and the fastest feasible variant once
            # more (5 repetitions) and keep each one's faster measurement, so a
            # single disturbed timing does not decide the context
            best = min(feas, key=lambda v: times[v])
            for v in {pick, best}:
                times[v] = min(times[v], judge.measure(v, A, B, C, tol=tol, warmup=1, reps=5,
                                                       dtype=dt))
            r = regret()
        viol += pick not in feas
        rs.append(r)
        if worst is None or r > worst["pct"] / 100.0:
            best = min(feas, key=lambda v: times[v])
            worst = {"context": i, "m": m, "n": n, "k": k, "dtype": int(dt), "tol": tol,
                     "pick": int(pick), "best": int(best), "feasible": sorted(int(v) for v in feas),
                     "times_us": {int(v): 1e3 * t for v, t in times.items()},
                     "pct": 100.0 * r}
    judge.close()
    return 100.0 * float(np.mean(rs)), viol, len(rs), worst


def online_study(ctx, cp, W, torch, dev, selector, count=120, calls=800):
    """Online selection (exploration and warm-start fine-tuning) from a
    selector that has not seen the call distribution: its mean regret on the
    first `count` held-out contexts, then `calls` calls drawn from the same
    law with another seed (54321) made with exploration probability 0.25 and
    a 300-step fine-tune every 100 new timing records, then the regret on the same
    held-out contexts again (exploration off)."""
    ctx.selector_load(selector)
    before = measure_regret(ctx, cp, W, torch, dev, count=count)
    ctx.set_online(epsilon=0.25, retrain_every=100, finetune_steps=300)
    for i, (m, n, k, dt, tol) in enumerate(W.heldout_contexts(count=calls, seed=54321)):
        g = torch.Generator(device=dev)
        g.manual_seed(70000 + i)
        A = torch.rand((m, k), generator=g, device=dev) * 2 - 1
        B = torch.rand((k, n), generator=g, device=dev) * 2 - 1
        if dt == cp.BF16:
            A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
        elif dt == cp.F8E4M3:
            A = A.to(torch.float8_e4m3fn).view(torch.uint8)
            B = B.to(torch.float8_e4m3fn).view(torch.uint8)
        C = torch.empty((m, n), device=dev)
        ctx.gemm(A, B, C, tol=tol, dtype=dt)
    torch.cuda.synchronize()
    explored, retrains, rejected = ctx.online_stats()
    ctx.set_online(0.0, 0, 0)
    after = measure_regret(ctx, cp, W, torch, dev, count=count)
    return {"selector": os.path.basename(selector), "contexts": after[2], "calls": calls,
            "explored": explored, "fine_tunes": retrains, "fine_tunes_discarded": rejected,
            "regret_before_pct": before[0], "violations_before": before[1],
            "regret_after_pct": after[0], "violations_after": after[1]}


if __name__ == "__main__":
    sys.exit(main())
