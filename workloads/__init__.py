"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws numbers and lists shapes.  It holds none of the
method's arithmetic (no GEMM, no rounding to a low-precision format, no
selection rule), so the CUDA path and the oracle can both take their inputs
from it without sharing any computation.

The paper's matrix-multiply application scales a square size N from 8 to 8192
(Table 2); its inputs are not published, so every matrix here is drawn from a
seeded NumPy ``default_rng`` (PCG64) stream.

Workloads (M, N, K):

* ``PARITY_256``: one 256^3 FP32 product, A and B uniform[-1, 1] (seed 1).
* ``sweep_shapes()``: FP32-accuracy size sweep, square n = 64, 128, ..., 8192
  (step 64) plus the skinny 4096x4096x64 and 16x4096x4096 (seed 2).
* precision study: 4096^3, normal(0, 1) (seed 3); ill-scaled variant multiplies
  column k of A by 10^u, u ~ U(-3, 3) (seed 4).
* ``batched_problems()``: 512 GEMMs, M, N, K each round(exp(U(ln 32,
  ln 2048))) (seed 5), dtype f32 or bf16 with probability 1/2.
* ``heldout_contexts()``: selector test contexts, M, N, K log-uniform
  integers in [16, 4096], dtype uniform over {f32, bf16, fp8}, tolerance from
  {1e-5 (f32 only), 1e-3, 1e-1} (seed 12345); ``heldout_tight_contexts()``:
  float32 only at tolerance 1e-6, same shape law (seed 24680).
* thermal stencil: ``stencil_inputs()`` (seeded chip: temperature, power map
  with hot blocks), ``STENCIL_PARAMS``, ``stencil_contexts()`` (grid sizes
  64 - 8192, 1 - 1000 iterations; training and held-out seeds differ).
"""
import math

import numpy as np

F32, BF16, F8E4M3 = 0, 1, 2
DTYPE_NAMES = {F32: "f32", BF16: "bf16", F8E4M3: "f8e4m3"}


def rng(seed):
    return np.random.default_rng(seed)


def uniform(rows, cols, seed, lo=-1.0, hi=1.0):
    """float32 (rows, cols) matrix, entries uniform in [lo, hi)."""
    return rng(seed).uniform(lo, hi, size=(rows, cols)).astype(np.float32)


def normal(rows, cols, seed):
    """float32 (rows, cols) matrix, entries normal(0, 1)."""
    return rng(seed).standard_normal(size=(rows, cols)).astype(np.float32)


def column_scales(cols, seed, decades=3.0):
    """Per-column factors 10^u, u ~ U(-decades, decades), float32."""
    u = rng(seed).uniform(-decades, decades, size=cols)
    return (10.0 ** u).astype(np.float32)


def ill_scaled(rows, cols, seed_values, seed_scales):
    """normal(0,1) matrix whose column k is multiplied by 10^U(-3, 3)."""
    return (normal(rows, cols, seed_values)
            * column_scales(cols, seed_scales)[None, :]).astype(np.float32)


def integer_matrix(rows, cols, seed, bound=8):
    """Integers in [-bound, bound] as float32 (exactly representable)."""
    return rng(seed).integers(-bound, bound + 1, size=(rows, cols)).astype(np.float32)


def bf16_input(rows, cols, seed):
    """bfloat16 input matrix as uint16 bit patterns.

    Drawn as uniform[-1, 1) float32 whose low 16 bits are cleared, so every
    value is a bfloat16 number; no rounding rule is applied.
    """
    x = uniform(rows, cols, seed)
    return (x.view(np.uint32) >> 16).astype(np.uint16)


def fp8_input(rows, cols, seed, max_exponent_field=10):
    """FP8 E4M3 input matrix as byte codes.

    Random sign, exponent field in [0, max_exponent_field] and fraction bits;
    exponent fields at most 14 never form the NaN code, so every code is a
    finite E4M3 number (magnitudes up to 2^(max_exponent_field-7)*1.875).
    """
    g = rng(seed)
    sign = g.integers(0, 2, size=(rows, cols)).astype(np.uint8) << 7
    expo = g.integers(0, max_exponent_field + 1, size=(rows, cols)).astype(np.uint8) << 3
    frac = g.integers(0, 8, size=(rows, cols)).astype(np.uint8)
    return (sign | expo | frac).astype(np.uint8)


PARITY_256 = (256, 256, 256)


def sweep_shapes(step=64, top=8192):
    """The FP32-accuracy sweep: squares step..top (step) plus two skinny shapes."""
    sq = [(n, n, n) for n in range(step, top + 1, step)]
    return sq + [(4096, 4096, 64), (16, 4096, 4096)]


def pow2_sweep_shapes():
    """Headline subset of the sweep: powers of two 64..8192 plus the skinny shapes."""
    return [(1 << e,) * 3 for e in range(6, 14)] + [(4096, 4096, 64), (16, 4096, 4096)]


def _log_uniform_int(g, lo, hi, size):
    return np.rint(np.exp(g.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def batched_problems(count=512, seed=5, lo=32, hi=2048):
    """List of (m, n, k, dtype) for the uneven batched workload."""
    g = rng(seed)
    mnk = _log_uniform_int(g, lo, hi, (count, 3))
    dt = np.where(g.uniform(size=count) < 0.5, F32, BF16)
    return [(int(a), int(b), int(c), int(d)) for (a, b, c), d in zip(mnk, dt)]


def heldout_contexts(count=2000, seed=12345, lo=16, hi=4096):
    """List of (m, n, k, dtype, tol) held out from selector training."""
    g = rng(seed)
    mnk = _log_uniform_int(g, lo, hi, (count, 3))
    dts = g.integers(0, 3, size=count)
    out = []
    for (m, n, k), d in zip(mnk, dts):
        if d == F32:
            tol = [1e-5, 1e-3, 1e-1][int(g.integers(0, 3))]
        else:
            tol = [1e-3, 1e-1][int(g.integers(0, 2))]
        out.append((int(m), int(n), int(k), int(d), float(tol)))
    return out


def heldout_tight_contexts(count=300, seed=24680, lo=16, hi=4096):
    """Float32 contexts at tolerance 1e-6 (below 3xBF16's error level),
    held out from selector training: (m, n, k, dtype, tol)."""
    g = rng(seed)
    mnk = _log_uniform_int(g, lo, hi, (count, 3))
    return [(int(m), int(n), int(k), F32, 1e-6) for (m, n, k) in mnk]


def training_contexts(count, seed=777, lo=16, hi=8192):
    """Selector training contexts (seed disjoint from the held-out set)."""
    return heldout_contexts(count=count, seed=seed, lo=lo, hi=hi)


# ---------------------------------------------------------------- stencil
# Thermal-stencil workload (the hotspot-like component; Table 2 lists Hotspot
# on square grids 64 - 8192).  Rodinia's input files are not available, so a
# seeded chip stands in: ambient 80, an initial temperature 80 + U(0, 20), a
# background power U(0, 1) and a few hot rectangular blocks of U(5, 20).
STENCIL_PARAMS = {"c": 0.2, "gx": 0.5, "gy": 0.5, "gz": 0.01, "amb": 80.0}
STENCIL_HEADLINE = (8192, 8192, 100)   # rows, cols, iterations


def stencil_inputs(rows, cols, seed, hot_blocks=6):
    """(T0, P) float32 arrays of shape rows x cols."""
    g = rng(seed)
    T0 = (80.0 + g.uniform(0.0, 20.0, size=(rows, cols))).astype(np.float32)
    P = g.uniform(0.0, 1.0, size=(rows, cols))
    for _ in range(hot_blocks):
        h = max(1, int(rows * g.uniform(0.05, 0.2)))
        w = max(1, int(cols * g.uniform(0.05, 0.2)))
        r0 = int(g.integers(0, max(1, rows - h + 1)))
        c0 = int(g.integers(0, max(1, cols - w + 1)))
        P[r0:r0 + h, c0:c0 + w] += g.uniform(5.0, 20.0)
    return T0, P.astype(np.float32)


def stencil_contexts(count, seed, lo=64, hi=8192, it_lo=1, it_hi=1000):
    """(rows, cols, iters): sizes log-uniform in [lo, hi], iterations
    log-uniform in [it_lo, it_hi]."""
    g = rng(seed)
    rc = _log_uniform_int(g, lo, hi, (count, 2))
    it = _log_uniform_int(g, it_lo, it_hi, count)
    return [(int(r), int(c), int(i)) for (r, c), i in zip(rc, it)]


def sample_rows(m, count, seed):
    """Sorted distinct row indices for checking large products row by row."""
    count = min(count, m)
    return np.sort(rng(seed).choice(m, size=count, replace=False)).astype(np.int64)


def tile_rows(m, seed, tile=128, inner=1):
    """Sorted distinct row indices that reach every block of `tile` rows:
    each block's first and last row (the last block may be ragged) plus
    `inner` seeded rows inside it.  A fault confined to one row tile of an
    output (one CTA's work, one lane quarter of it) then meets a checked
    row."""
    g = rng(seed)
    rows = set()
    for r0 in range(0, m, tile):
        r1 = min(m, r0 + tile) - 1
        rows.update((r0, r1))
        if r1 - r0 > 1 and inner:
            rows.update(int(x) for x in g.integers(r0 + 1, r1, size=inner))
    return np.array(sorted(rows), dtype=np.int64)
