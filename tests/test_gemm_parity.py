"""Parity of every GEMM variant with the FP64 oracle (GPU, through the C ABI).

Tolerances (relative Frobenius error):
* FP32-accurate variants (naive, SIMT, 3xBF16, 6-product split, 3xTF32) on
  float32 inputs: <= 1e-5 against the oracle on the float32 values; the
  6-product split and 3xTF32 also <= 2e-6 (their pieces hold 24 / 22 bits
  and the dropped terms are ~2^-26 / 2^-22 relative).
* BF16 / FP8 tensor-core variants: <= 1e-5 against the oracle evaluated on
  the exact values the kernel multiplies (its inputs as given, or the oracle's
  own bf16 rounding / e4m3 quantisation of the float32 inputs) — only FP32
  accumulation error remains; the total error against the float32 values is
  reported and bounded by the format's rounding (2^-8, 2^-4 relative).
* TF32 (tensor cores read 10 fraction bits): total error <= 2e-3.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import numerics as N

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_SPLIT6 = 2e-6


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_03543_b300 as cp
    c = cp.Context(0)
    yield c
    c.close()


def _run(ctx, v, A, B, dtype=None, alpha=1.0, beta=0.0, C0=None, tol=0.0, pairs=-1):
    from gpu_util import dev, empty_c, host
    import paper_2311_03543_b300 as cp
    m, n = A.shape[0], B.shape[1]
    C = dev(C0.astype(np.float32)) if C0 is not None else empty_c(m, n)
    ctx.set_scalars(alpha, beta)
    ctx.force_variant(v)
    ctx.set_tc_pairs(pairs)
    try:
        ctx.gemm(dev(A), dev(B), C, tol=tol, dtype=dtype)
        out = host(C)
    finally:
        ctx.force_variant(None)
        ctx.set_scalars(1.0, 0.0)
        ctx.set_tc_pairs(-1)
    assert ctx.check_device_error() == cp.OK
    return out


SHAPES = [(1, 1, 1), (3, 5, 7), (16, 16, 16), (33, 65, 17), (127, 129, 130),
          (255, 257, 256), (256, 256, 256), (300, 200, 1000), (129, 520, 64)]


@pytest.mark.parametrize("v", [0, 1, 5, 7, 8])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_fp32_accurate_variants(ctx, v, m, n, k):
    from gpu_util import assert_elementwise, elem_bound
    A = W.uniform(m, k, seed=100 + m); B = W.uniform(k, n, seed=200 + n)
    got = _run(ctx, v, A, B)
    ref = oracle.gemm(A, B)
    assert N.rel_frobenius(got, ref) <= (TOL_SPLIT6 if v in (7, 8) else TOL_F32)
    assert_elementwise(got, ref, oracle.gemm(np.abs(A), np.abs(B)), elem_bound(v, k))


def test_config1_naive_then_simt(ctx):
    """256^3, uniform[-1,1] seed 1, alpha=1 beta=0; naive and SIMT forced in turn."""
    m, n, k = W.PARITY_256
    A = W.uniform(m, k, seed=1); B = W.uniform(k, n, seed=1001)
    ref = oracle.gemm(A, B)
    for v in (0, 1):
        assert N.rel_frobenius(_run(ctx, v, A, B), ref) <= TOL_F32


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 40, 9), (128, 256, 64), (200, 300, 333),
                                   (256, 512, 1024)])
def test_tf32_total_error(ctx, m, n, k):
    from gpu_util import assert_elementwise, elem_bound
    A = W.uniform(m, k, seed=3 + m); B = W.uniform(k, n, seed=4 + n)
    got = _run(ctx, 2, A, B)
    err = N.rel_frobenius(got, oracle.gemm(A, B))
    assert err <= 2e-3
    absp = oracle.gemm(np.abs(A), np.abs(B))
    assert_elementwise(got, oracle.gemm(A, B), absp, elem_bound(2, k))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 40, 9), (128, 256, 64), (200, 300, 333),
                                   (256, 512, 1024)])
def test_bf16_on_f32_inputs(ctx, m, n, k):
    from gpu_util import assert_elementwise, elem_bound
    A = W.uniform(m, k, seed=5 + m); B = W.uniform(k, n, seed=6 + n)
    got = _run(ctx, 3, A, B)
    Ar, Br = N.bf16_round(A), N.bf16_round(B)
    exact_inputs = oracle.gemm(Ar, Br)
    assert N.rel_frobenius(got, exact_inputs) <= TOL_F32
    assert N.rel_frobenius(got, oracle.gemm(A, B)) <= 2.0 ** -7
    assert_elementwise(got, exact_inputs, oracle.gemm(np.abs(Ar), np.abs(Br)), elem_bound(3, k))


@pytest.mark.parametrize("m,n,k", [(1, 1, 8), (17, 40, 24), (128, 256, 64), (200, 300, 336),
                                   (256, 512, 1024), (100, 90, 13)])
def test_bf16_native_inputs(ctx, m, n, k):
    import paper_2311_03543_b300 as cp
    A = W.bf16_input(m, k, seed=7 + m); B = W.bf16_input(k, n, seed=8 + n)
    got = _run(ctx, 3, A, B, dtype=cp.BF16)
    ref = oracle.gemm(N.bf16_to_f32(A), N.bf16_to_f32(B))
    assert N.rel_frobenius(got, ref) <= TOL_F32


@pytest.mark.parametrize("m,n,k", [(1, 1, 16), (17, 40, 48), (128, 256, 128), (200, 300, 336),
                                   (256, 512, 1024), (100, 90, 13)])
def test_fp8_native_inputs_with_scales(ctx, m, n, k):
    import paper_2311_03543_b300 as cp
    A = W.fp8_input(m, k, seed=9 + m); B = W.fp8_input(k, n, seed=10 + n)
    ctx.set_fp8_scales(0.5, 0.25)
    try:
        got = _run(ctx, 4, A, B, dtype=cp.F8E4M3)
    finally:
        ctx.set_fp8_scales(1.0, 1.0)
    ref = 0.125 * oracle.gemm(N.e4m3_to_f64(A), N.e4m3_to_f64(B))
    assert N.rel_frobenius(got, ref) <= TOL_F32


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 40, 9), (128, 256, 64), (200, 300, 333),
                                   (256, 512, 1024)])
def test_fp8_on_f32_inputs(ctx, m, n, k):
    from gpu_util import assert_elementwise, elem_bound
    A = W.normal(m, k, seed=11 + m); B = W.normal(k, n, seed=12 + n)
    got = _run(ctx, 4, A, B)
    qa, sa = N.fp8_quantize(A); qb, sb = N.fp8_quantize(B)
    Aq, Bq = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb)
    exact_inputs = oracle.gemm(Aq, Bq) / (float(sa) * float(sb))
    assert N.rel_frobenius(got, exact_inputs) <= TOL_F32
    assert N.rel_frobenius(got, oracle.gemm(A, B)) <= 0.1
    absp = oracle.gemm(np.abs(Aq), np.abs(Bq)) / (float(sa) * float(sb))
    assert_elementwise(got, exact_inputs, absp, elem_bound(4, k))


@pytest.mark.parametrize("ea,eb", [(-120, 0), (-64, -64), (-140, 0)])
def test_fp8_on_tiny_f32_inputs(ctx, ea, eb):
    """Float32 operands far below 1 (A times 2^ea, B times 2^eb; 2^-140 is
    subnormal).  The per-tensor scales are capped at 2^126, where 448 / amax
    would overflow, and jointly reduced by powers of two so that the
    dequantisation 1 / (s_a s_b) stays a normal float32.  The result is finite,
    matches the oracle on the codes it multiplies element by element, and
    keeps FP8's usual accuracy while the operands are normal floats."""
    from gpu_util import assert_elementwise, elem_bound
    m, n, k = 96, 80, 256
    A = (W.uniform(m, k, seed=41) * np.float32(2.0 ** ea)).astype(np.float32)
    B = (W.uniform(k, n, seed=42) * np.float32(2.0 ** eb)).astype(np.float32)
    got = _run(ctx, 4, A, B)
    assert np.all(np.isfinite(got))
    qa, sa, qb, sb = N.fp8_quantize_pair(A, B)
    Aq, Bq = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb)
    d = float(sa) * float(sb)
    assert_elementwise(got, oracle.gemm(Aq, Bq) / d, oracle.gemm(np.abs(Aq), np.abs(Bq)) / d,
                       elem_bound(4, k))
    if ea > -126:   # operands in the normal range keep FP8's usual accuracy
        assert N.rel_frobenius(got, oracle.gemm(A, B)) <= 0.1


def test_non_finite_operands_stay_local(ctx):
    """An infinity and a NaN in A reach only their rows of C, in every
    variant.  The split variants give NaN there (inf - inf), and FP8
    encodes both as its NaN code after taking the scale over finite values.
    The other rows match the oracle: FP8's on the codes it multiplies."""
    import paper_2311_03543_b300 as cp
    from gpu_util import assert_elementwise, elem_bound
    m, n, k = 96, 80, 128
    A = W.uniform(m, k, seed=43); B = W.uniform(k, n, seed=44)
    A[5, 7], A[9, 2] = np.inf, np.nan
    ok_rows = np.setdiff1d(np.arange(m), [5, 9])
    Af = A.copy(); Af[5, 7] = Af[9, 2] = 0.0
    ref = oracle.gemm(Af, B)
    absp = oracle.gemm(np.abs(Af), np.abs(B))
    for v in (0, 1, 2, 3, 4, 5, 7, 8, 9):
        got = _run(ctx, v, A, B)
        assert not np.isfinite(got[[5, 9]]).any(), v
        assert np.isfinite(got[ok_rows]).all(), v
        if v == 4:
            qa, sa, qb, sb = N.fp8_quantize_pair(A, B)
            Aq, Bq = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb)
            d = float(sa) * float(sb)
            assert_elementwise(got[ok_rows], (oracle.gemm_rows(Aq, Bq, ok_rows)) / d,
                               oracle.gemm_rows(np.abs(Aq), np.abs(Bq), ok_rows) / d,
                               elem_bound(4, k))
        elif v == 3:
            Ar, Br = N.bf16_round(Af), N.bf16_round(B)
            assert_elementwise(got[ok_rows], oracle.gemm(Ar, Br)[ok_rows],
                               oracle.gemm(np.abs(Ar), np.abs(Br))[ok_rows], elem_bound(3, k))
        else:
            assert_elementwise(got[ok_rows], ref[ok_rows], absp[ok_rows], elem_bound(v, k))


def test_split3_matches_its_three_products(ctx):
    m, n, k = 192, 320, 512
    A = W.uniform(m, k, seed=13); B = W.uniform(k, n, seed=14)
    got = _run(ctx, 5, A, B)
    ah, al, bh, bl = N.split3_operands(A, B)
    three = oracle.gemm(ah, bh) + oracle.gemm(ah, bl) + oracle.gemm(al, bh)
    assert N.rel_frobenius(got, three) <= TOL_F32


@pytest.mark.parametrize("m,n,k", [(1, 4, 4), (3, 8, 12), (17, 40, 12), (33, 68, 20),
                                   (127, 132, 128), (128, 256, 64), (200, 300, 332),
                                   (300, 520, 1000), (2500, 2000, 1000), (16, 4096, 512)])
def test_fused_split_matches_split3_bitwise(ctx, m, n, k):
    """The fused variant splits in shared memory what the 3xBF16 pre-pass
    splits in global memory (same rounding), and issues the same products in
    the same order, tile decomposition and promotion: the results agree bit
    for bit, ragged edges, split K and stream-K tails included.  (It needs
    16-byte rows: N and K multiples of 4 for contiguous operands.)"""
    A = W.normal(m, k, seed=71)
    B = W.normal(k, n, seed=72)
    C0 = W.uniform(m, n, seed=73)
    got = _run(ctx, 9, A, B, alpha=0.75, beta=0.5, C0=C0)
    ref3 = _run(ctx, 5, A, B, alpha=0.75, beta=0.5, C0=C0)
    assert np.array_equal(got, ref3)
    assert N.rel_frobenius(got, oracle.gemm(A, B, alpha=0.75, beta=0.5, C0=C0)) <= TOL_F32


def test_fused_split_refuses_unaligned_operands(ctx):
    import torch
    import paper_2311_03543_b300 as cp
    m, n, k = 64, 64, 30                      # 120-byte rows of A
    A = torch.zeros((m, k), device="cuda")
    B = torch.zeros((k, n), device="cuda")
    C = torch.zeros((m, n), device="cuda")
    ctx.force_variant(cp.V_SPLIT3_FUSED)
    try:
        with pytest.raises(cp.ComparError):
            ctx.gemm(A, B, C)
    finally:
        ctx.force_variant(None)
    assert ctx.supported(cp.V_SPLIT3_FUSED, 64, 64, 32, cp.F32)
    assert not ctx.supported(cp.V_SPLIT3_FUSED, 64, 64, 30, cp.F32)


def test_split3_tf32_matches_its_three_products(ctx):
    import paper_2311_03543_b300 as cp
    m, n, k = 192, 320, 512
    A = W.normal(m, k, seed=44); B = W.normal(k, n, seed=45)
    got = _run(ctx, cp.V_SPLIT3_TF32, A, B)
    three = N.split3_tf32_product(A, B, oracle.gemm)
    assert N.rel_frobenius(got, three) <= TOL_SPLIT6


def test_split6_matches_its_six_products(ctx):
    m, n, k = 192, 320, 512
    A = W.normal(m, k, seed=23); B = W.normal(k, n, seed=24)
    got = _run(ctx, 7, A, B)
    six = N.split6_product(A, B, oracle.gemm)
    assert N.rel_frobenius(got, six) <= TOL_SPLIT6


@pytest.mark.parametrize("m,n,k", [(256, 512, 4096), (64, 128, 16384)])
def test_split6_at_simt_error_level(ctx, m, n, k):
    """Normal inputs at long K: the 6-product split stays within 2x of the
    FP32 SIMT variant's error (or below 1e-6) and well below 3xBF16's."""
    A = W.normal(m, k, seed=25); B = W.normal(k, n, seed=26)
    ref = oracle.gemm(A, B)
    e6 = N.rel_frobenius(_run(ctx, 7, A, B), ref)
    e1 = N.rel_frobenius(_run(ctx, 1, A, B), ref)
    e5 = N.rel_frobenius(_run(ctx, 5, A, B), ref)
    assert e6 <= max(2 * e1, 1e-6)
    assert e6 <= 0.5 * e5


@pytest.mark.parametrize("v", [0, 1, 2, 3, 4, 5, 7, 8, 9])
def test_all_ones_every_entry_is_k(ctx, v):
    m, n, k = 130, 260, 300
    got = _run(ctx, v, np.ones((m, k), np.float32), np.ones((k, n), np.float32))
    if v == 4:   # fp8 of float32 input: the dequantisation factor 1/448 is inexact
        assert np.allclose(got, k, rtol=1e-6, atol=0)
    else:
        assert np.all(got == k)


@pytest.mark.parametrize("v", [0, 1, 2, 3, 5, 7, 8, 9])
def test_identity_exact_on_representable_values(ctx, v):
    n = 192
    A = W.integer_matrix(n, n, seed=15)           # integers are exact in every format
    got = _run(ctx, v, A, np.eye(n, dtype=np.float32))
    assert np.array_equal(got, A)


@pytest.mark.parametrize("v", [0, 1, 2, 3, 4, 5, 7, 8])
def test_alpha_beta(ctx, v):
    m, n, k = 70, 90, 110
    A = W.integer_matrix(m, k, seed=16, bound=4)
    B = W.integer_matrix(k, n, seed=17, bound=4)
    C0 = W.integer_matrix(m, n, seed=18)
    got = _run(ctx, v, A, B, alpha=2.0, beta=-0.5, C0=C0)
    ref = oracle.gemm(A, B, alpha=2.0, beta=-0.5, C0=C0)
    tol = 1e-1 if v == 4 else TOL_F32   # fp8 quantises integers up to 16 exactly
    assert N.rel_frobenius(got, ref) <= tol


@pytest.mark.parametrize("v", [2, 3, 4, 5, 7, 8, 9])
def test_split_k_few_tiles_with_alpha_beta(ctx, v):
    """Few output tiles and a long K: the tensor-core variants split K over
    the SMs (partials reduced afterwards, beta applied once)."""
    m, n, k = 100, 300, 2048
    A = W.integer_matrix(m, k, seed=27, bound=2)
    B = W.integer_matrix(k, n, seed=28, bound=2)
    C0 = W.integer_matrix(m, n, seed=29)
    got = _run(ctx, v, A, B, alpha=2.0, beta=-0.5, C0=C0)
    ref = oracle.gemm(A, B, alpha=2.0, beta=-0.5, C0=C0)
    # small integers are exact in every format (fp8 scaling of 2 -> 448 too)
    tol = 1e-3 if v == 4 else TOL_F32
    assert N.rel_frobenius(got, ref) <= tol


_KELEMS = {2: 32, 3: 64, 4: 128, 5: 32, 9: 32}


@pytest.mark.parametrize("splits", [2, 3, 5, 7, 8, 12, 16])
@pytest.mark.parametrize("v", [2, 3, 4, 5, 9])
def test_k_split_summed_in_cluster(ctx, v, splits):
    """Four ragged tiles (200 x 300) with K = 8 * splits K blocks: the plan
    splits K `splits` ways and the splits of a tile, one thread-block cluster,
    add their accumulators through distributed shared memory (every slot of
    the tile shared out over the cluster's CTAs, odd cluster sizes included);
    12 and 16 splits take the HBM partials and the reduce kernel.
    Small integers are exact in every format, so a split counted twice or
    not at all, or a slot stored at the wrong element, changes the result."""
    import paper_2311_03543_b300 as cp
    m, n, k = 200, 300, _KELEMS[v] * 8 * splits
    assert cp.Context.tc_plan(v, m, n, k, 148)["splits"] == splits
    A = W.integer_matrix(m, k, seed=61, bound=2)
    B = W.integer_matrix(k, n, seed=62, bound=2)
    C0 = W.integer_matrix(m, n, seed=63)
    got = _run(ctx, v, A, B, alpha=2.0, beta=-0.5, C0=C0)
    ref = oracle.gemm(A, B, alpha=2.0, beta=-0.5, C0=C0)
    if v == 4:   # the fp8 scales of float32 inputs are not powers of two
        assert N.rel_frobenius(got, ref) <= 1e-3
    else:
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("v", [5, 9])
def test_k_split_in_cluster_normal_data(ctx, v):
    """The in-cluster K split on normal data (five splits): element by element
    within the variant's bound of the oracle."""
    from gpu_util import assert_elementwise, elem_bound
    m, n, k = 250, 500, 32 * 8 * 5
    A = W.normal(m, k, seed=64); B = W.normal(k, n, seed=65)
    got = _run(ctx, v, A, B)
    ref = oracle.gemm(A, B)
    assert N.rel_frobenius(got, ref) <= TOL_F32
    assert_elementwise(got, ref, oracle.gemm(np.abs(A), np.abs(B)), elem_bound(v, k))


@pytest.mark.parametrize("pairs", [0, 1])
@pytest.mark.parametrize("v", [2, 3, 4, 5, 7, 8, 9])
def test_partial_last_wave_with_alpha_beta(ctx, v, pairs):
    """180 tiles of 128 x 256 on 148 SMs (a partial second wave of the
    persistent CTAs, cut into stream-K pieces for the promoted variants), or
    90 tiles of 256 x 256 on 74 CTA pairs; integer inputs, alpha and beta."""
    import paper_2311_03543_b300 as cp
    if pairs and v not in (2, 3, 4, 5):
        pytest.skip("no pair kernel")
    m, n, k = 2560, 2304, 1024
    A = W.integer_matrix(m, k, seed=41, bound=2)
    B = W.integer_matrix(k, n, seed=42, bound=2)
    C0 = W.integer_matrix(m, n, seed=43)
    got = _run(ctx, v, A, B, alpha=2.0, beta=-0.5, C0=C0, pairs=pairs)
    ref = oracle.gemm(A, B, alpha=2.0, beta=-0.5, C0=C0)
    assert N.rel_frobenius(got, ref) <= TOL_F32


@pytest.mark.parametrize("pairs", [0, 1])
@pytest.mark.parametrize("v,m,n,k", [(5, 2500, 2000, 1000), (7, 2500, 2000, 1000),
                                     (8, 2500, 2000, 1000), (5, 1536, 2048, 4096),
                                     (7, 1400, 2048, 777), (9, 2500, 2000, 1000),
                                     (9, 1536, 2048, 4096), (5, 4096, 4096, 2048)])
def test_stream_k_tail_matches_oracle_and_is_deterministic(ctx, v, m, n, k, pairs):
    """A partial last wave of tiles (160 tiles: one full wave and 12 more) or
    a single partial wave (96 or 88 tiles) is cut into stream-K pieces of
    whole promotion chunks; 2 - 5 CTAs contribute to a tile and the last to
    finish adds the pieces in a fixed order.  Ragged M, N and K, alpha and
    beta; the same call twice gives the same bits.  With pairs (3xBF16),
    the tiles are 256 x 256 on 74 CTA pairs and each CTA of a pair publishes
    and sums its own rows of a tail tile."""
    if pairs and v != 5:
        pytest.skip("no pair kernel")
    A = W.uniform(m, k, seed=61)
    B = W.uniform(k, n, seed=62)
    C0 = W.uniform(m, n, seed=63)
    got = _run(ctx, v, A, B, alpha=1.5, beta=-0.25, C0=C0, pairs=pairs)
    again = _run(ctx, v, A, B, alpha=1.5, beta=-0.25, C0=C0, pairs=pairs)
    assert np.array_equal(got, again)
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    rows = W.tile_rows(m, seed=64)
    ref = oracle.gemm_rows(A, B, rows, alpha=1.5, beta=-0.25, C0=C0)
    assert N.rel_frobenius(got[rows], ref) <= (TOL_F32 if v in (5, 9) else TOL_SPLIT6)
    scale = 1.5 * abs_product_rows(A, B, rows) + 0.25 * np.abs(C0[rows])
    assert_elementwise(got[rows], ref, scale, elem_bound(v, k))


@pytest.mark.parametrize("pairs", [0, 1])
@pytest.mark.parametrize("v,tol,m,n,k", [(2, 2e-3, 2500, 2000, 4096), (2, 2e-3, 1536, 2048, 8192),
                                         (3, 5e-3, 2500, 2000, 4096), (3, 5e-3, 1536, 2048, 8192),
                                         (4, 6e-2, 2500, 2000, 8192)])
def test_stream_k_plain_variants(ctx, v, tol, m, n, k, pairs):
    """TF32, BF16 and FP8 (float32 inputs) with a stream-K tail: each piece
    is an accumulator of its own K range, published from TMEM; the result is
    within the variant's error level of the oracle and repeatable bit for
    bit."""
    A = W.uniform(m, k, seed=81)
    B = W.uniform(k, n, seed=82)
    C0 = W.uniform(m, n, seed=83)
    got = _run(ctx, v, A, B, alpha=1.25, beta=0.5, C0=C0, pairs=pairs)
    again = _run(ctx, v, A, B, alpha=1.25, beta=0.5, C0=C0, pairs=pairs)
    assert np.array_equal(got, again)
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    rows = W.tile_rows(m, seed=84)
    ref = oracle.gemm_rows(A, B, rows, alpha=1.25, beta=0.5, C0=C0)
    assert N.rel_frobenius(got[rows], ref) <= tol
    # against the float32 values: the format's rounding of each operand
    # (bf16 2^-9, e4m3 2^-4 plus the subnormal step 2^-10 / s, below
    # 2^-10 of amax here) on top of the accumulation bound
    fmt = {2: 0.0, 3: 2.0 ** -8 + 2.0 ** -18, 4: 2.0 ** -3 + 2.0 ** -6}[v]
    scale = 1.25 * abs_product_rows(A, B, rows) + 0.5 * np.abs(C0[rows])
    assert_elementwise(got[rows], ref, scale, fmt + elem_bound(v, k))


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_alpha_zero_reads_neither_a_nor_b(ctx, beta):
    """alpha == 0: C = beta * C and A and B are not read (BLAS convention), so
    NaNs and infinities in them do not reach C; also with a variant forced
    and through the batched call."""
    import torch
    import paper_2311_03543_b300 as cp
    m, n, k = 70, 90, 110
    A = W.uniform(m, k, seed=45); B = W.uniform(k, n, seed=46)
    A[3, 4], B[7, 8] = np.nan, np.inf
    C0 = W.uniform(m, n, seed=47)
    want = np.float32(beta) * C0 if beta != 0.0 else np.zeros_like(C0)
    for v in (None, 1, 5):
        got = _run(ctx, v, A, B, alpha=0.0, beta=beta,
                   C0=C0 if beta != 0.0 else np.full_like(C0, np.nan))
        assert np.array_equal(got, want), v
    from gpu_util import dev, host
    dA, dB, dC = dev(A), dev(B), dev(C0 if beta != 0.0 else np.full_like(C0, np.nan))
    probs = [dict(m=m, n=n, k=k, lda=k, ldb=n, ldc=n, dtype=cp.F32, A=dA.data_ptr(),
                  B=dB.data_ptr(), C=dC.data_ptr(), alpha=0.0, beta=beta)]
    ctx.gemm_batched(probs, tol=1e-5)
    assert np.array_equal(host(dC), want)


def test_k_zero_scales_c(ctx):
    from gpu_util import dev, host
    import torch
    C = dev(np.full((5, 6), 2.0, np.float32))
    ctx.set_scalars(1.0, 3.0)
    try:
        ctx.gemm(torch.zeros((5, 0), device="cuda"), torch.zeros((0, 6), device="cuda"), C)
    finally:
        ctx.set_scalars(1.0, 0.0)
    assert np.all(host(C) == 6.0)


def test_empty_m_or_n_is_a_no_op(ctx):
    import torch
    C = torch.zeros((0, 4), device="cuda")
    ctx.gemm(torch.zeros((0, 3), device="cuda"), torch.zeros((3, 4), device="cuda"), C)


def test_forced_unsupported_variant_is_refused(ctx):
    import paper_2311_03543_b300 as cp
    from gpu_util import dev, empty_c
    ctx.force_variant(cp.V_SPLIT3)
    try:
        with pytest.raises(cp.ComparError) as e:
            ctx.gemm(dev(W.bf16_input(8, 8, 1)), dev(W.bf16_input(8, 8, 2)), empty_c(8, 8),
                     dtype=cp.BF16)
        assert e.value.status == cp.ERR_UNSUPPORTED
    finally:
        ctx.force_variant(None)


@pytest.mark.parametrize("v,m,n,k", [(1, 4096, 4096, 64), (1, 16, 4096, 4096),
                                     (5, 4096, 4096, 64), (5, 16, 4096, 4096),
                                     (5, 2048, 2048, 2048), (1, 2048, 2048, 2048),
                                     (7, 2048, 2048, 2048), (7, 16, 4096, 4096),
                                     (7, 4096, 4096, 64), (8, 2048, 2048, 2048),
                                     (8, 16, 4096, 4096)])
def test_sweep_shapes_sampled_rows(ctx, v, m, n, k):
    """Full-size sweep shapes, checked against the oracle on the first and
    last row of every 128-row tile plus one seeded row inside it (every
    output tile holds a checked row), relative Frobenius and element by
    element."""
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    A = W.uniform(m, k, seed=20); B = W.uniform(k, n, seed=21)
    got = _run(ctx, v, A, B)
    rows = W.tile_rows(m, seed=22)
    ref = oracle.gemm_rows(A, B, rows)
    assert N.rel_frobenius(got[rows], ref) <= TOL_F32
    assert_elementwise(got[rows], ref, abs_product_rows(A, B, rows), elem_bound(v, k))
    assert np.all(np.isfinite(got))


def test_largest_sweep_shape_through_the_selector(ctx):
    """8192^3, the sweep's largest shape, through the selector at tol 1e-5 as
    the benchmark calls it (3xBF16 on CTA pairs): the first and last row of
    every 128-row tile plus one seeded row inside it, element by element."""
    import paper_2311_03543_b300 as cp
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    n = 8192
    A = W.uniform(n, n, seed=30); B = W.uniform(n, n, seed=31)
    got = _run(ctx, None, A, B, tol=1e-5)
    v = ctx.last_variant()
    assert v in (cp.V_SPLIT3, cp.V_SPLIT3_FUSED)
    rows = W.tile_rows(n, seed=32)
    ref = oracle.gemm_rows(A, B, rows)
    assert N.rel_frobenius(got[rows], ref) <= TOL_F32
    assert_elementwise(got[rows], ref, abs_product_rows(A, B, rows), elem_bound(v, n))
    assert np.all(np.isfinite(got))


# The SIMT variant's skinny-M plan (a few rows of A against a wide, deep B):
# every branch of the plan — clusters of 1, 2, 4 or 8 CTAs along K, their
# sums written straight to C or through the reduce pass — with 8- and 16-row
# groups and ragged rows, column blocks with idle threads, ragged K chunks,
# alpha and beta; the same call twice gives the same bits.
SKINNY = [(16, 512, 64), (5, 300, 20), (16, 16384, 1024), (64, 8192, 1024), (48, 65536, 1030),
          (64, 15360, 2048), (64, 8192, 4096), (33, 1000, 3000), (7, 4096, 4096)]


@pytest.mark.parametrize("m,n,k", SKINNY)
def test_simt_skinny_plan_matches_oracle_and_is_deterministic(ctx, m, n, k):
    import paper_2311_03543_b300 as cp
    assert cp.Context.simt_plan(m, n, k)["skinny"] == 1
    A = W.uniform(m, k, seed=71); B = W.uniform(k, n, seed=72); C0 = W.uniform(m, n, seed=73)
    got = _run(ctx, cp.V_SIMT, A, B, alpha=1.5, beta=-0.5, C0=C0)
    again = _run(ctx, cp.V_SIMT, A, B, alpha=1.5, beta=-0.5, C0=C0)
    assert np.array_equal(got, again)
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    rows = np.arange(m)
    ref = oracle.gemm_rows(A, B, rows, alpha=1.5, beta=-0.5, C0=C0)
    assert N.rel_frobenius(got[rows], ref) <= TOL_F32
    scale = 1.5 * abs_product_rows(A, B, rows) + 0.5 * np.abs(C0)
    assert_elementwise(got, ref, scale, elem_bound(1, k))


@pytest.mark.parametrize("m,n,k", [(16, 4096, 1000), (3, 1024, 333)])
def test_simt_skinny_plan_bf16_and_fp8_inputs(ctx, m, n, k):
    import paper_2311_03543_b300 as cp
    A = W.bf16_input(m, k, seed=75); B = W.bf16_input(k, n, seed=76)
    got = _run(ctx, cp.V_SIMT, A, B, dtype=cp.BF16)
    assert N.rel_frobenius(got, oracle.gemm(N.bf16_to_f32(A), N.bf16_to_f32(B))) <= TOL_F32
    A8 = W.fp8_input(m, k, seed=77); B8 = W.fp8_input(k, n, seed=78)
    ctx.set_fp8_scales(0.5, 0.25)
    try:
        got = _run(ctx, cp.V_SIMT, A8, B8, dtype=cp.F8E4M3)
    finally:
        ctx.set_fp8_scales(1.0, 1.0)
    ref = 0.125 * oracle.gemm(N.e4m3_to_f64(A8), N.e4m3_to_f64(B8))
    assert N.rel_frobenius(got, ref) <= TOL_F32


def test_simt_skinny_plan_unaligned_c_and_b(ctx):
    """C one element past a 16-byte boundary takes the scalar stores; B one
    element past it cannot be read 4 columns at a time and takes the tiled
    kernel.  Both still match the oracle."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import host
    m, n, k = 16, 1024, 700
    A = W.uniform(m, k, seed=79); B = W.uniform(k, n, seed=80); C0 = W.uniform(m, n, seed=81)
    ref = oracle.gemm(A, B, alpha=2.0, beta=0.5, C0=C0)
    dA = torch.from_numpy(A).cuda()
    bbuf = torch.zeros(k * n + 1, device="cuda")
    cbuf = torch.zeros(m * n + 1, device="cuda")
    for b_off, c_off in ((0, 1), (1, 0)):
        dB = bbuf[b_off:b_off + k * n].view(k, n)
        dB.copy_(torch.from_numpy(B))
        dC = cbuf[c_off:c_off + m * n].view(m, n)
        dC.copy_(torch.from_numpy(C0))
        ctx.set_scalars(2.0, 0.5)
        ctx.force_variant(cp.V_SIMT)
        try:
            ctx.gemm(dA, dB, dC)
        finally:
            ctx.force_variant(None)
            ctx.set_scalars(1.0, 0.0)
        assert ctx.check_device_error() == cp.OK
        assert N.rel_frobenius(host(dC), ref) <= TOL_F32


def test_simt_skinny_counters_carry_nothing_between_shapes(ctx):
    """The skinny plan's last-cluster slab sum counts arrivals in one word per
    (row group, column block) of the context's workspace.  Shapes of
    different grids and cluster counts run back to back on one context (the
    later grids cover the earlier ones' words), each checked against the
    oracle: a count left over from one call would make a later call sum
    unfinished slabs."""
    import paper_2311_03543_b300 as cp
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    seq = [(16, 4096, 4096), (64, 15360, 2048), (48, 4096, 2048), (16, 4096, 4096),
           (8, 227328, 1000), (64, 15360, 2048)]
    for i, (m, n, k) in enumerate(seq):
        plan = cp.Context.simt_plan(m, n, k)
        assert plan["skinny"] == 1 and 1 < plan["splits"] <= 8
        A = W.uniform(m, k, seed=300 + i); B = W.uniform(k, n, seed=400 + i)
        got = _run(ctx, cp.V_SIMT, A, B)
        rows = np.arange(m)
        ref = oracle.gemm_rows(A, B, rows)
        assert N.rel_frobenius(got, ref) <= TOL_F32, (m, n, k)
        assert_elementwise(got, ref, abs_product_rows(A, B, rows), elem_bound(1, k))


def test_simt_skinny_counters_recover_after_overlapping_calls(ctx):
    """Calls on one context must be ordered on the GPU; two that overlap (two
    streams, no ordering) give undefined results for themselves.  What must
    not happen is that their mixed-up arrival counts spoil later, ordered
    calls: every launch counts under its own epoch.  (The skinny kernel has
    no waits, so overlapping launches cannot block each other.)"""
    import torch
    import paper_2311_03543_b300 as cp
    m, n, k = 16, 4096, 4096
    A = W.uniform(m, k, seed=501); B = W.uniform(k, n, seed=502)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C1 = torch.empty((m, n), device="cuda"); C2 = torch.empty((m, n), device="cuda")
    ctx.force_variant(cp.V_SIMT)
    try:
        ctx.gemm(dA, dB, C1)                      # sizes the workspace first
        torch.cuda.synchronize()
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        for _ in range(8):
            with torch.cuda.stream(s1):
                ctx.gemm(dA, dB, C1)
            with torch.cuda.stream(s2):
                ctx.gemm(dA, dB, C2)
        torch.cuda.synchronize()
        C3 = torch.full((m, n), float("nan"), device="cuda")
        ctx.gemm(dA, dB, C3)
        torch.cuda.synchronize()
    finally:
        ctx.force_variant(None)
    assert ctx.check_device_error() == cp.OK
    assert N.rel_frobenius(C3.cpu().numpy(), oracle.gemm(A, B)) <= TOL_F32


# CTA pairs (cta_group::2): one 256 x 256 tile per pair of CTAs, each CTA
# holding half of A's rows and half of B's columns; tiles smaller than a
# pair's, ragged edges in M, N and K, a stream-K tail, alpha and beta.
PAIR_SHAPES = [(256, 256, 32), (300, 260, 100), (1000, 3000, 777), (2560, 2304, 1024),
               (4096, 4096, 512)]


@pytest.mark.parametrize("v", [2, 3, 4, 5])
@pytest.mark.parametrize("m,n,k", PAIR_SHAPES)
def test_pair_kernels_match_oracle(ctx, v, m, n, k):
    from gpu_util import abs_product_rows, assert_elementwise, elem_bound
    A = W.uniform(m, k, seed=91); B = W.uniform(k, n, seed=92); C0 = W.uniform(m, n, seed=93)
    got = _run(ctx, v, A, B, alpha=1.5, beta=-0.25, C0=C0, pairs=1)
    again = _run(ctx, v, A, B, alpha=1.5, beta=-0.25, C0=C0, pairs=1)
    assert np.array_equal(got, again)
    rows = W.tile_rows(m, seed=94)
    if v == 3:                      # against the product of the bf16 values multiplied
        Ae, Be, s = N.bf16_round(A).astype(np.float64), N.bf16_round(B).astype(np.float64), 1.0
    elif v == 4:                    # ... of the e4m3 codes, dequantised
        qa, sa = N.fp8_quantize(A); qb, sb = N.fp8_quantize(B)
        Ae, Be, s = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb), 1.0 / (float(sa) * float(sb))
    else:                           # TF32: total error; 3xBF16: FP32 accuracy
        Ae, Be, s = A.astype(np.float64), B.astype(np.float64), 1.0
    ref = oracle.gemm_rows(Ae, Be, rows, alpha=1.5 * s, beta=-0.25, C0=C0)
    scale = 1.5 * s * abs_product_rows(Ae, Be, rows) + 0.25 * np.abs(C0[rows])
    assert_elementwise(got[rows], ref, scale, elem_bound(v, k))
    if v == 5:
        exact = oracle.gemm_rows(A, B, rows, alpha=1.5, beta=-0.25, C0=C0)
        assert N.rel_frobenius(got[rows], exact) <= TOL_F32


def test_pairs_are_chosen_for_a_wave_of_tiles(ctx):
    """The automatic rule takes pairs from a full wave of 128 x 256 tiles up:
    at 2304^2 (162 tiles) the automatic call gives the bits of the forced
    pair call."""
    import paper_2311_03543_b300 as cp
    assert cp.Context.tc_plan(cp.V_SPLIT3, 2048, 2048, 2048)["tiles"] < 148
    assert cp.Context.tc_plan(cp.V_SPLIT3, 2304, 2304, 2304)["tiles"] >= 148
    m = n = 2304
    k = 512
    A = W.uniform(m, k, seed=95); B = W.uniform(k, n, seed=96)
    auto = _run(ctx, cp.V_SPLIT3, A, B, pairs=-1)
    forced = _run(ctx, cp.V_SPLIT3, A, B, pairs=1)
    assert np.array_equal(auto, forced)


@pytest.mark.parametrize("m,n,k", [(2560, 2304, 1024), (256, 512, 4096), (1024, 1024, 1024)])
def test_dependent_calls_back_to_back(ctx, m, n, k):
    """Calls enqueued with no synchronisation between them, each reading what
    the previous one wrote (C of one call is A of the next, then the C input
    with beta = 1): the tensor-core chain starts its pre-pass and GEMM
    set-up before the previous kernel completes, so this checks that no
    operand is read early and that no workspace is overwritten while a
    previous GEMM still reads it.  Shapes: a stream-K tail on CTA pairs, an
    in-cluster K split, and one wave of single CTAs."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev, host
    A0 = (W.uniform(m, k, seed=81) * 0.5).astype(np.float32)
    B0 = (W.uniform(k, k, seed=82) / np.sqrt(k)).astype(np.float32)
    B1 = (W.uniform(k, n, seed=83) / np.sqrt(k)).astype(np.float32)
    X = torch.empty((m, k), device="cuda")
    Y = torch.empty((m, n), device="cuda")
    dA0, dB0, dB1 = dev(A0), dev(B0), dev(B1)
    torch.cuda.synchronize()
    ctx.force_variant(cp.V_SPLIT3)
    try:
        ctx.gemm(dA0, dB0, X, tol=1e-5)          # X = A0 B0
        ctx.gemm(X, dB1, Y, tol=1e-5)            # Y = X B1 (reads X right after it is written)
        ctx.set_scalars(1.0, 1.0)
        ctx.gemm(X, dB1, Y, tol=1e-5)            # Y = X B1 + Y
        got = host(Y)
    finally:
        ctx.force_variant(None)
        ctx.set_scalars(1.0, 0.0)
    assert ctx.check_device_error() == cp.OK
    x = oracle.gemm(A0, B0)
    y = oracle.gemm(x, B1)
    ref = 2.0 * y
    assert N.rel_frobenius(got, ref) <= 3 * TOL_F32


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "e4m3"])
def test_operands_one_element_off_alignment(ctx, dt_name):
    """A, B and C each start one element past an aligned address (4, 2 or 1
    byte for A and B, 4 bytes for C): no 16-byte rows or bases, so TMA,
    vector loads and vector or bulk stores must all step aside.  Every
    variant the library accepts is forced in turn and matches the oracle
    element by element; one it cannot run on such operands refuses with
    COMPAR_ERR_UNSUPPORTED.  Then the selector's own pick."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import assert_elementwise, elem_bound
    m, n, k = 130, 203, 517
    if dt_name == "f32":
        A, B, dt = W.uniform(m, k, seed=61), W.uniform(k, n, seed=62), cp.F32
        Ax, Bx = A.astype(np.float64), B.astype(np.float64)
        tdt = torch.float32
    elif dt_name == "bf16":
        A, B, dt = W.bf16_input(m, k, seed=61), W.bf16_input(k, n, seed=62), cp.BF16
        Ax, Bx = N.bf16_to_f32(A).astype(np.float64), N.bf16_to_f32(B).astype(np.float64)
        tdt = torch.int16
    else:
        A, B, dt = W.fp8_input(m, k, seed=61), W.fp8_input(k, n, seed=62), cp.F8E4M3
        Ax, Bx = N.e4m3_to_f64(A), N.e4m3_to_f64(B)
        tdt = torch.uint8

    def off_by_one(x):     # a contiguous view one element past the allocation
        t = torch.empty(x.size + 1, dtype=tdt, device="cuda")[1:].view(x.shape)
        t.copy_(torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).cuda())
        return t
    dA, dB = off_by_one(A), off_by_one(B)
    assert dA.data_ptr() % 16 != 0 and dB.data_ptr() % 16 != 0
    ref = oracle.gemm(Ax, Bx)
    absp = oracle.gemm(np.abs(Ax), np.abs(Bx))
    ran = []
    for v in (None, 0, 1, 2, 3, 4, 5, 7, 8, 9):
        if v is not None and not ctx.supported(v, m, n, k, dt):
            continue
        C = torch.full((m * n + 1,), float("nan"), device="cuda")[1:].view(m, n)
        assert C.data_ptr() % 8 != 0
        ctx.force_variant(v)
        try:
            ctx.gemm(dA, dB, C, tol=1e-5, dtype=dt)
        except cp.ComparError as e:
            assert e.status == cp.ERR_UNSUPPORTED and v is not None, (v, e.status)
            continue
        finally:
            ctx.force_variant(None)
        used = ctx.last_variant() if v is None else v
        got = C.cpu().numpy()
        if dt == cp.F32 and used == 3:        # bf16 tensor cores multiply the roundings
            Ar, Br = N.bf16_round(A), N.bf16_round(B)
            assert_elementwise(got, oracle.gemm(Ar, Br), oracle.gemm(np.abs(Ar), np.abs(Br)),
                               elem_bound(3, k))
        elif dt == cp.F32 and used == 4:      # e4m3 with per-tensor scales
            qa, sa = N.fp8_quantize(A)
            qb, sb = N.fp8_quantize(B)
            Aq, Bq = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb)
            d = float(sa) * float(sb)
            assert_elementwise(got, oracle.gemm(Aq, Bq) / d, oracle.gemm(np.abs(Aq), np.abs(Bq)) / d,
                               elem_bound(4, k))
        else:
            assert_elementwise(got, ref, absp, elem_bound(used, k))
        ran.append(used)
    assert ctx.check_device_error() == cp.OK
    assert len(ran) >= 3, ran


@pytest.mark.parametrize("m,n,k", [(8, 24, 600000), (130, 40, 200000)])
def test_very_deep_k_many_splits(ctx, m, n, k):
    """A few outputs over a very deep K: the tensor-core plans split K 72 -
    148 ways (partial slabs and the reduce pass over them, batched 8 at a
    time) and SIMT 32 ways.  Every variant forced, and the selector's pick,
    element by element against the oracle."""
    import paper_2311_03543_b300 as cp
    from gpu_util import assert_elementwise, elem_bound
    A = W.uniform(m, k, seed=63); B = W.uniform(k, n, seed=64)
    ref = oracle.gemm(A, B)
    absp = oracle.gemm(np.abs(A), np.abs(B))
    for v in (None, 0, 1, 2, 3, 4, 5, 7, 8, 9):
        if v is not None and not ctx.supported(v, m, n, k, cp.F32):
            continue
        got = _run(ctx, v, A, B, tol=1e-5)
        used = ctx.last_variant() if v is None else v
        if used == 3:
            Ar, Br = N.bf16_round(A), N.bf16_round(B)
            assert_elementwise(got, oracle.gemm(Ar, Br), oracle.gemm(np.abs(Ar), np.abs(Br)),
                               elem_bound(3, k))
        elif used == 4:
            qa, sa = N.fp8_quantize(A)
            qb, sb = N.fp8_quantize(B)
            Aq, Bq = N.e4m3_to_f64(qa), N.e4m3_to_f64(qb)
            d = float(sa) * float(sb)
            assert_elementwise(got, oracle.gemm(Aq, Bq) / d,
                               oracle.gemm(np.abs(Aq), np.abs(Bq)) / d, elem_bound(4, k))
        else:
            assert_elementwise(got, ref, absp, elem_bound(used, k))
            if used in (1, 5, 7, 8, 9):        # FP32-accurate, split K shortens the chains
                assert N.rel_frobenius(got, ref) <= TOL_F32, (used, N.rel_frobenius(got, ref))


def test_output_beyond_two_to_the_31_elements(ctx):
    """C of 46341 x 46344 (2.15e9 elements, 8.6 GB: offsets past 2^31) with
    K = 3: the selector's pick and the SIMT, TF32, BF16 and 3xBF16 variants
    forced.  Rows sampled per 128-row tile (the last ones included) against
    the oracle, element by element."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import assert_elementwise, elem_bound
    m, n, k = 46341, 46344, 3
    assert m * n > 2 ** 31
    A = W.uniform(m, k, seed=65); B = W.uniform(k, n, seed=66)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    rows = W.tile_rows(m, seed=67)
    rows = np.unique(np.concatenate([rows, [m - 1]]))
    ref = oracle.gemm_rows(A, B, rows)
    absp = oracle.gemm_rows(np.abs(A), np.abs(B), rows)
    C = torch.empty((m, n), device="cuda")
    for v in (None, 1, 2, 3, 5):
        C.fill_(float("nan"))
        ctx.force_variant(v)
        try:
            ctx.gemm(dA, dB, C, tol=1e-5)
        finally:
            ctx.force_variant(None)
        used = ctx.last_variant() if v is None else v
        got = C[torch.from_numpy(rows).cuda()].cpu().numpy()
        if used == 3:
            Ar, Br = N.bf16_round(A), N.bf16_round(B)
            assert_elementwise(got, oracle.gemm_rows(Ar, Br, rows),
                               oracle.gemm_rows(np.abs(Ar), np.abs(Br), rows), elem_bound(3, k))
        else:
            assert_elementwise(got, ref, absp, elem_bound(used, k))
        assert not torch.isnan(C[-1]).any()
    del C
    torch.cuda.empty_cache()
    assert ctx.check_device_error() == cp.OK


def test_recording_skips_captured_calls():
    """With timing records on, a call captured into a graph records nothing
    (its events would belong to the graph), and the eager calls around it are
    recorded, run the same variant and match the oracle; nothing is
    quarantined."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev, host
    m, n, k = 1024, 768, 512
    A = W.uniform(m, k, seed=97); B = W.uniform(k, n, seed=98)
    ref = oracle.gemm(A, B)
    dA, dB = dev(A), dev(B)
    C = torch.empty((m, n), device="cuda")
    with cp.Context(0) as c:
        c.record_enable(True)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            c.gemm(dA, dB, C, tol=1e-5, stream=s)             # decision and workspace
        s.synchronize()
        v = c.last_variant()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            c.gemm(dA, dB, C, tol=1e-5, stream=s)
        for _ in range(2):
            C.fill_(float("nan"))
            g.replay()
            assert N.rel_frobenius(host(C), ref) <= TOL_F32
        C.fill_(float("nan"))
        c.gemm(dA, dB, C, tol=1e-5)
        assert c.last_variant() == v
        assert N.rel_frobenius(host(C), ref) <= TOL_F32
        recs = c.records()
        assert len(recs) == 2 and all(r.variant == v and r.time_ms > 0 for r in recs)
        c.clear_decisions()
        assert c.select(m, n, k, cp.F32, 1e-5) == v
        assert c.check_device_error() == cp.OK


@pytest.mark.parametrize("m,n,k", [(2560, 2304, 1024), (16, 4096, 4096), (1024, 1024, 1024)])
def test_captured_call_replays(ctx, m, n, k):
    """A call captured into a CUDA graph (after one call of the shape outside
    the capture) and replayed three times gives the oracle's result every
    time: the counter words of a stream-K tail (first shape) or of the
    skinny plan's cluster sums (second, forced SIMT) start from zero on each
    replay, and in-cluster K splits (third) need none."""
    import torch
    import paper_2311_03543_b300 as cp
    from gpu_util import dev, host
    A = W.uniform(m, k, seed=95); B = W.uniform(k, n, seed=96)
    ref = oracle.gemm(A, B)
    dA, dB = dev(A), dev(B)
    C = torch.empty((m, n), device="cuda")
    v = cp.V_SIMT if m == 16 else cp.V_SPLIT3
    ctx.force_variant(v)
    try:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            ctx.gemm(dA, dB, C, tol=1e-5, stream=s)        # decision and workspace
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctx.gemm(dA, dB, C, tol=1e-5, stream=s)
        for _ in range(3):
            C.fill_(float("nan"))
            g.replay()
            got = host(C)
            assert N.rel_frobenius(got, ref) <= TOL_F32
    finally:
        ctx.force_variant(None)
    assert ctx.check_device_error() == cp.OK
