"""Pins for the oracle's number-format definitions (CPU only).

bf16 and E4M3 conversions are checked against PyTorch's CPU conversions (an
independent library routine) and against values fixed by the format
definitions; the split and the error metric against exact identities.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import numerics as N


def _torch_bf16_bits(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def test_bf16_matches_library_on_random_values():
    x = np.concatenate([W.uniform(1, 100000, seed=1).ravel(),
                        W.normal(1, 100000, seed=2).ravel() * 1e20,
                        W.normal(1, 100000, seed=3).ravel() * 1e-30])
    assert np.array_equal(N.bf16_bits(x), _torch_bf16_bits(x))


def test_bf16_ties_go_to_even():
    # kept pattern even -> stays; odd -> rounds up
    even = np.array([0x3F800000 | 0x8000], np.uint32).view(np.float32)   # 1.0 + half ulp
    odd = np.array([0x3F810000 | 0x8000], np.uint32).view(np.float32)
    assert N.bf16_bits(even)[0] == 0x3F80
    assert N.bf16_bits(odd)[0] == 0x3F82
    assert np.array_equal(N.bf16_bits(np.concatenate([even, odd])),
                          _torch_bf16_bits(np.concatenate([even, odd])))


def test_bf16_identity_on_representable():
    bits = W.bf16_input(64, 64, seed=4)
    assert np.array_equal(N.bf16_bits(N.bf16_to_f32(bits)), bits)


def test_e4m3_table_fixed_points():
    assert N.e4m3_to_f64(np.uint8(0x7E)) == 448.0          # largest finite
    assert N.e4m3_to_f64(np.uint8(0x01)) == 2.0 ** -9       # smallest subnormal
    assert N.e4m3_to_f64(np.uint8(0x08)) == 2.0 ** -6       # smallest normal
    assert N.e4m3_to_f64(np.uint8(0x38)) == 1.0
    assert N.e4m3_to_f64(np.uint8(0xB8)) == -1.0
    assert np.isnan(N.e4m3_to_f64(np.uint8(0x7F)))
    assert np.isnan(N.e4m3_to_f64(np.uint8(0xFF)))
    vals = N.e4m3_to_f64(np.arange(0x7F, dtype=np.uint8))
    assert np.all(np.diff(vals) > 0)                        # monotone code order


def test_e4m3_round_trip_all_finite_codes():
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], np.uint8)
    vals = N.e4m3_to_f64(codes).astype(np.float32)
    assert np.array_equal(N.e4m3_codes(vals), codes)


def test_e4m3_matches_library_in_range():
    x = np.concatenate([W.uniform(1, 200000, seed=5, lo=-447.0, hi=447.0).ravel(),
                        W.normal(1, 100000, seed=6).ravel(),
                        W.normal(1, 100000, seed=7).ravel() * 1e-3])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(N.e4m3_codes(x), ref)


def test_e4m3_ties_and_saturation():
    # midpoint of 1.0 (0x38) and 1.125 (0x39) -> even code 0x38;
    # midpoint of 1.125 and 1.25 (0x3A) -> 0x3A
    assert N.e4m3_codes(np.float32(1.0625)) == 0x38
    assert N.e4m3_codes(np.float32(1.1875)) == 0x3A
    assert N.e4m3_codes(np.float32(1000.0)) == 0x7E
    assert N.e4m3_codes(np.float32(-1e6)) == 0xFE
    assert N.e4m3_codes(np.float32(2.0 ** -10)) == 0x00     # half the smallest subnormal
    assert N.e4m3_codes(np.float32(-0.0)) == 0x80


def test_fp8_quantize_scale_and_amax():
    x = W.uniform(32, 32, seed=8)
    x[3, 5] = -4.0                       # amax a power of two -> s exact
    codes, s = N.fp8_quantize(x)
    assert s == np.float32(112.0)
    assert codes[3, 5] == 0xFE           # -448
    assert np.all(np.abs(N.e4m3_to_f64(codes)) <= 448)
    zc, zs = N.fp8_quantize(np.zeros((4, 4), np.float32))
    assert zs == 1.0 and np.all(zc == 0)


def test_fp8_scale_is_capped_for_tiny_tensors():
    # amax = 2^-120: 448 / amax = 2^128.8 overflows float32; the cap gives
    # s = 2^126, so x * s <= 64 and the largest code is exactly 64
    x = W.uniform(16, 16, seed=10) * np.float32(2.0 ** -121)
    x[2, 3] = np.float32(2.0 ** -120)
    codes, s = N.fp8_quantize(x)
    assert s == np.float32(2.0 ** 126)
    assert N.e4m3_to_f64(codes)[2, 3] == 64.0
    assert np.float32(1.0) / s == np.float32(2.0 ** -126)   # a normal float32
    # a subnormal amax: still the cap, and every code finite
    y = np.full((4, 4), np.float32(2.0 ** -130), np.float32)
    cy, sy = N.fp8_quantize(y)
    assert sy == np.float32(2.0 ** 126) and np.all(np.isfinite(N.e4m3_to_f64(cy)))
    # below the cap the rule is unchanged: amax = 2^-117 gives 448 * 2^117 < 2^126
    z = np.full((2, 2), np.float32(2.0 ** -117), np.float32)
    assert N.fp8_scale(z) == np.float32(448.0 * 2.0 ** 117)


def test_fp8_pair_scales():
    a = W.uniform(16, 16, seed=11)
    b = W.uniform(16, 16, seed=12)
    # ordinary data: the pair rule changes nothing
    assert N.fp8_scales_pair(a, b) == (N.fp8_scale(a), N.fp8_scale(b))
    for ea, eb in [(-120, 0), (-64, -64), (-140, -10), (0, -126)]:
        A, B = a * np.float32(2.0 ** ea), b * np.float32(2.0 ** eb)
        sa, sb = N.fp8_scales_pair(A, B)
        # the dequantisation of the product stays a normal float32
        assert 1.0 / (float(sa) * float(sb)) >= 2.0 ** -126
        # each scale is its own scale divided by a power of two, split evenly
        ra = float(N.fp8_scale(A)) / float(sa)
        rb = float(N.fp8_scale(B)) / float(sb)
        assert ra == 2.0 ** round(np.log2(ra)) and rb == 2.0 ** round(np.log2(rb))
        assert 0 <= np.log2(ra) - np.log2(rb) <= 1
    # the worked case: A at 2^-120 (scale capped at 2^126), B ordinary
    sa, sb = N.fp8_scales_pair(a * np.float32(2.0 ** -120), b)
    assert sa == np.float32(2.0 ** 121) and sb == np.float32(N.fp8_scale(b) / 32)


def test_fp8_quantize_non_finite_values():
    x = W.uniform(8, 8, seed=13)
    x[1, 1] = -4.0                       # the largest finite magnitude
    y = x.copy()
    y[2, 5], y[6, 0], y[7, 7] = np.inf, -np.inf, np.nan
    cx, sx = N.fp8_quantize(x)
    cy, sy = N.fp8_quantize(y)
    assert sy == sx == np.float32(112.0)  # non-finite values leave amax alone
    bad = ~np.isfinite(y)
    assert np.all(cy[bad] == 0x7F) and np.all(np.isnan(N.e4m3_to_f64(cy[bad])))
    assert np.array_equal(cy[~bad], cx[~bad])


def test_fp8_quantize_exact_multiples_round_trip():
    codes = W.fp8_input(16, 16, seed=9)
    vals = N.e4m3_to_f64(codes)
    s = np.float32(4.0)
    x = (vals / s).astype(np.float32)    # exact multiples of 1/s
    got = N.e4m3_codes((x * s).astype(np.float32))
    nz = vals != 0
    assert np.array_equal(got[nz], codes[nz])


def test_split_exact_for_16_bit_significands():
    # values with at most 16 significant bits are exactly hi + lo
    x = W.uniform(64, 64, seed=10)
    x16 = (x.view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)
    hi, lo = N.split_bf16(x16)
    recon = N.bf16_to_f32(hi).astype(np.float64) + N.bf16_to_f32(lo).astype(np.float64)
    assert np.array_equal(recon, x16.astype(np.float64))


def test_split_residual_bound():
    x = W.normal(128, 128, seed=11)
    hi, lo = N.split_bf16(x)
    recon = N.bf16_to_f32(hi).astype(np.float64) + N.bf16_to_f32(lo).astype(np.float64)
    err = np.abs(recon - x.astype(np.float64))
    # hi leaves a residual below 2^-8|x|; rounding that residual to 8 bits
    # leaves at most 2^-9 of it: total <= 2^-17 |x|
    assert np.all(err <= 2.0 ** -17 * np.abs(x.astype(np.float64)))


def test_three_piece_split_is_exact_for_24_bit_significands():
    # every float32 has 24 significant bits: hi + mid + lo reproduces it
    # exactly unless the exponent range of the pieces runs out (not for
    # moderate magnitudes)
    x = np.concatenate([W.uniform(1, 5000, seed=12).ravel(), W.normal(1, 5000, seed=13).ravel()])
    hi, mid, lo = N.split_bf16_3(x)
    recon = sum(N.bf16_to_f32(p).astype(np.float64) for p in (hi, mid, lo))
    assert np.array_equal(recon, x.astype(np.float64))


def test_three_piece_split_pieces_shrink():
    x = W.normal(64, 64, seed=14)
    hi, mid, lo = N.split_bf16_3(x)
    h, m, l = (np.abs(N.bf16_to_f32(p).astype(np.float64)) for p in (hi, mid, lo))
    ax = np.abs(x.astype(np.float64))
    assert np.all(m <= 2.0 ** -8 * ax + 1e-45)
    assert np.all(l <= 2.0 ** -16 * ax + 1e-45)


def test_split6_product_on_exact_pieces():
    # matrices whose entries are exact bf16 values: mid = lo = 0 and the
    # 6-product sum is the plain product
    import oracle
    A = N.bf16_to_f32(W.bf16_input(7, 9, seed=15)).astype(np.float32)
    B = N.bf16_to_f32(W.bf16_input(9, 5, seed=16)).astype(np.float32)
    got = N.split6_product(A, B, oracle.gemm)
    assert np.array_equal(got, oracle.gemm(A, B))


def _tf32_by_fractions(v):
    """Nearest value with 11 significant bits, ties away from zero (exact
    rational arithmetic; normal float32 values)."""
    from fractions import Fraction
    import math
    f = Fraction(float(v))
    if f == 0:
        return 0.0
    e = math.floor(math.log2(abs(float(v))))
    unit = Fraction(2) ** (e - 10)          # spacing of 11-bit significands
    q = abs(f) / unit
    n = math.floor(q)
    if q - n >= Fraction(1, 2):
        n += 1
    return float(math.copysign(float(n * unit), float(v)))


def test_tf32_round_matches_exact_rounding():
    x = np.concatenate([W.uniform(1, 2000, seed=17).ravel(), W.normal(1, 2000, seed=18).ravel()])
    got = N.tf32_round(x)
    want = np.array([_tf32_by_fractions(v) for v in x], np.float64)
    assert np.array_equal(got.astype(np.float64), want)


def test_tf32_ties_away_and_exact_values():
    one_half_ulp = np.float32(1.0 + 2.0 ** -11)          # halfway between 1 and 1 + 2^-10
    assert N.tf32_round(one_half_ulp) == np.float32(1.0 + 2.0 ** -10)
    assert N.tf32_round(-one_half_ulp) == np.float32(-(1.0 + 2.0 ** -10))
    exact = np.float32(1.0 + 2.0 ** -10 + 2.0 ** -9)   # 11 significant bits
    assert N.tf32_round(exact) == exact
    assert N.tf32_round(np.float32(0.0)) == 0.0


def test_tf32_split_reconstructs_22_bit_values():
    x = W.uniform(64, 64, seed=19)
    x22 = (x.view(np.uint32) & np.uint32(0xFFFFFFFC)).view(np.float32)   # 22 significant bits
    hi, lo = N.split_tf32(x22)
    assert np.array_equal(hi.astype(np.float64) + lo.astype(np.float64), x22.astype(np.float64))
    hi, lo = N.split_tf32(x)
    err = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - x.astype(np.float64))
    assert np.all(err <= 2.0 ** -21 * np.abs(x.astype(np.float64)))


def test_rel_frobenius_closed_forms():
    a = np.array([[3.0, 4.0]])
    assert N.rel_frobenius(a, a) == 0.0
    assert N.rel_frobenius(np.zeros((1, 2)), a) == 1.0
    assert N.rel_frobenius(2 * a, a) == 1.0
    assert N.rel_frobenius(a + np.array([[0.0, 0.5]]), a) == pytest.approx(0.1)
    assert N.rel_frobenius(np.zeros(3), np.zeros(3)) == 0.0


# ------------------------------------------------------------------------------
# The product compositions of the split methods, pinned by exact arithmetic.
#
# Each operand entry is built from pieces chosen first (random mantissas and
# exponents, the pieces' bit ranges disjoint and every piece away from a
# rounding boundary), so the split is known without calling the split code,
# and every one of the piece products has a different size.  The method's
# product is then fixed by a rule stated apart from the oracle's list of
# terms: keep the products whose piece orders (hi 0, mid 1, lo 2) add up to
# at most the number of pieces minus one.  Exact rational sums decide
# equality, so replacing, dropping or transposing any one term fails.

def _pieces(rows, cols, seed, offsets, sigs):
    """Matrices of pieces p_0 > p_1 > ... and their exact sum (float32).

    Piece j of an entry has sigs[j] significant bits, a mantissa strictly
    between 1 and 2 - 2^-(sigs[j]-1) (never a power of two, never the
    largest mantissa) and exponent e - offsets[j] (e in [-3, 3]).  The
    offsets put every piece below half the spacing of the piece before it
    (strictly, with the rest added), so rounding the sum to the first
    piece's width gives the first piece back, rounding what remains gives
    the second, and so on; and the widths keep the sum within float32's 24
    significant bits.  Signs are independent per piece.
    """
    r = np.random.default_rng(seed)
    e = r.integers(-3, 4, size=(rows, cols))
    out = []
    for off, sig in zip(offsets, sigs):
        scale = 2 ** (sig - 1)
        mant = r.integers(scale + 1, 2 * scale - 1, size=(rows, cols))     # m / 2^(sig-1)
        sign = r.choice([-1, 1], size=(rows, cols))
        out.append(sign * mant.astype(np.float64) * np.exp2((e - off - (sig - 1)).astype(np.float64)))
    total = sum(out)
    f32 = total.astype(np.float32)
    assert np.array_equal(f32.astype(np.float64), total)     # the sum is exact in float32
    return f32, out


def _exact_matmul(X, Y):
    from fractions import Fraction
    m, k = X.shape
    n = Y.shape[1]
    Xf = [[Fraction(float(v)) for v in row] for row in X]
    Yf = [[Fraction(float(v)) for v in row] for row in Y]
    return [[sum((Xf[i][p] * Yf[p][j] for p in range(k)), Fraction(0)) for j in range(n)]
            for i in range(m)]


def _as_fractions(C):
    from fractions import Fraction
    return [[Fraction(float(v)) for v in row] for row in np.asarray(C, np.float64)]


def _add(*mats):
    return [[sum(vals) for vals in zip(*rows)] for rows in zip(*mats)]


def _sub(X, Y):
    return [[a - b for a, b in zip(rx, ry)] for rx, ry in zip(X, Y)]


def _kept_by_order_rule(pa, pb):
    """Sum of the piece products whose orders add up to <= len(pa) - 1."""
    n = len(pa)
    terms = [_exact_matmul(pa[i], pb[j]) for i in range(n) for j in range(n) if i + j <= n - 1]
    dropped = [_exact_matmul(pa[i], pb[j]) for i in range(n) for j in range(n) if i + j > n - 1]
    return _add(*terms), _add(*dropped), len(terms), len(dropped)


def _all_products_distinct(pa, pb):
    n = len(pa)
    prods = {(i, j): _exact_matmul(pa[i], pb[j]) for i in range(n) for j in range(n)}
    keys = list(prods)
    for x in range(len(keys)):
        for y in range(x + 1, len(keys)):
            assert prods[keys[x]] != prods[keys[y]], (keys[x], keys[y])
    for key, P in prods.items():                          # and no product is its own transpose
        assert all(v != 0 for row in P for v in row), key


def test_split6_product_is_exactly_the_six_leading_piece_products():
    import oracle
    # bf16 pieces: hi and mid 8 significant bits, lo 6, each 9 binades below the last
    A, pa = _pieces(5, 7, seed=31, offsets=(0, 9, 18), sigs=(8, 8, 6))
    B, pb = _pieces(7, 4, seed=32, offsets=(0, 9, 18), sigs=(8, 8, 6))
    # the oracle's split returns the chosen pieces
    for X, px in ((A, pa), (B, pb)):
        got = [N.bf16_to_f32(p).astype(np.float64) for p in N.split_bf16_3(X)]
        for g, want in zip(got, px):
            assert np.array_equal(g, want)
    _all_products_distinct(pa, pb)
    kept, dropped, nk, nd = _kept_by_order_rule(pa, pb)
    assert (nk, nd) == (6, 3)
    got = _as_fractions(N.split6_product(A, B, oracle.gemm))
    assert got == kept
    # the three dropped products are exactly what separates it from A*B
    assert _sub(_exact_matmul(A, B), got) == dropped


def test_split3_tf32_product_is_exactly_the_three_leading_piece_products():
    import oracle
    # TF32 pieces: 11 significant bits each, lo 12 binades below hi
    A, pa = _pieces(6, 5, seed=33, offsets=(0, 12), sigs=(11, 11))
    B, pb = _pieces(5, 3, seed=34, offsets=(0, 12), sigs=(11, 11))
    for X, px in ((A, pa), (B, pb)):
        got = [p.astype(np.float64) for p in N.split_tf32(X)]
        for g, want in zip(got, px):
            assert np.array_equal(g, want)
    _all_products_distinct(pa, pb)
    kept, dropped, nk, nd = _kept_by_order_rule(pa, pb)
    assert (nk, nd) == (3, 1)
    got = _as_fractions(N.split3_tf32_product(A, B, oracle.gemm))
    assert got == kept
    assert _sub(_exact_matmul(A, B), got) == dropped


def test_split3_operands_give_the_three_leading_bf16_piece_products():
    # the 2-piece bf16 split's three products (the 3xBF16 variant's sum)
    import oracle
    A, pa = _pieces(4, 6, seed=35, offsets=(0, 9), sigs=(8, 8))
    B, pb = _pieces(6, 5, seed=36, offsets=(0, 9), sigs=(8, 8))
    ah, al, bh, bl = N.split3_operands(A, B)
    for g, want in zip((ah, al, bh, bl), (pa[0], pa[1], pb[0], pb[1])):
        assert np.array_equal(g, want)
    kept, dropped, nk, nd = _kept_by_order_rule(pa, pb)
    got = _as_fractions(oracle.gemm(ah, bh) + oracle.gemm(ah, bl) + oracle.gemm(al, bh))
    assert got == kept and (nk, nd) == (3, 1)


def _abs_product(A, B):
    import oracle
    return oracle.gemm(np.abs(A.astype(np.float64)), np.abs(B.astype(np.float64)))


def test_split6_product_error_bound_on_float32_data():
    # |mid| <= 2^-8 |x| and |lo| <= 2^-16 |x| (test_three_piece_split_pieces_shrink),
    # hi + mid + lo = x exactly, so the dropped mid*lo + lo*mid + lo*lo is at
    # most (2^-23 + 2^-32) |a||b| per product; the float64 sums add K 2^-53.
    import oracle
    for seed, (m, n, k) in ((41, (33, 29, 300)), (42, (16, 64, 1024))):
        A = W.normal(m, k, seed=seed)
        B = W.uniform(k, n, seed=seed + 100)
        exact = oracle.gemm(A, B)
        s6 = N.split6_product(A, B, oracle.gemm)
        bound = (2.0 ** -23 + 2.0 ** -32 + 4 * k * 2.0 ** -53) * _abs_product(A, B)
        assert np.all(np.abs(s6 - exact) <= bound)
        # and it is closer to A*B than the two-piece, three-product split
        ah, al, bh, bl = N.split3_operands(A, B)
        s3 = oracle.gemm(ah, bh) + oracle.gemm(ah, bl) + oracle.gemm(al, bh)
        assert N.rel_frobenius(s6, exact) < N.rel_frobenius(s3, exact) / 100


def test_split3_tf32_product_error_bound_on_float32_data():
    # a = hi + lo + r with |r| <= 2^-22 |a| and |lo| <= 2^-11 |a| (rounding to
    # 11 significant bits twice), so a*b - kept = lo_a lo_b + r_a b + (hi_b + lo_b) r_b... is at
    # most about 3 * 2^-22 |a||b|
    import oracle
    for seed, (m, n, k) in ((43, (31, 17, 500)), (44, (8, 40, 2048))):
        A = W.uniform(m, k, seed=seed)
        B = W.normal(k, n, seed=seed + 100)
        exact = oracle.gemm(A, B)
        s3 = N.split3_tf32_product(A, B, oracle.gemm)
        bound = (3.01 * 2.0 ** -22 + 4 * k * 2.0 ** -53) * _abs_product(A, B)
        assert np.all(np.abs(s3 - exact) <= bound)
        one = oracle.gemm(N.tf32_round(A), N.tf32_round(B))   # the plain TF32 product
        assert N.rel_frobenius(s3, exact) < N.rel_frobenius(one, exact) / 100
