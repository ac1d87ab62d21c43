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
